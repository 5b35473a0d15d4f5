// Dense nonsymmetric eigensolver for the sketched Rayleigh-Ritz matrix
// M-hat (d x d, FP64, d <= 232): Algorithm 2's "solve eigenvalue problem"
// step, written for one GPU.
//
//   1. Householder reduction to upper Hessenberg form H = P^T M P (an 8-CTA
//      cluster; reflectors kept below the subdiagonal).
//   2. Eigenvalues of H by the implicit double-shift QR iteration (Golub &
//      Van Loan, Algorithms 7.5.1 and 7.5.2), eigenvalues only, run by one
//      warp on H packed by columns in shared memory (francis_kernel).
//   3. Eigenvectors for the selected eigenvalues by inverse iteration on the
//      Hessenberg matrix, (H - lambda I) y = y_prev in complex arithmetic with
//      partial pivoting between adjacent rows (one CTA per eigenvalue), then
//      back-transformed with the Householder reflectors of step 1.
#include <cmath>
#include <cooperative_groups.h>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace sk {

static constexpr int kEigMaxN = 256;  // per-CTA work arrays of the reduction and inverse iteration
static constexpr int kEigThreads = 256;

__device__ __forceinline__ double block_sum_d(double v, double* sh) {
  v = warp_sum(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double a = 0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) a += sh[w];
  return a;
}

// ---- 1. Hessenberg reduction (in place, global memory, ld = n) ---------------------
// On an 8-CTA cluster: the FP64 updates of a step are spread over 8 SMs (one
// SM's FP64 rate bounded a one-CTA reduction at ~11 ms for n = 200).  Step
// k: every CTA forms the reflector of column k itself (same loads, same
// fixed-order sum, so the same bits everywhere); CTA q owns the columns j with
// j % 8 == q and applies the left update to them alone; for the right update
// each CTA sums H[:, j] v_j over its columns, the eight partial vectors are
// read through distributed shared memory and added in rank order, and each
// CTA updates its columns; a second cluster barrier publishes column k + 1.
static constexpr int kHessCluster = 8;

__global__ void __launch_bounds__(kEigThreads)
hessenberg_cluster_kernel(double* __restrict__ H, int n, double* __restrict__ tau) {
  cg::cluster_group cluster = cg::this_cluster();
  const int q = (int)cluster.block_rank();
  __shared__ double sh[32];
  __shared__ double v[kEigMaxN];
  __shared__ double wpart[kEigMaxN];  // this CTA's sum of H[:, j] v_j over its columns
  __shared__ double s_sc[3];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  cluster.sync();  // every CTA of the cluster has started before the first remote read
  for (int k = 0; k + 2 < n; ++k) {
    // reflector for x = H[k+1:n, k] (v in shared memory, v_i for i >= k+1)
    double part = 0;
    for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) {
      const double x = __ldcg(H + i + (int64_t)k * n);
      v[i] = x;
      part += x * x;
    }
    const double nrm2 = block_sum_d(part, sh);
    if (threadIdx.x == 0) {
      const double x0 = v[k + 1];
      const double nrm = sqrt(nrm2);
      const double alpha = x0 >= 0 ? -nrm : nrm;
      const double v0 = x0 - alpha;
      const double vtv = nrm2 - x0 * x0 + v0 * v0;
      s_sc[0] = vtv > 0 ? 2.0 / vtv : 0.0;
      s_sc[1] = alpha;
      s_sc[2] = v0;
      v[k + 1] = v0;
    }
    __syncthreads();
    const double t = s_sc[0];
    // this CTA's first column right of k
    const int j0 = k + 1 + ((q - (k + 1)) % kHessCluster + kHessCluster) % kHessCluster;
    // left: H[k+1:, j] -= t v (v^T H[k+1:, j]) for this CTA's columns, a warp per column
    for (int j = j0 + wid * kHessCluster; j < n; j += nw * kHessCluster) {
      double* col = H + (int64_t)j * n;
      double a = 0;
      for (int i = k + 1 + lane; i < n; i += 32) a += v[i] * col[i];
      a = warp_sum(a) * t;
      for (int i = k + 1 + lane; i < n; i += 32) col[i] -= v[i] * a;
    }
    __syncthreads();  // this CTA's left-updated columns, before its own sums read them
    // right: w = t H[:, k+1:] v; this CTA's part over its columns, every row
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      double a[4] = {0, 0, 0, 0};  // four independent chains (FP64 FMA latency)
      int u = 0;
      for (int j = j0; j < n; j += kHessCluster, u = (u + 1) & 3) a[u] += H[i + (int64_t)j * n] * v[j];
      wpart[i] = (a[0] + a[1]) + (a[2] + a[3]);
    }
    cluster.sync();  // every CTA's partial sums (and left updates) are complete
    const double* wp[kHessCluster];
#pragma unroll
    for (int r = 0; r < kHessCluster; ++r) wp[r] = cluster.map_shared_rank(wpart, r);
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      double a = 0;
#pragma unroll
      for (int r = 0; r < kHessCluster; ++r) a += wp[r][i];
      const double wi = a * t;
      for (int j = j0; j < n; j += kHessCluster) H[i + (int64_t)j * n] -= wi * v[j];
    }
    if (q == 0 && threadIdx.x == 0) {
      H[k + 1 + (int64_t)k * n] = v[k + 1];  // v_0 (v kept in H[k+1:, k]); every CTA has read column k
      tau[k] = t;
      tau[n + k] = s_sc[1];  // subdiagonal entry H[k+1, k]
    }
    cluster.sync();  // right updates done (column k + 1 among them); wpart is free again
  }
}

// ---- 2. Eigenvalues of H by the implicit double-shift QR iteration ---------------------
// Written from the description of the Francis QR step and of the practical
// QR algorithm in Golub & Van Loan, "Matrix Computations" (4th ed.),
// Algorithms 7.5.1 and 7.5.2: the shifts are the two eigenvalues of the
// trailing 2 x 2 block of the active window, entered implicitly through the
// first column of (H - a I)(H - b I) = H^2 - s H + t I (s = a + b, t = a b),
// and the bulge they create is chased down the subdiagonal with 3 x 3
// Householder reflectors; a subdiagonal entry below eps (|h_{l,l}| +
// |h_{l-1,l-1}|) is set to zero and splits the problem; 1 x 1 and 2 x 2
// blocks at the bottom of the window give eigenvalues.  Eigenvalues only:
// the reflectors touch the active window's rows and columns, nothing else.
//
// One CTA does the whole iteration (the work split is described at
// francis_kernel).  H lives in shared memory, packed by columns: column j
// keeps rows 0 .. min(j + 3, n - 1), which holds the Hessenberg part and the
// bulge.
static constexpr int kFrancisMaxN = 232;  // packed storage of n = 232 fills 221.7 KB

__host__ __device__ inline int francis_col_len(int j, int n) { return (j + 4 < n) ? j + 4 : n; }

size_t francis_smem_bytes(int n) {
  size_t o = 0;
  for (int j = 0; j < n; ++j) o += (size_t)francis_col_len(j, n);
  return o * sizeof(double) + (size_t)(n + 1) * sizeof(int);
}

struct PackedH {
  double* a;
  const int* off;
  __device__ __forceinline__ double& at(int i, int j) const { return a[off[j] + i]; }
};

// Householder reflector for (x, y, z): v = (x - alpha, y, z) with alpha =
// -sign(x) ||(x, y, z)||, returned scaled so that the reflector is I - v v^T
// (v^T v = 2); v = 0 (the identity) for a zero vector.  The input is scaled
// by a power of two (exact, from the exponent bits) so that squaring neither
// overflows nor underflows.  Branch-free, so the compiler can interleave
// this dependent FP64 chain with independent updates.
__device__ __forceinline__ void house3(double x, double y, double z, double& alpha, double& v0, double& v1,
                                       double& v2) {
  const double m = fmax(fabs(x), fmax(fabs(y), fabs(z)));
  int ex = (int)((__double_as_longlong(m) >> 52) & 0x7ff);
  ex = min(max(ex, 1), 2045);
  const double sc = __longlong_as_double((long long)(2046 - ex) << 52);  // 2^(1023 - ex)
  const double isc = __longlong_as_double((long long)ex << 52);          // 2^(ex - 1023)
  const double xs = x * sc, ys = y * sc, zs = z * sc;
  const double nrm = sqrt(xs * xs + ys * ys + zs * zs);
  const double as = (xs >= 0.0) ? -nrm : nrm;
  const bool nz = m > 0.0;
  // w = (xs - as, ys, zs), w^T w = 2 nrm (nrm + |xs|); v = w sqrt(2 / w^T w)
  const double f = nz ? rsqrt(nrm * (nrm + fabs(xs))) : 0.0;
  alpha = as * isc;
  v0 = (xs - as) * f;
  v1 = ys * f;
  v2 = zs * f;
}

// One CTA of kFrancisWarps warps; warp 0 is the chain warp.  Each SM
// sub-partition has its own FP64 unit (on this GPU a warp's FP64
// instruction issues once per 64 cycles on its sub-partition), so the far
// updates of a bulge step go to the other warps, in parallel with warp 0's
// near updates and the next reflector's dependent chain.  Bulge step k, with
// reflector k acting on rows k..k+2 and columns k..k+2:
//   near(k), warp 0: rows k..k+2 of columns c0..k+3 (c0 = k, or lo for the
//     first step), then rows k..k+3 of columns k..k+2; then reflector k+1
//     from rows k+1..k+3 of column k;
//   far(k), other warps: rows k..k+2 of columns k+4..hi, rows lo..k-1 of
//     columns k..k+2.
// near(k) and far(k) touch disjoint entries, far(k) reads nothing near(k)
// writes, and near(k) reads far(k-1)'s results only after the barrier that
// opens step k, so every entry sees the updates of the plain
// row-then-column order, in that order.
static constexpr int kFrancisWarps = 4;
static constexpr int kFrancisThreads = 32 * kFrancisWarps;

__global__ void __launch_bounds__(kFrancisThreads)
francis_kernel(const double* __restrict__ Hg, const double* __restrict__ tau, int n, double* __restrict__ wr,
               double* __restrict__ wi, int* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char fr_smem[];
  __shared__ double s_ref[2][4];  // reflector (alpha, v0, v1, v2) of steps of each parity
  __shared__ double s_norm[kFrancisWarps];
  __shared__ int s_lo;
  int* off = reinterpret_cast<int*>(fr_smem);
  double* a = reinterpret_cast<double*>(fr_smem + (((size_t)(n + 1) * sizeof(int) + 15) & ~(size_t)15));
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ftid = tid - 32, nft = kFrancisThreads - 32;  // far threads
  const unsigned full = 0xffffffffu;
  if (tid == 0) {
    int o = 0;
    for (int j = 0; j < n; ++j) { off[j] = o; o += francis_col_len(j, n); }
    off[n] = o;
  }
  __syncthreads();
  const PackedH H{a, off};
  // the Hessenberg matrix (subdiagonal from tau[n + j]), zero below it
  double nrm_part = 0;
  for (int j = tid; j < n; j += kFrancisThreads) {
    const int len = francis_col_len(j, n);
    for (int i = 0; i < len; ++i) {
      double v = 0;
      if (i <= j) v = Hg[i + (int64_t)j * n];
      else if (i == j + 1) v = (j + 2 < n) ? tau[n + j] : Hg[i + (int64_t)j * n];
      H.at(i, j) = v;
      nrm_part += fabs(v);
    }
  }
  nrm_part = warp_sum(nrm_part);
  if (lane == 0) s_norm[warp] = nrm_part;
  __syncthreads();
  double hnorm = 0;
  for (int w = 0; w < kFrancisWarps; ++w) hnorm += s_norm[w];
  const double eps = 2.220446049250313e-16;
  int hi = n - 1, its = 0, total = 0, fail = 0;
  const int max_total = 40 * n;
  while (hi >= 0) {
    // lo: the largest l <= hi whose subdiagonal entry is negligible (0 if none)
    if (warp == 0) {
      int lo = 0;
      for (int base = hi; base >= 1; base -= 32) {
        const int l = base - lane;
        bool small = false;
        if (l >= 1) {
          double sz = fabs(H.at(l, l)) + fabs(H.at(l - 1, l - 1));
          if (sz == 0.0) sz = hnorm;
          small = fabs(H.at(l, l - 1)) <= eps * sz;
        }
        const unsigned m = __ballot_sync(full, small);
        if (m) {
          lo = base - (__ffs(m) - 1);
          break;
        }
      }
      if (lane == 0) {
        if (lo > 0) H.at(lo, lo - 1) = 0.0;
        s_lo = lo;
      }
    }
    __syncthreads();
    const int lo = s_lo;
    if (lo == hi) {
      if (tid == 0) { wr[hi] = H.at(hi, hi); wi[hi] = 0.0; }
      hi -= 1;
      its = 0;
      __syncthreads();
      continue;
    }
    if (lo == hi - 1) {
      // eigenvalues of the 2 x 2 block [[p, q], [r, u]]: mean +- sqrt(disc)
      if (tid == 0) {
        const double p = H.at(lo, lo), q = H.at(lo, hi), r = H.at(hi, lo), u = H.at(hi, hi);
        const double mean = 0.5 * (p + u), half = 0.5 * (p - u);
        const double disc = half * half + q * r;
        if (disc >= 0.0) {
          const double rt = sqrt(disc);
          const double big = mean + (mean >= 0.0 ? rt : -rt);  // no cancellation
          const double det = p * u - q * r;
          wr[lo] = big;
          wr[hi] = (big != 0.0) ? det / big : mean - rt;
          wi[lo] = wi[hi] = 0.0;
        } else {
          const double im = sqrt(-disc);
          wr[lo] = wr[hi] = mean;
          wi[lo] = im;
          wi[hi] = -im;
        }
      }
      hi -= 2;
      its = 0;
      __syncthreads();
      continue;
    }
    if (total >= max_total) {
      fail = 1;
      break;
    }
    ++its;
    ++total;
    if (warp == 0) {
      // shifts: the trailing 2 x 2 block of the window (s = trace, t = det);
      // every 10th iteration without a deflation, a double shift at
      // h_hi,hi + 1.5 |h_hi,hi-1| instead (breaks cycles of the standard shift)
      double s, t;
      const int m = hi - 1;
      if (its % 10 == 0) {
        const double mu = H.at(hi, hi) + 1.5 * fabs(H.at(hi, m));
        s = 2.0 * mu;
        t = mu * mu;
      } else {
        s = H.at(m, m) + H.at(hi, hi);
        t = H.at(m, m) * H.at(hi, hi) - H.at(m, hi) * H.at(hi, m);
      }
      // first column of H^2 - s H + t I on the window
      const double x0 = H.at(lo, lo) * H.at(lo, lo) + H.at(lo, lo + 1) * H.at(lo + 1, lo) - s * H.at(lo, lo) + t;
      const double y0 = H.at(lo + 1, lo) * (H.at(lo, lo) + H.at(lo + 1, lo + 1) - s);
      const double z0 = H.at(lo + 1, lo) * H.at(lo + 2, lo + 1);
      double al, u0, u1, u2;
      house3(x0, y0, z0, al, u0, u1, u2);
      if (lane == 0) {
        s_ref[lo & 1][0] = al;
        s_ref[lo & 1][1] = u0;
        s_ref[lo & 1][2] = u1;
        s_ref[lo & 1][3] = u2;
      }
    }
    for (int k = lo; k <= hi - 2; ++k) {
      __syncthreads();  // reflector k published; far(k - 1) done
      const double alpha = s_ref[k & 1][0], v0 = s_ref[k & 1][1], v1 = s_ref[k & 1][2], v2 = s_ref[k & 1][3];
      if (warp == 0) {
        if (k > lo && lane == 0) {
          H.at(k, k - 1) = alpha;  // column k-1, rows k..k+2 -> (alpha, 0, 0)
          H.at(k + 1, k - 1) = 0.0;
          H.at(k + 2, k - 1) = 0.0;
        }
        const int c = ((k > lo) ? k : lo) + lane;
        if (lane < 4 && c <= min(k + 3, hi)) {
          const double h0 = H.at(k, c), h1 = H.at(k + 1, c), h2 = H.at(k + 2, c);
          const double w = v0 * h0 + v1 * h1 + v2 * h2;
          H.at(k, c) = h0 - w * v0;
          H.at(k + 1, c) = h1 - w * v1;
          H.at(k + 2, c) = h2 - w * v2;
        }
        __syncwarp();
        const int r = k + lane;
        if (lane < 4 && r <= min(k + 3, hi)) {
          const double h0 = H.at(r, k), h1 = H.at(r, k + 1), h2 = H.at(r, k + 2);
          const double w = h0 * v0 + h1 * v1 + h2 * v2;
          H.at(r, k) = h0 - w * v0;
          H.at(r, k + 1) = h1 - w * v1;
          H.at(r, k + 2) = h2 - w * v2;
        }
        __syncwarp();
        // the next reflector (the last one of the sweep has two entries)
        const double xn = H.at(k + 1, k), yn = H.at(k + 2, k), zn = (k < hi - 2) ? H.at(k + 3, k) : 0.0;
        double an, u0, u1, u2;
        house3(xn, yn, zn, an, u0, u1, u2);
        if (lane == 0) {
          s_ref[(k + 1) & 1][0] = an;
          s_ref[(k + 1) & 1][1] = u0;
          s_ref[(k + 1) & 1][2] = u1;
          s_ref[(k + 1) & 1][3] = u2;
        }
      } else {
        for (int c = k + 4 + ftid; c <= hi; c += nft) {
          const double h0 = H.at(k, c), h1 = H.at(k + 1, c), h2 = H.at(k + 2, c);
          const double w = v0 * h0 + v1 * h1 + v2 * h2;
          H.at(k, c) = h0 - w * v0;
          H.at(k + 1, c) = h1 - w * v1;
          H.at(k + 2, c) = h2 - w * v2;
        }
        for (int r = lo + ftid; r <= k - 1; r += nft) {
          const double h0 = H.at(r, k), h1 = H.at(r, k + 1), h2 = H.at(r, k + 2);
          const double w = h0 * v0 + h1 * v1 + h2 * v2;
          H.at(r, k) = h0 - w * v0;
          H.at(r, k + 1) = h1 - w * v1;
          H.at(r, k + 2) = h2 - w * v2;
        }
      }
    }
    __syncthreads();
    // the last reflector (two entries, v2 = 0) acts on rows hi-1, hi
    {
      const int k = hi - 1;
      const double alpha = s_ref[k & 1][0], v0 = s_ref[k & 1][1], v1 = s_ref[k & 1][2];
      if (k > lo && tid == 0) {
        H.at(k, k - 1) = alpha;
        H.at(k + 1, k - 1) = 0.0;
      }
      const int c0 = (k > lo) ? k : lo;
      for (int c = c0 + tid; c <= hi; c += kFrancisThreads) {
        const double h0 = H.at(k, c), h1 = H.at(k + 1, c);
        const double w = v0 * h0 + v1 * h1;
        H.at(k, c) = h0 - w * v0;
        H.at(k + 1, c) = h1 - w * v1;
      }
      __syncthreads();
      for (int r = lo + tid; r <= hi; r += kFrancisThreads) {
        const double h0 = H.at(r, k), h1 = H.at(r, k + 1);
        const double w = h0 * v0 + h1 * v1;
        H.at(r, k) = h0 - w * v0;
        H.at(r, k + 1) = h1 - w * v1;
      }
      __syncthreads();
    }
  }
  if (tid == 0) *status = fail;
}


// ---- selection: nev eigenvalues of largest real part (ties: larger imaginary
// part, then index) ----------------------------------------------------------------------
__global__ void select_kernel(const double* __restrict__ wr, const double* __restrict__ wi, int n, int nev,
                              int* __restrict__ sel) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int used[kEigMaxN];
  for (int i = 0; i < n; ++i) used[i] = 0;
  for (int t = 0; t < nev; ++t) {
    int best = -1;
    for (int i = 0; i < n; ++i) {
      if (used[i]) continue;
      if (best < 0 || wr[i] > wr[best] || (wr[i] == wr[best] && (wi[i] > wi[best] || (wi[i] == wi[best] && i < best))))
        best = i;
    }
    used[best] = 1;
    sel[t] = best;
  }
}

// ---- 3. inverse iteration on H (complex), back-transform ----------------------------
// One CTA per selected eigenvalue.  W: per-CTA workspace of n*n complex
// (re, im planes) for the LU of H - lambda I.
__global__ void __launch_bounds__(kEigThreads)
invit_kernel(const double* __restrict__ Hg, const double* __restrict__ tau, int n, const double* __restrict__ wr,
             const double* __restrict__ wi, const int* __restrict__ sel, double* __restrict__ Wre,
             double* __restrict__ Wim, double* __restrict__ Yre, double* __restrict__ Yim) {
  __shared__ double yr[kEigMaxN], yi[kEigMaxN];
  __shared__ int piv[kEigMaxN];
  __shared__ double lre[kEigMaxN], lim[kEigMaxN];
  __shared__ double sh[32];
  const int t = blockIdx.x;
  const int e = sel[t];
  const double lr = wr[e], li = wi[e];
  double* Ur = Wre + (int64_t)t * n * n;
  double* Ui = Wim + (int64_t)t * n * n;
  // U = H - lambda I (Hessenberg: rows i <= j+1)
  for (int q = threadIdx.x; q < n * n; q += blockDim.x) {
    const int j = q / n, i = q % n;
    double a = 0;
    if (i <= j) a = Hg[i + (int64_t)j * n];
    else if (i == j + 1) a = (j + 2 < n) ? tau[n + j] : Hg[i + (int64_t)j * n];
    Ur[q] = a - (i == j ? lr : 0.0);
    Ui[q] = (i == j ? -li : 0.0);
  }
  __syncthreads();
  // Hessenberg LU with partial pivoting between rows j and j+1; an exactly
  // zero pivot (lambda an exact eigenvalue) is replaced by 1e-14 max|U|
  double eps_u = 0;
  {
    double m = 0;
    for (int q = threadIdx.x; q < n * n; q += blockDim.x) m = fmax(m, fabs(Ur[q]) + fabs(Ui[q]));
    for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
    __syncthreads();
    m = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, sh[w]);
    eps_u = m * 1e-14;
  }
  __syncthreads();
  for (int j = 0; j + 1 < n; ++j) {
    if (threadIdx.x == 0) {
      const double ar = Ur[j + (int64_t)j * n], ai = Ui[j + (int64_t)j * n];
      const double br = Ur[j + 1 + (int64_t)j * n], bi = Ui[j + 1 + (int64_t)j * n];
      piv[j] = (br * br + bi * bi > ar * ar + ai * ai) ? 1 : 0;
    }
    __syncthreads();
    if (piv[j]) {
      for (int c = j + threadIdx.x; c < n; c += blockDim.x) {
        const int64_t a0 = j + (int64_t)c * n, a1 = j + 1 + (int64_t)c * n;
        double tr = Ur[a0], ti = Ui[a0];
        Ur[a0] = Ur[a1]; Ui[a0] = Ui[a1];
        Ur[a1] = tr; Ui[a1] = ti;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double pr = Ur[j + (int64_t)j * n], pi = Ui[j + (int64_t)j * n];
      if (pr * pr + pi * pi == 0.0) { pr = eps_u; Ur[j + (int64_t)j * n] = pr; }
      const double br = Ur[j + 1 + (int64_t)j * n], bi = Ui[j + 1 + (int64_t)j * n];
      const double den = pr * pr + pi * pi;
      lre[j] = (br * pr + bi * pi) / den;  // l = b / p
      lim[j] = (bi * pr - br * pi) / den;
    }
    __syncthreads();
    const double mr = lre[j], mi = lim[j];
    for (int c = j + 1 + threadIdx.x; c < n; c += blockDim.x) {
      const int64_t a0 = j + (int64_t)c * n, a1 = j + 1 + (int64_t)c * n;
      const double ur = Ur[a0], ui = Ui[a0];
      Ur[a1] -= mr * ur - mi * ui;
      Ui[a1] -= mr * ui + mi * ur;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const int64_t d0 = (n - 1) + (int64_t)(n - 1) * n;
    if (Ur[d0] * Ur[d0] + Ui[d0] * Ui[d0] == 0.0) Ur[d0] = eps_u;
  }
  // start vector: entries in [0.5, 1.5) from the counter hash of (t, i), so
  // that copies of a repeated eigenvalue start from different vectors and
  // return independent vectors of its eigenspace
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const uint64_t h = mix64(0x5851F42D4C957F2Dull * (uint64_t)(t + 1) + (uint64_t)i);
    yr[i] = 0.5 + (double)(h >> 11) * (1.0 / 9007199254740992.0);
    yi[i] = 0.0;
  }
  __syncthreads();
  for (int iter = 0; iter < 3; ++iter) {
    // forward: apply the row swaps and multipliers
    if (threadIdx.x == 0) {
      for (int j = 0; j + 1 < n; ++j) {
        if (piv[j]) { double a = yr[j]; yr[j] = yr[j + 1]; yr[j + 1] = a; a = yi[j]; yi[j] = yi[j + 1]; yi[j + 1] = a; }
        yr[j + 1] -= lre[j] * yr[j] - lim[j] * yi[j];
        yi[j + 1] -= lre[j] * yi[j] + lim[j] * yr[j];
      }
    }
    __syncthreads();
    // back substitution with U (column sweep)
    for (int j = n - 1; j >= 0; --j) {
      __shared__ double s_r, s_i;
      if (threadIdx.x == 0) {
        const double ur = Ur[j + (int64_t)j * n], ui = Ui[j + (int64_t)j * n];
        const double den = ur * ur + ui * ui;
        const double xr = (yr[j] * ur + yi[j] * ui) / den;
        const double xi = (yi[j] * ur - yr[j] * ui) / den;
        yr[j] = xr; yi[j] = xi;
        s_r = xr; s_i = xi;
      }
      __syncthreads();
      const double xr = s_r, xi = s_i;
      for (int i = threadIdx.x; i < j; i += blockDim.x) {
        const double ur = Ur[i + (int64_t)j * n], ui = Ui[i + (int64_t)j * n];
        yr[i] -= ur * xr - ui * xi;
        yi[i] -= ur * xi + ui * xr;
      }
      __syncthreads();
    }
    // normalise
    double part = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) part += yr[i] * yr[i] + yi[i] * yi[i];
    const double nrm = sqrt(block_sum_d(part, sh));
    for (int i = threadIdx.x; i < n; i += blockDim.x) { yr[i] /= nrm; yi[i] /= nrm; }
    __syncthreads();
  }
  // back-transform: y <- P_0 P_1 ... P_{n-3} y, P_k = I - tau_k v_k v_k^T on rows k+1..
  for (int k = n - 3; k >= 0; --k) {
    const double tk = tau[k];
    const double* v = Hg + (int64_t)k * n;  // v[i], i >= k+1 (v_0 stored at row k+1)
    double pr = 0, pi = 0;
    for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) { pr += v[i] * yr[i]; pi += v[i] * yi[i]; }
    const double sr = block_sum_d(pr, sh);
    const double si = block_sum_d(pi, sh);
    __syncthreads();
    for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) { yr[i] -= tk * sr * v[i]; yi[i] -= tk * si * v[i]; }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    Yre[(int64_t)t * n + i] = yr[i];
    Yim[(int64_t)t * n + i] = yi[i];
  }
}

// M (n x n, col-major, overwritten), outputs: wr, wi (n), sel (nev), Yre/Yim
// (n x nev col-major), status (device int; 1 = QR iteration did not converge).
sk_status enqueue_eig(double* M, int n, int nev, double* tau, double* wr, double* wi, int* sel, double* Wre,
                      double* Wim, double* Yre, double* Yim, int* status, cudaStream_t st) {
  if (n > kFrancisMaxN || n < 3) { set_error("eigensolver supports 3 <= d <= %d", kFrancisMaxN); return SK_EINVAL; }
  {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kHessCluster);
    cfg.blockDim = dim3(kEigThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kHessCluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    SK_CUDA(cudaLaunchKernelEx(&cfg, hessenberg_cluster_kernel, M, n, tau));
  }
  // one attribute value for every launch (graph capture keeps launch sizes)
  SK_CUDA(cudaFuncSetAttribute(francis_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)francis_smem_bytes(kFrancisMaxN) + 16));
  francis_kernel<<<1, kFrancisThreads, francis_smem_bytes(n) + 16, st>>>(M, tau, n, wr, wi, status);
  SK_CUDA(cudaGetLastError());
  select_kernel<<<1, 1, 0, st>>>(wr, wi, n, nev, sel);
  SK_CUDA(cudaGetLastError());
  invit_kernel<<<nev, kEigThreads, 0, st>>>(M, tau, n, wr, wi, sel, Wre, Wim, Yre, Yim);
  SK_CUDA(cudaGetLastError());
  return SK_OK;
}

}  // namespace sk
