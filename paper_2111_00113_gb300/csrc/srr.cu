// Sketched Rayleigh-Ritz after the sketches: Algorithm 2's reduction
// (§6.3-§6.4) and the stabilized form of §6.5 (eq. (qz)), Ritz vectors and
// residual estimates; sRR on a caller's basis; restarted sRR on block
// Chebyshev bases (§7.2, §7.5).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "dense.cuh"
#include "srr.cuh"

namespace sk {

static constexpr int kSrrThreads = 256;

static int grid_for(int64_t n, int threads, int cap) {
  int64_t g = (n + threads - 1) / threads;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

// M-hat = T^{-1} (U^T D): column c of the D block (rows 0..d-1 after the QR)
// solved against the triangle (one CTA per column, column sweep).
__global__ void __launch_bounds__(256)
mhat_kernel(const double* __restrict__ Aug, const double* __restrict__ rdiag, int s, int d,
            double* __restrict__ Mhat) {
  __shared__ double z[kMaxSrrD];
  __shared__ double s_y;
  const int c = blockIdx.x;
  const double* Dc = Aug + (int64_t)(d + c) * s;
  for (int i = threadIdx.x; i < d; i += blockDim.x) z[i] = Dc[i];
  __syncthreads();
  for (int i = d - 1; i >= 0; --i) {
    if (threadIdx.x == 0) { s_y = z[i] / rdiag[i]; z[i] = s_y; }
    __syncthreads();
    const double yi = s_y;
    const double* Ri = Aug + (int64_t)i * s;
    for (int t = threadIdx.x; t < i; t += blockDim.x) z[t] -= yi * Ri[t];
    __syncthreads();
  }
  for (int i = threadIdx.x; i < d; i += blockDim.x) Mhat[i + (int64_t)c * d] = z[i];
}

// Residual estimate (eq. (srr-resid-est)) of selected pair t, computed in the
// rotated basis after the QR: ||Q^T D y - lambda [T y; 0]|| / ||T y||.
__global__ void __launch_bounds__(256)
srr_resid_kernel(const double* __restrict__ Aug, const double* __restrict__ rdiag, int s, int d,
                 const double* __restrict__ wr, const double* __restrict__ wi, const int* __restrict__ sel,
                 const double* __restrict__ Yre, const double* __restrict__ Yim, int symmetric,
                 double* __restrict__ out /* nev x 3: lam_re, lam_im, rhat */) {
  __shared__ double yr[kMaxSrrD], yi[kMaxSrrD];
  __shared__ double sh[32];
  const int t = blockIdx.x;
  const int e = sel[t];
  const double lr = wr[e], li = symmetric ? 0.0 : wi[e];
  for (int j = threadIdx.x; j < d; j += blockDim.x) {
    yr[j] = Yre[(int64_t)t * d + j];
    yi[j] = symmetric ? 0.0 : Yim[(int64_t)t * d + j];
  }
  __syncthreads();
  double num = 0, den = 0;
  for (int r = threadIdx.x; r < s; r += blockDim.x) {
    double vr = 0, vi = 0, ur = 0, ui = 0;
    for (int j = 0; j < d; ++j) {
      const double dq = Aug[(int64_t)(d + j) * s + r];
      vr += dq * yr[j];
      vi += dq * yi[j];
      if (r < d && j >= r) {
        const double tq = (j == r) ? rdiag[r] : Aug[(int64_t)j * s + r];
        ur += tq * yr[j];
        ui += tq * yi[j];
      }
    }
    const double rr = vr - (lr * ur - li * ui);
    const double ri = vi - (lr * ui + li * ur);
    num += rr * rr + ri * ri;
    den += ur * ur + ui * ui;
  }
  num = warp_sum(num);
  den = warp_sum(den);
  __shared__ double s2[32];
  if ((threadIdx.x & 31) == 0) { sh[threadIdx.x >> 5] = num; s2[threadIdx.x >> 5] = den; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, b = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { a += sh[w]; b += s2[w]; }
    out[t * 3 + 0] = lr;
    out[t * 3 + 1] = li;
    out[t * 3 + 2] = sqrt(a) / sqrt(b);
  }
}

// X = B Y for the selected pairs (complex), one pass over B; per-CTA partial
// squared norms of each column for the normalisation.
template <typename T>
__global__ void __launch_bounds__(256)
ritz_kernel(const T* __restrict__ B, int64_t ldb, int64_t n, int d, int nev, const double* __restrict__ Yre,
            const double* __restrict__ Yim, int symmetric, double* __restrict__ Xre, double* __restrict__ Xim,
            double* __restrict__ part) {
  extern __shared__ double ys[];  // 2 * nev * d
  __shared__ double sh[kMaxNev * 2 * 8];
  for (int q = threadIdx.x; q < nev * d; q += blockDim.x) {
    ys[q] = Yre[q];
    ys[nev * d + q] = symmetric ? 0.0 : Yim[q];
  }
  __syncthreads();
  double nrm[kMaxNev];
  for (int t = 0; t < nev; ++t) nrm[t] = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double ar[kMaxNev], ai[kMaxNev];
    for (int t = 0; t < nev; ++t) { ar[t] = 0; ai[t] = 0; }
    for (int j = 0; j < d; ++j) {
      const double b = to_c(B[i + (int64_t)j * ldb]);
      for (int t = 0; t < nev; ++t) {
        ar[t] += b * ys[t * d + j];
        ai[t] += b * ys[nev * d + t * d + j];
      }
    }
    for (int t = 0; t < nev; ++t) {
      Xre[i + (int64_t)t * n] = ar[t];
      if (Xim) Xim[i + (int64_t)t * n] = ai[t];
      nrm[t] += ar[t] * ar[t] + ai[t] * ai[t];
    }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int t = 0; t < nev; ++t) {
    const double v = warp_sum(nrm[t]);
    if (lane == 0) sh[t * 8 + wid] = v;
  }
  __syncthreads();
  if (threadIdx.x < nev) {
    double a = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) a += sh[threadIdx.x * 8 + w];
    part[blockIdx.x * nev + threadIdx.x] = a;
  }
}

__global__ void ritz_normalize_kernel(double* __restrict__ Xre, double* __restrict__ Xim, int64_t n, int nev,
                                      const double* __restrict__ part, int nblk) {
  __shared__ double inv[kMaxNev];
  if (threadIdx.x < nev) {
    double a = 0;
    for (int b = 0; b < nblk; ++b) a += part[b * nev + threadIdx.x];
    inv[threadIdx.x] = a > 0 ? 1.0 / sqrt(a) : 0.0;
  }
  __syncthreads();
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n * nev; q += (int64_t)gridDim.x * blockDim.x) {
    const int t = (int)(q / n);
    Xre[q] *= inv[t];
    if (Xim) Xim[q] *= inv[t];
  }
}


__device__ __forceinline__ double block_sum_srr(double v, double* sh) {
  v = warp_sum(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double a = 0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) a += sh[w];
  return a;
}

// ---- column-pivoted Householder QR of C in [C | D] -------------------------------------
// Step j: the remaining column of C with the largest norm (over rows j..)
// moves to position j, and D's column j with it, so that C' = C P and
// D' = D P describe the same permuted basis B P; its Householder reflector
// is formed (v from the diagonal down, v_0 on the diagonal, R's diagonal in
// rdiag, tau = 2 / v^T v); every later column of C' and all of D' receive
// the reflector, and the later columns of C' their norm over the rows below
// j, recomputed from the updated entries.

// squared norms of C's columns c0 + blockIdx.x over rows r0..s-1
__global__ void __launch_bounds__(kSrrThreads)
colnorm2_kernel(const double* __restrict__ Aug, int s, int r0, int c0, double* __restrict__ cn2) {
  __shared__ double sh[32];
  const int c = c0 + blockIdx.x;
  double p = 0;
  for (int r = r0 + threadIdx.x; r < s; r += blockDim.x) p += Aug[(int64_t)c * s + r] * Aug[(int64_t)c * s + r];
  p = block_sum_srr(p, sh);
  if (threadIdx.x == 0) cn2[c] = p;
}

__global__ void __launch_bounds__(kSrrThreads)
pivot_reflector_kernel(double* __restrict__ Aug, int s, int d, int j, double* __restrict__ cn2,
                       int* __restrict__ perm, double* __restrict__ rdiag, double* __restrict__ tau) {
  __shared__ double sv[32];
  __shared__ int si[32];
  __shared__ double sh[32];
  __shared__ int s_p;
  // pivot: the largest remaining norm, the smaller index on ties
  double bv = -1.0;
  int bi = d;
  for (int c = j + threadIdx.x; c < d; c += blockDim.x) {
    const double v = cn2[c];
    if (v > bv) { bv = v; bi = c; }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
  }
  if ((threadIdx.x & 31) == 0) { sv[threadIdx.x >> 5] = bv; si[threadIdx.x >> 5] = bi; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = sv[0];
    int i = si[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
      if (sv[w] > b || (sv[w] == b && si[w] < i)) { b = sv[w]; i = si[w]; }
    s_p = i;
  }
  __syncthreads();
  const int p = s_p;
  if (p != j && p < d) {
    for (int r = threadIdx.x; r < s; r += blockDim.x) {
      double* cj = Aug + (int64_t)j * s;
      double* cp = Aug + (int64_t)p * s;
      const double t = cj[r]; cj[r] = cp[r]; cp[r] = t;
      double* dj = Aug + (int64_t)(d + j) * s;
      double* dp = Aug + (int64_t)(d + p) * s;
      const double u = dj[r]; dj[r] = dp[r]; dp[r] = u;
    }
    if (threadIdx.x == 0) {
      const double t = cn2[j]; cn2[j] = cn2[p]; cn2[p] = t;
      const int q = perm[j]; perm[j] = perm[p]; perm[p] = q;
    }
  }
  __syncthreads();
  double* x = Aug + (int64_t)j * s;
  double part = 0;
  for (int r = j + threadIdx.x; r < s; r += blockDim.x) part += x[r] * x[r];
  const double nrm2 = block_sum_srr(part, sh);
  if (threadIdx.x == 0) {
    const double x0 = x[j];
    const double nrm = sqrt(nrm2);
    const double alpha = (x0 >= 0) ? -nrm : nrm;
    const double v0 = x0 - alpha;
    const double vtv = nrm2 - x0 * x0 + v0 * v0;
    x[j] = v0;
    rdiag[j] = (vtv > 0) ? alpha : x0;
    tau[j] = (vtv > 0) ? 2.0 / vtv : 0.0;
  }
}

// column c = j + 1 + blockIdx.x (later columns of C', then all of D')
__global__ void __launch_bounds__(kSrrThreads)
pivot_apply_kernel(double* __restrict__ Aug, int s, int d, int j, const double* __restrict__ tau,
                   double* __restrict__ cn2) {
  __shared__ double sh[32];
  const int c = j + 1 + blockIdx.x;
  const double* v = Aug + (int64_t)j * s;
  double* a = Aug + (int64_t)c * s;
  double part = 0;
  for (int r = j + threadIdx.x; r < s; r += blockDim.x) part += v[r] * a[r];
  const double w = block_sum_srr(part, sh) * tau[j];
  double nq = 0;
  for (int r = j + threadIdx.x; r < s; r += blockDim.x) {
    const double nv = a[r] - w * v[r];
    a[r] = nv;
    if (r > j) nq += nv * nv;
  }
  if (c < d) {
    nq = block_sum_srr(nq, sh);
    if (threadIdx.x == 0) cn2[c] = nq;
  }
}

__global__ void iota_kernel(int* p, int d) {
  for (int i = threadIdx.x; i < d; i += blockDim.x) p[i] = i;
}

static sk_status enqueue_pivoted_qr(double* Aug, int s, int d, double* rdiag, double* tau, double* cn2, int* perm,
                                    cudaStream_t st) {
  iota_kernel<<<1, 256, 0, st>>>(perm, d);
  colnorm2_kernel<<<d, kSrrThreads, 0, st>>>(Aug, s, 0, 0, cn2);
  for (int j = 0; j < d; ++j) {
    pivot_reflector_kernel<<<1, kSrrThreads, 0, st>>>(Aug, s, d, j, cn2, perm, rdiag, tau);
    pivot_apply_kernel<<<2 * d - j - 1, kSrrThreads, 0, st>>>(Aug, s, d, j, tau, cn2);
  }
  SK_CUDA(cudaGetLastError());
  return SK_OK;
}

// ---- SVD of R by one-sided Jacobi on W = R^T -------------------------------------------
// Rotations J make the columns of W V (V = the product of the J) mutually
// orthogonal: R^T V = U~ Sigma, i.e. R = V Sigma U~^T, so V holds R's left and
// U~ = (W V) Sigma^{-1} its right singular vectors (one-sided Jacobi of
// Hestenes; on the triangle of a column-pivoted QR it converges in few
// sweeps).  One sweep visits every pair of columns once in the round-robin
// (circle) order: m = d rounded up to even, in round r the positions
// L(0) = 0, L(q) = 1 + (q - 1 + r) mod (m - 1) are paired as (L(k), L(m-1-k)),
// so a round's pairs are disjoint and run in parallel (one CTA each).

// W[i, c] = R[c, i] (R's upper triangle: rdiag on the diagonal, Aug above), V = I
__global__ void jacobi_init_kernel(const double* __restrict__ Aug, const double* __restrict__ rdiag, int s, int d,
                                   double* __restrict__ W, double* __restrict__ V) {
  const int64_t total = (int64_t)d * d;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(q % d), c = (int)(q / d);
    W[q] = (i > c) ? Aug[(int64_t)i * s + c] : (i == c ? rdiag[c] : 0.0);
    V[q] = (i == c) ? 1.0 : 0.0;
  }
}

// off: running max of |w_a^T w_b| / (||w_a|| ||w_b||) over the sweep, as the
// bit pattern of a non-negative double (ordered like the value)
__global__ void __launch_bounds__(kSrrThreads)
jacobi_round_kernel(double* __restrict__ W, double* __restrict__ V, int d, int m, int r, double tol,
                    unsigned long long* __restrict__ off) {
  __shared__ double sh[3][32];
  __shared__ double s_cs[2];
  const int k = blockIdx.x;
  auto pos = [&](int q) { return q == 0 ? 0 : 1 + (q - 1 + r) % (m - 1); };
  int a = pos(k), b = pos(m - 1 - k);
  if (a > b) { const int t = a; a = b; b = t; }
  if (b >= d) return;  // the padding column of an odd d
  double* wa = W + (int64_t)a * d;
  double* wb = W + (int64_t)b * d;
  double pa = 0, pb = 0, pg = 0;
  for (int i = threadIdx.x; i < d; i += blockDim.x) {
    const double x = wa[i], y = wb[i];
    pa += x * x;
    pb += y * y;
    pg += x * y;
  }
  pa = warp_sum(pa);
  pb = warp_sum(pb);
  pg = warp_sum(pg);
  if ((threadIdx.x & 31) == 0) { sh[0][threadIdx.x >> 5] = pa; sh[1][threadIdx.x >> 5] = pb; sh[2][threadIdx.x >> 5] = pg; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double al = 0, be = 0, ga = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { al += sh[0][w]; be += sh[1][w]; ga += sh[2][w]; }
    double c = 1.0, sn = 0.0;
    if (al > 0 && be > 0 && ga != 0.0) {
      const double rel = fabs(ga) / sqrt(al * be);
      atomicMax(off, (unsigned long long)__double_as_longlong(rel));
      if (rel > tol) {
        const double zeta = (be - al) / (2.0 * ga);
        const double t = (fabs(zeta) > 1e150) ? 0.5 / zeta
                                              : copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        c = 1.0 / sqrt(1.0 + t * t);
        sn = c * t;
      }
    }
    s_cs[0] = c;
    s_cs[1] = sn;
  }
  __syncthreads();
  const double c = s_cs[0], sn = s_cs[1];
  if (sn == 0.0) return;
  double* va = V + (int64_t)a * d;
  double* vb = V + (int64_t)b * d;
  for (int i = threadIdx.x; i < d; i += blockDim.x) {
    const double x = wa[i], y = wb[i];
    wa[i] = c * x - sn * y;
    wb[i] = sn * x + c * y;
    const double p = va[i], q = vb[i];
    va[i] = c * p - sn * q;
    vb[i] = sn * p + c * q;
  }
}

// sigma_c = ||W[:, c]||; then (one thread) the order of decreasing sigma
// (ties by index) and the kept count r = #{sigma_t >= sigma_1 / trunc_tol}.
__global__ void __launch_bounds__(kSrrThreads)
jacobi_sigma_kernel(const double* __restrict__ W, int d, double* __restrict__ sigma) {
  __shared__ double sh[32];
  const int c = blockIdx.x;
  double p = 0;
  for (int i = threadIdx.x; i < d; i += blockDim.x) p += W[(int64_t)c * d + i] * W[(int64_t)c * d + i];
  p = block_sum_srr(p, sh);
  if (threadIdx.x == 0) sigma[c] = sqrt(p);
}

__global__ void sigma_order_kernel(const double* __restrict__ sigma, int d, double trunc_tol, int* __restrict__ ord,
                                   int* __restrict__ rank) {
  if (threadIdx.x != 0) return;
  for (int i = 0; i < d; ++i) ord[i] = i;
  for (int i = 1; i < d; ++i) {  // insertion sort, decreasing sigma, ties by index
    const int v = ord[i];
    int p = i - 1;
    while (p >= 0 && (sigma[ord[p]] < sigma[v] || (sigma[ord[p]] == sigma[v] && ord[p] > v))) {
      ord[p + 1] = ord[p];
      --p;
    }
    ord[p + 1] = v;
  }
  const double s1 = sigma[ord[0]];
  int r = 0;
  if (s1 > 0)
    for (int t = 0; t < d; ++t)
      if (sigma[ord[t]] >= s1 / trunc_tol) ++r;
  *rank = r;
}

// T1[i, u] = sum_l Dtop[i, l] U~[l, u],  U~[:, u] = W[:, ord[u]] / sigma[ord[u]]
// (Dtop = the first d rows of Q^T D', i.e. of Aug's D part), for u < r.
__global__ void g_left_kernel(const double* __restrict__ Aug, int s, int d, const double* __restrict__ W,
                              const double* __restrict__ sigma, const int* __restrict__ ord,
                              const int* __restrict__ rank, double* __restrict__ T1) {
  const int r = *rank;
  const int64_t total = (int64_t)d * r;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(q % d), u = (int)(q / d);
    const int cu = ord[u];
    const double* wc = W + (int64_t)cu * d;
    double acc = 0;
    for (int l = 0; l < d; ++l) acc += Aug[(int64_t)(d + l) * s + i] * wc[l];
    T1[q] = acc / sigma[cu];
  }
}

// Ms[t, u] = (1 / sigma_t) sum_i V[i, ord[t]] T1[i, u]  (r x r, ld r): the
// matrix Sigma_r^{-1} U_r^T D V_r of the generalized problem, made standard.
__global__ void g_right_kernel(const double* __restrict__ V, const double* __restrict__ T1, int d,
                               const double* __restrict__ sigma, const int* __restrict__ ord,
                               const int* __restrict__ rank, double* __restrict__ Ms) {
  const int r = *rank;
  const int64_t total = (int64_t)r * r;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int t = (int)(q % r), u = (int)(q / r);
    const double* vt = V + (int64_t)ord[t] * d;
    double acc = 0;
    for (int i = 0; i < d; ++i) acc += vt[i] * T1[(int64_t)u * d + i];
    Ms[q] = acc / sigma[ord[t]];
  }
}

// Y'[:, c] = U~_r Z[:, c] (d x nev, complex): Ritz coefficients in the
// permuted basis B P.
__global__ void ritz_coef_kernel(const double* __restrict__ W, const double* __restrict__ sigma,
                                 const int* __restrict__ ord, const int* __restrict__ rank, int d, int nev,
                                 const double* __restrict__ Zre, const double* __restrict__ Zim,
                                 double* __restrict__ Yre, double* __restrict__ Yim) {
  const int r = *rank;
  const int64_t total = (int64_t)d * nev;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(q % d), c = (int)(q / d);
    double ar = 0, ai = 0;
    for (int u = 0; u < r; ++u) {
      const int cu = ord[u];
      const double wu = W[(int64_t)cu * d + i] / sigma[cu];
      ar += wu * Zre[(int64_t)c * r + u];
      ai += wu * Zim[(int64_t)c * r + u];
    }
    Yre[q] = ar;
    Yim[q] = ai;
  }
}

// y = P y' (B's coordinates) times the basis column scale: Yp[perm[k]] = Y'[k] * cs[perm[k]]
__global__ void unpermute_kernel(const double* __restrict__ Yre, const double* __restrict__ Yim,
                                 const int* __restrict__ perm, const double* __restrict__ cs, int d, int nev,
                                 double* __restrict__ Pre, double* __restrict__ Pim) {
  const int64_t total = (int64_t)d * nev;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(q % d), c = (int)(q / d);
    const int j = perm ? perm[k] : k;
    const double f = cs ? cs[j] : 1.0;
    Pre[(int64_t)c * d + j] = Yre[q] * f;
    Pim[(int64_t)c * d + j] = Yim[q] * f;
  }
}

// ---- the reduction after the sketches ------------------------------------------------
sk_status srr_tail(double* Aug, int s, int d, const void* B, int64_t ldb, int64_t n, sk_dtype dt,
                   const double* colscale, int nev, int symmetric, double tau_conv, double trunc_tol, SrrOut out,
                   Scratch& sc, cudaStream_t st, int* eig_fail) {
  const bool stab = trunc_tol > 0;
  double *rdiag, *qtau, *etau, *wr, *wi, *Wre, *Wim, *Zre, *Zim, *Yre, *Yim, *Pre, *Pim, *res, *part, *Mx;
  int *sel, *estat, *perm = nullptr, *ord = nullptr, *rankd = nullptr;
  SK_TRY(sc.alloc(&rdiag, d));
  SK_TRY(sc.alloc(&qtau, (size_t)((d + kQrNb - 1) / kQrNb) * kQrNb * kQrNb + d));
  SK_TRY(sc.alloc(&etau, 2 * (size_t)d));
  SK_TRY(sc.alloc(&wr, d));
  SK_TRY(sc.alloc(&wi, d));
  SK_TRY(sc.alloc(&Wre, (size_t)2 * nev * d * d));
  Wim = Wre + (size_t)nev * d * d;
  SK_TRY(sc.alloc(&Zre, (size_t)4 * nev * d));
  Zim = Zre + (size_t)nev * d;
  Yre = Zim + (size_t)nev * d;
  Yim = Yre + (size_t)nev * d;
  SK_TRY(sc.alloc(&Pre, (size_t)2 * nev * d));
  Pim = Pre + (size_t)nev * d;
  SK_TRY(sc.alloc(&res, (size_t)nev * 3));
  SK_TRY(sc.alloc(&Mx, (size_t)d * d));
  SK_TRY(sc.alloc(&sel, nev));
  SK_TRY(sc.alloc(&estat, 1));
  SK_CUDA(cudaMemsetAsync(estat, 0, sizeof(int), st));
  int r = d;
  if (!stab) {
    // Algorithm 2: C = U T; M-hat = T^{-1} (U^T D)
    double* tau = qtau + (size_t)((d + kQrNb - 1) / kQrNb) * kQrNb * kQrNb;
    SK_TRY(enqueue_qr(Aug, s, d, 2 * d, rdiag, tau, qtau, st));
    mhat_kernel<<<d, 256, 0, st>>>(Aug, rdiag, s, d, Mx);
    SK_CUDA(cudaGetLastError());
    SK_TRY(enqueue_eig(Mx, d, nev, etau, wr, wi, sel, Wre, Wim, Yre, Yim, estat, st));
  } else {
    // §6.5: C P = Q R (column pivoting), R = V Sigma U~^T (Jacobi); with
    // U_r = Q V_r and V_r = P U~_r the generalized problem
    // (U_r^T D V_r) z = theta Sigma_r z is solved as eig(Sigma_r^{-1} U_r^T D V_r)
    double *cn2, *W, *V, *sigma, *T1;
    unsigned long long* off;
    SK_TRY(sc.alloc(&cn2, d));
    SK_TRY(sc.alloc(&perm, d));
    SK_TRY(sc.alloc(&W, (size_t)2 * d * d));
    V = W + (size_t)d * d;
    SK_TRY(sc.alloc(&sigma, d));
    SK_TRY(sc.alloc(&ord, d + 1));
    rankd = ord + d;
    SK_TRY(sc.alloc(&T1, (size_t)d * d));
    SK_TRY(sc.alloc(&off, 1));
    SK_TRY(enqueue_pivoted_qr(Aug, s, d, rdiag, qtau, cn2, perm, st));
    jacobi_init_kernel<<<grid_for((int64_t)d * d, 256, 8 * num_sms()), 256, 0, st>>>(Aug, rdiag, s, d, W, V);
    SK_CUDA(cudaGetLastError());
    const int m = d + (d & 1);
    const double tol = (double)d * 2.220446049250313e-16;
    unsigned long long hoff = 0;
    int sweeps = 0;
    for (; sweeps < 40; ++sweeps) {
      SK_CUDA(cudaMemsetAsync(off, 0, sizeof(unsigned long long), st));
      for (int rr = 0; rr < m - 1; ++rr) jacobi_round_kernel<<<m / 2, kSrrThreads, 0, st>>>(W, V, d, m, rr, tol, off);
      SK_CUDA(cudaGetLastError());
      SK_CUDA(cudaMemcpyAsync(&hoff, off, sizeof(hoff), cudaMemcpyDeviceToHost, st));
      SK_CUDA(cudaStreamSynchronize(st));
      double rel;
      std::memcpy(&rel, &hoff, sizeof(rel));
      if (rel <= tol) break;
    }
    if (sweeps >= 40) { set_error("stabilized sRR: Jacobi SVD did not converge in 40 sweeps"); return SK_ENOCONV; }
    jacobi_sigma_kernel<<<d, kSrrThreads, 0, st>>>(W, d, sigma);
    sigma_order_kernel<<<1, 32, 0, st>>>(sigma, d, trunc_tol, ord, rankd);
    SK_CUDA(cudaGetLastError());
    SK_CUDA(cudaMemcpyAsync(&r, rankd, sizeof(int), cudaMemcpyDeviceToHost, st));
    SK_CUDA(cudaStreamSynchronize(st));
    if (out.rank) *out.rank = r;
    if (r < 3 || r < nev) {
      set_error("stabilized sRR: the truncated SVD keeps %d singular values, fewer than max(3, nev = %d)", r, nev);
      return SK_EILLCOND;
    }
    g_left_kernel<<<grid_for((int64_t)d * r, 256, 8 * num_sms()), 256, 0, st>>>(Aug, s, d, W, sigma, ord, rankd, T1);
    g_right_kernel<<<grid_for((int64_t)r * r, 256, 8 * num_sms()), 256, 0, st>>>(V, T1, d, sigma, ord, rankd, Mx);
    SK_CUDA(cudaGetLastError());
    SK_TRY(enqueue_eig(Mx, r, nev, etau, wr, wi, sel, Wre, Wim, Zre, Zim, estat, st));
    ritz_coef_kernel<<<grid_for((int64_t)d * nev, 256, 4 * num_sms()), 256, 0, st>>>(W, sigma, ord, rankd, d, nev, Zre,
                                                                                      Zim, Yre, Yim);
    SK_CUDA(cudaGetLastError());
  }
  srr_resid_kernel<<<nev, 256, 0, st>>>(Aug, rdiag, s, d, wr, wi, sel, Yre, Yim, symmetric, res);
  unpermute_kernel<<<grid_for((int64_t)d * nev, 256, 4 * num_sms()), 256, 0, st>>>(Yre, Yim, perm, colscale, d, nev,
                                                                                     Pre, Pim);
  SK_CUDA(cudaGetLastError());
  const int nblk = grid_for(n, kSrrThreads * 4, 2 * num_sms());
  SK_TRY(sc.alloc(&part, (size_t)nblk * nev));
  const size_t smem = (size_t)2 * nev * d * sizeof(double);
  double* Xi = (out.X_im && !symmetric) ? out.X_im : nullptr;
  if (dt == SK_F64) {
    SK_CUDA(cudaFuncSetAttribute(ritz_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, kDynSmemLimit));
    ritz_kernel<double><<<nblk, 256, smem, st>>>((const double*)B, ldb, n, d, nev, Pre, Pim, symmetric, out.X_re, Xi,
                                                 part);
  } else if (dt == SK_F32) {
    SK_CUDA(cudaFuncSetAttribute(ritz_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, kDynSmemLimit));
    ritz_kernel<float><<<nblk, 256, smem, st>>>((const float*)B, ldb, n, d, nev, Pre, Pim, symmetric, out.X_re, Xi,
                                                part);
  } else {
    SK_CUDA(cudaFuncSetAttribute(ritz_kernel<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kDynSmemLimit));
    ritz_kernel<__nv_bfloat16><<<nblk, 256, smem, st>>>((const __nv_bfloat16*)B, ldb, n, d, nev, Pre, Pim, symmetric,
                                                        out.X_re, Xi, part);
  }
  SK_CUDA(cudaGetLastError());
  ritz_normalize_kernel<<<grid_for(n * nev, 256, 2 * num_sms()), 256, 0, st>>>(out.X_re, Xi, n, nev, part, nblk);
  SK_CUDA(cudaGetLastError());
  if (out.X_im && symmetric) SK_CUDA(cudaMemsetAsync(out.X_im, 0, sizeof(double) * (size_t)n * nev, st));
  double hres[3 * kMaxNev];
  int hstat = 0;
  SK_CUDA(cudaMemcpyAsync(hres, res, sizeof(double) * 3 * nev, cudaMemcpyDeviceToHost, st));
  SK_CUDA(cudaMemcpyAsync(&hstat, estat, sizeof(int), cudaMemcpyDeviceToHost, st));
  SK_CUDA(cudaStreamSynchronize(st));
  int conv = 0;
  for (int t = 0; t < nev; ++t) {
    out.lam_re[t] = hres[3 * t];
    if (out.lam_im) out.lam_im[t] = hres[3 * t + 1];
    if (out.rhat) out.rhat[t] = hres[3 * t + 2];
    if (hres[3 * t + 2] <= tau_conv) ++conv;
  }
  if (out.nconv) *out.nconv = conv;
  if (eig_fail) *eig_fail = hstat;
  return SK_OK;
}

}  // namespace sk

// ---- sRR on a caller's basis; restarted sRR on block Chebyshev bases ----------------
namespace sk {

// M[:, j] = A B[:, j] (FP64) for j < d
template <typename T>
__global__ void apply_cols_kernel(OpView<double> A, const T* __restrict__ B, int64_t ldb, int d,
                                  double* __restrict__ M) {
  const int64_t n = A.n, total = n * d;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = q % n;
    const int j = (int)(q / n);
    M[q] = A.apply(B + (int64_t)j * ldb, i);
  }
}

// One step of the block Chebyshev recurrence (§7.5, the recurrence of §4.3
// on a block; blocks column-major, ld n): Bn = alpha ((A - c) Bj - beta Bm).
__global__ void block_cheb_kernel(OpView<double> A, const double* __restrict__ Bj, const double* __restrict__ Bm,
                                  double* __restrict__ Bn, int b, double c, double alpha, double beta) {
  const int64_t n = A.n, total = n * b;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = q % n;
    const double* x = Bj + (q - i);
    const double m = A.apply(x, i) - c * x[i];
    Bn[q] = alpha * (Bm ? m - beta * Bm[q] : m);
  }
}

// 1 / ||B[:, j]|| for each column (0 for a zero column)
__global__ void __launch_bounds__(kSrrThreads)
inv_colnorm_kernel(const double* __restrict__ B, int64_t n, double* __restrict__ inv) {
  __shared__ double sh[32];
  const double* x = B + (int64_t)blockIdx.x * n;
  double p = 0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) p += x[i] * x[i];
  p = block_sum_srr(p, sh);
  if (threadIdx.x == 0) inv[blockIdx.x] = p > 0 ? 1.0 / sqrt(p) : 0.0;
}

// C and D of the unit-column basis from the sketch of the raw blocks
// SB (s x (p+1) b): with A B_0 = c B_0 + 2 rho B_1 and A B_j = c B_j +
// rho B_{j+1} + gamma B_{j-1}, column (j, q) of S A B is
// (c SB_j + rho_j SB_{j+1} + gamma_j SB_{j-1})[:, q], each scaled by inv[(j, q)].
__global__ void block_cheb_sketch_kernel(const double* __restrict__ SB, const double* __restrict__ inv, int s, int b,
                                         int p, double c, double rho, double gamma, double* __restrict__ Aug) {
  const int d = b * p;
  const int64_t total = (int64_t)s * d;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(q % s), col = (int)(q / s);
    const int j = col / b;
    const double f = inv[col];
    const double* cur = SB + (int64_t)col * s;
    double dv = c * cur[r] + (j == 0 ? 2.0 * rho : rho) * cur[(int64_t)b * s + r];
    if (j >= 1) dv += gamma * cur[r - (int64_t)b * s];
    Aug[q] = cur[r] * f;
    Aug[(int64_t)d * s + q] = dv * f;
  }
}

// G = X^T X (b x b) for X n x b (one CTA per entry i <= j, mirrored)
__global__ void __launch_bounds__(kSrrThreads)
gram_kernel(const double* __restrict__ X, int64_t n, int b, double* __restrict__ G) {
  __shared__ double sh[32];
  const int i = blockIdx.x % b, j = blockIdx.x / b;
  if (i > j) return;
  const double* xi = X + (int64_t)i * n;
  const double* xj = X + (int64_t)j * n;
  double p = 0;
  for (int64_t r = threadIdx.x; r < n; r += blockDim.x) p += xi[r] * xj[r];
  p = block_sum_srr(p, sh);
  if (threadIdx.x == 0) { G[i + j * b] = p; G[j + i * b] = p; }
}

// Cholesky G + sigma I = R^T R (upper R, in place), one thread, with
// sigma = shift * trace(G) (0 for shift = 0); *fail on a non-positive pivot
__global__ void chol_kernel(double* G, int b, double shift, int* fail) {
  if (threadIdx.x != 0) return;
  double tr = 0;
  for (int j = 0; j < b; ++j) tr += G[j + j * b];
  const double sigma = shift * tr;
  for (int j = 0; j < b; ++j) {
    double a = G[j + j * b] + sigma;
    for (int k = 0; k < j; ++k) a -= G[k + j * b] * G[k + j * b];
    if (!(a > 0)) { *fail = 1; return; }
    const double rjj = sqrt(a);
    G[j + j * b] = rjj;
    for (int c = j + 1; c < b; ++c) {
      double v = G[j + c * b];
      for (int k = 0; k < j; ++k) v -= G[k + j * b] * G[k + c * b];
      G[j + c * b] = v / rjj;
    }
  }
}

// X <- X R^{-1}, row by row (forward substitution with the upper triangle R)
__global__ void right_trsm_kernel(double* __restrict__ X, int64_t n, int b, const double* __restrict__ R) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    double row[kMaxNev];
    for (int j = 0; j < b; ++j) {
      double v = X[r + (int64_t)j * n];
      for (int k = 0; k < j; ++k) v -= row[k] * R[k + j * b];
      row[j] = v / R[j + j * b];
    }
    for (int j = 0; j < b; ++j) X[r + (int64_t)j * n] = row[j];
  }
}

// the next start block: real parts, then imaginary parts, of the Ritz
// vectors, keeping the first b columns with norm > 1e-10 (host-chosen list)
__global__ void gather_cols_kernel(const double* __restrict__ Xre, const double* __restrict__ Xim, int64_t n,
                                   const int* __restrict__ src, int b, double* __restrict__ out) {
  const int64_t total = n * b;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = q % n;
    const int c = (int)(q / n);
    const int sc = src[c];
    out[q] = (sc >= 0) ? Xre[i + (int64_t)sc * n] : Xim[i + (int64_t)(-sc - 1) * n];
  }
}

__global__ void __launch_bounds__(kSrrThreads)
colnorm_kernel(const double* __restrict__ X, int64_t n, double* __restrict__ nrm) {
  __shared__ double sh[32];
  const double* x = X + (int64_t)blockIdx.x * n;
  double p = 0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) p += x[i] * x[i];
  p = block_sum_srr(p, sh);
  if (threadIdx.x == 0) nrm[blockIdx.x] = sqrt(p);
}

// X[:, c] *= f[c] and Y[:, c] *= f[c], f = 1 / nrm
__global__ void scale_two_kernel(double* __restrict__ X, double* __restrict__ Y, int64_t n, int b,
                                 const double* __restrict__ nrm) {
  const int64_t total = n * b;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const double f = 1.0 / nrm[q / n];
    X[q] *= f;
    Y[q] *= f;
  }
}

// Q with orthonormal columns spanning X, in place: shifted CholeskyQR3
// (Fukaya, Kannan, Nakatsukasa, Yamamoto, Yanagisawa, "Shifted Cholesky QR
// for computing the QR factorization of ill-conditioned matrices", SIAM J.
// Sci. Comput. 2020): a first pass on X^T X + sigma I with sigma =
// 11 (n b + b (b + 1)) u ||X||_F^2 makes the factor well enough conditioned
// for two plain CholeskyQR passes (condition numbers up to about 1/u).
static sk_status orthonormalize(double* X, int64_t n, int b, double* G, int* fail, cudaStream_t st) {
  const double u = 1.1102230246251565e-16;
  for (int pass = 0; pass < 3; ++pass) {
    gram_kernel<<<b * b, kSrrThreads, 0, st>>>(X, n, b, G);
    const double shift = pass == 0 ? 11.0 * ((double)n * b + (double)b * (b + 1)) * u : 0.0;
    chol_kernel<<<1, 32, 0, st>>>(G, b, shift, fail);
    right_trsm_kernel<<<grid_for(n, 256, 8 * num_sms()), 256, 0, st>>>(X, n, b, G);
  }
  SK_CUDA(cudaGetLastError());
  return SK_OK;
}

}  // namespace sk

using namespace sk;

extern "C" sk_status srr_basis(const sk_op* A, const void* B, int64_t ldb, int d, sk_dtype dtype, int nev, int s,
                               const sk_opts* opts, double* lam_re, double* lam_im, double* X_re, double* X_im,
                               double* rhat, int* nconv, int* rank, void* stream) {
  SK_CHECK_ARG(A != nullptr && B != nullptr && lam_re != nullptr && X_re != nullptr, "NULL argument");
  SK_CHECK_ARG(d >= 3 && d <= kMaxSrrD, "sRR needs 3 <= d <= 232");
  SK_CHECK_ARG(nev >= 1 && nev <= d && nev <= kMaxNev, "need 1 <= nev <= min(d, 32)");
  SK_CHECK_ARG(s >= d, "need s >= d");
  SK_CHECK_ARG(ldb >= A->n, "ldb >= n");
  SK_CHECK_ARG(dtype == SK_F64 || dtype == SK_F32 || dtype == SK_BF16, "dtype");
  cudaStream_t st = (cudaStream_t)stream;
  sk_opts o;
  resolve_opts(opts, &o, d);
  const int64_t n = A->n;
  Scratch sc(st);
  double *M, *Aug, *ws;
  SK_TRY(sc.alloc(&M, (size_t)n * d));
  SK_TRY(sc.alloc(&Aug, (size_t)s * 2 * d));
  OpView<double> Av;
  make_view(A, &Av);
  const int g = grid_for(n * d, 256, 16 * num_sms());
  if (dtype == SK_F64) apply_cols_kernel<double><<<g, 256, 0, st>>>(Av, (const double*)B, ldb, d, M);
  else if (dtype == SK_F32) apply_cols_kernel<float><<<g, 256, 0, st>>>(Av, (const float*)B, ldb, d, M);
  else apply_cols_kernel<__nv_bfloat16><<<g, 256, 0, st>>>(Av, (const __nv_bfloat16*)B, ldb, d, M);
  SK_CUDA(cudaGetLastError());
  Sketcher skt;
  sk_sketch sks{o.sketch, n, s, o.zeta, o.seed};
  SK_TRY(skt.create(sks, sc, st));
  const size_t w1 = skt.ws(d, dtype, true), w2 = skt.ws(d, SK_F64, true);
  SK_TRY(sc.alloc(&ws, w1 > w2 ? w1 : w2));
  SK_TRY(skt.apply(B, ldb, d, dtype, Aug, ws, st, true));
  SK_TRY(skt.apply(M, n, d, SK_F64, Aug + (size_t)s * d, ws, st, true));
  SrrOut out{lam_re, lam_im, X_re, X_im, rhat, nconv, rank};
  if (rank) *rank = d;
  int eig_fail = 0;
  SK_TRY(srr_tail(Aug, s, d, B, ldb, n, dtype, nullptr, nev, o.symmetric, o.tau, o.srr_trunc_tol, out, sc, st,
                  &eig_fail));
  if (eig_fail) { set_error("eigensolver: QR iteration did not converge"); return SK_ENOCONV; }
  return SK_OK;
}

extern "C" sk_status srr_restarted(const sk_op* A, const double* Omega, int b, int p, int nev, double lo, double hi,
                                   int max_restarts, int filter_degree, const sk_opts* opts, double* lam_re, double* lam_im,
                                   double* X_re, double* X_im, double* rhat, int* nconv, int* restarts,
                                   double* history, void* stream) {
  SK_CHECK_ARG(A != nullptr && Omega != nullptr && lam_re != nullptr && X_re != nullptr, "NULL argument");
  SK_CHECK_ARG(b >= 1 && b <= kMaxNev && p >= 1 && b * p >= 3 && b * p <= kMaxSrrD,
               "need 1 <= b <= 32, p >= 1, 3 <= b p <= 232");
  SK_CHECK_ARG(nev >= 1 && nev <= b, "need 1 <= nev <= b");
  SK_CHECK_ARG(hi > lo && std::isfinite(lo) && std::isfinite(hi), "need finite lo < hi");
  SK_CHECK_ARG(max_restarts >= 1, "max_restarts >= 1");
  SK_CHECK_ARG(filter_degree >= 0 && filter_degree <= 100000, "0 <= filter_degree <= 100000");
  cudaStream_t st = (cudaStream_t)stream;
  const int d = b * p;
  sk_opts o;
  resolve_opts(opts, &o, d);
  const double trunc_tol = o.srr_trunc_tol > 0 ? o.srr_trunc_tol : 1e13;
  const int s = 2 * d;
  const int64_t n = A->n;
  Scratch sc(st);
  double *Bk, *X, *inv, *SB, *Aug, *ws, *G, *Xre, *Xim, *nrm;
  int *fail, *src;
  SK_TRY(sc.alloc(&Bk, (size_t)n * b * (p + 1)));
  SK_TRY(sc.alloc(&X, (size_t)n * b));
  SK_TRY(sc.alloc(&inv, d));
  SK_TRY(sc.alloc(&SB, (size_t)s * b * (p + 1)));
  SK_TRY(sc.alloc(&Aug, (size_t)s * 2 * d));
  SK_TRY(sc.alloc(&G, (size_t)b * b));
  SK_TRY(sc.alloc(&Xre, (size_t)2 * n * b));
  Xim = Xre + (size_t)n * b;
  SK_TRY(sc.alloc(&nrm, 2 * b));
  SK_TRY(sc.alloc(&fail, 1));
  double* Yf = nullptr;
  if (filter_degree > 0) SK_TRY(sc.alloc(&Yf, (size_t)3 * n * b));
  SK_TRY(sc.alloc(&src, b));
  SK_CUDA(cudaMemsetAsync(fail, 0, sizeof(int), st));
  SK_CUDA(cudaMemcpyAsync(X, Omega, sizeof(double) * (size_t)n * b, cudaMemcpyDeviceToDevice, st));
  OpView<double> Av;
  make_view(A, &Av);
  std::vector<double> lr(b), li(b), rh(b);
  double cut = hi;
  int t = 0, conv = 0;
  for (; t < max_restarts; ++t) {
    // B_0 = orth(X), optionally orth(T_m((A - c)/rho) orth(X)); the block
    // Chebyshev basis for [lo, cut]
    SK_TRY(orthonormalize(X, n, b, G, fail, st));
    const double c = 0.5 * (lo + cut), rho = 0.5 * (cut - lo), gamma = rho / 4.0;
    const int g = grid_for(n * b, 256, 16 * num_sms());
    if (filter_degree > 0) {
      // Y_1 = (A - c) Y_0 / rho, Y_{j+1} = 2 (A - c) Y_j / rho - Y_{j-1}; after
      // every 10th step both carried blocks divided by the newest one's
      // column norms
      double* Y[3] = {Yf, Yf + (size_t)n * b, Yf + (size_t)2 * n * b};
      SK_CUDA(cudaMemcpyAsync(Y[0], X, sizeof(double) * (size_t)n * b, cudaMemcpyDeviceToDevice, st));
      block_cheb_kernel<<<g, 256, 0, st>>>(Av, Y[0], nullptr, Y[1], b, c, 1.0 / rho, 0.0);
      int i0 = 0, i1 = 1;
      for (int j = 2; j <= filter_degree; ++j) {
        const int i2 = 3 - i0 - i1;
        block_cheb_kernel<<<g, 256, 0, st>>>(Av, Y[i1], Y[i0], Y[i2], b, c, 2.0 / rho, 0.5 * rho);
        i0 = i1;
        i1 = i2;
        if (j % 10 == 0) {
          colnorm_kernel<<<b, kSrrThreads, 0, st>>>(Y[i1], n, nrm);
          scale_two_kernel<<<g, 256, 0, st>>>(Y[i0], Y[i1], n, b, nrm);
        }
      }
      SK_CUDA(cudaGetLastError());
      SK_CUDA(cudaMemcpyAsync(X, Y[i1], sizeof(double) * (size_t)n * b, cudaMemcpyDeviceToDevice, st));
      SK_TRY(orthonormalize(X, n, b, G, fail, st));
    }
    SK_CUDA(cudaMemcpyAsync(Bk, X, sizeof(double) * (size_t)n * b, cudaMemcpyDeviceToDevice, st));
    for (int j = 0; j <= p - 1; ++j) {
      const double* Bj = Bk + (size_t)j * n * b;
      const double* Bm = j >= 1 ? Bk + (size_t)(j - 1) * n * b : nullptr;
      block_cheb_kernel<<<g, 256, 0, st>>>(Av, Bj, Bm, Bk + (size_t)(j + 1) * n * b, b, c,
                                           j == 0 ? 0.5 / rho : 1.0 / rho, j == 0 ? 0.0 : gamma);
    }
    SK_CUDA(cudaGetLastError());
    inv_colnorm_kernel<<<d, kSrrThreads, 0, st>>>(Bk, n, inv);
    // sketch of the p + 1 raw blocks (a fresh sketch each restart)
    Sketcher skt;
    sk_sketch sks{o.sketch, n, s, o.zeta, o.seed + (uint64_t)t};
    Scratch sct(st);
    SK_TRY(skt.create(sks, sct, st));
    SK_TRY(sct.alloc(&ws, skt.ws(b * (p + 1), SK_F64, true)));
    SK_TRY(skt.apply(Bk, n, b * (p + 1), SK_F64, SB, ws, st, true));
    block_cheb_sketch_kernel<<<grid_for((int64_t)s * d, 256, 8 * num_sms()), 256, 0, st>>>(SB, inv, s, b, p, c, rho,
                                                                                          gamma, Aug);
    SK_CUDA(cudaGetLastError());
    int hf = 0;
    SK_CUDA(cudaMemcpyAsync(&hf, fail, sizeof(int), cudaMemcpyDeviceToHost, st));
    SK_CUDA(cudaStreamSynchronize(st));
    if (hf) { set_error("srr_restarted: the start block is numerically rank deficient"); return SK_EILLCOND; }
    SrrOut out{lr.data(), li.data(), Xre, Xim, rh.data(), nullptr, nullptr};
    int eig_fail = 0;
    SK_TRY(srr_tail(Aug, s, d, Bk, n, n, SK_F64, inv, b, o.symmetric, o.tau, trunc_tol, out, sct, st, &eig_fail));
    if (eig_fail) { set_error("eigensolver: QR iteration did not converge"); return SK_ENOCONV; }
    double h = 0;
    for (int q = 0; q < nev; ++q) h = std::max(h, rh[q]);
    if (history) history[t] = h;
    if (h <= o.tau || t + 1 == max_restarts) { ++t; break; }
    // next start block: real parts, then imaginary parts, first b with norm > 1e-10
    cut = lr[b - 1];
    colnorm_kernel<<<b, kSrrThreads, 0, st>>>(Xre, n, nrm);
    colnorm_kernel<<<b, kSrrThreads, 0, st>>>(Xim, n, nrm + b);
    double hn[2 * kMaxNev];
    SK_CUDA(cudaMemcpyAsync(hn, nrm, sizeof(double) * 2 * b, cudaMemcpyDeviceToHost, st));
    SK_CUDA(cudaStreamSynchronize(st));
    int hs[kMaxNev], cnt = 0;
    for (int q = 0; q < 2 * b && cnt < b; ++q)
      if (hn[q] > 1e-10) hs[cnt++] = q < b ? q : -(q - b) - 1;
    if (cnt < b) { set_error("srr_restarted: fewer than b independent Ritz vector parts"); return SK_EILLCOND; }
    SK_CUDA(cudaMemcpyAsync(src, hs, sizeof(int) * b, cudaMemcpyHostToDevice, st));
    gather_cols_kernel<<<grid_for(n * b, 256, 8 * num_sms()), 256, 0, st>>>(Xre, Xim, n, src, b, X);
    SK_CUDA(cudaGetLastError());
    SK_CUDA(cudaStreamSynchronize(st));  // hs lives on the host stack
  }
  // the nev leading pairs of the last restart
  for (int q = 0; q < nev; ++q) {
    lam_re[q] = lr[q];
    if (lam_im) lam_im[q] = li[q];
    if (rhat) rhat[q] = rh[q];
    if (rh[q] <= o.tau) ++conv;
  }
  SK_CUDA(cudaMemcpyAsync(X_re, Xre, sizeof(double) * (size_t)n * nev, cudaMemcpyDeviceToDevice, st));
  if (X_im) SK_CUDA(cudaMemcpyAsync(X_im, Xim, sizeof(double) * (size_t)n * nev, cudaMemcpyDeviceToDevice, st));
  SK_CUDA(cudaStreamSynchronize(st));
  if (nconv) *nconv = conv;
  if (restarts) *restarts = t;
  return conv == nev ? SK_OK : SK_ENOCONV;
}
