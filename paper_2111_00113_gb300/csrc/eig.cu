// Dense nonsymmetric eigensolver for the sketched Rayleigh-Ritz matrix
// M-hat (d x d, FP64, d <= 256): Algorithm 2's "solve eigenvalue problem"
// step, written for one GPU.
//
//   1. Householder reduction to upper Hessenberg form H = P^T M P (one CTA;
//      reflectors kept below the subdiagonal).
//   2. Eigenvalues of H by the implicitly shifted double-shift (Francis) QR
//      iteration with deflation on small subdiagonals and exceptional shifts
//      (Golub & Van Loan §7.5), eigenvalues only; H lives in shared memory in
//      a packed band-upper layout (row i keeps columns >= i-3, which holds
//      the bulge); each 3x3 reflector's row and column updates are spread over
//      the CTA's threads.
//   3. Eigenvectors for the selected eigenvalues by inverse iteration on the
//      Hessenberg matrix, (H - lambda I) y = y_prev in complex arithmetic with
//      partial pivoting between adjacent rows (one CTA per eigenvalue), then
//      back-transformed with the Householder reflectors of step 1.
#include <cmath>

#include "common.cuh"

namespace sk {

static constexpr int kEigMaxN = 256;
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
__global__ void __launch_bounds__(kEigThreads)
hessenberg_kernel(double* __restrict__ H, int n, double* __restrict__ tau) {
  __shared__ double sh[32];
  __shared__ double w[kEigMaxN];
  __shared__ double s_sc[2];
  for (int k = 0; k + 2 < n; ++k) {
    // reflector for x = H[k+1:n, k]
    double part = 0;
    for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) part += H[i + (int64_t)k * n] * H[i + (int64_t)k * n];
    const double nrm2 = block_sum_d(part, sh);
    // the reflector's scalars once (FP64 sqrt and divide are slow here), broadcast
    if (threadIdx.x == 0) {
      const double x0 = H[k + 1 + (int64_t)k * n];
      const double nrm = sqrt(nrm2);
      const double alpha = x0 >= 0 ? -nrm : nrm;
      const double v0 = x0 - alpha;
      const double vtv = nrm2 - x0 * x0 + v0 * v0;
      s_sc[0] = vtv > 0 ? 2.0 / vtv : 0.0;
      s_sc[1] = alpha;
      H[k + 1 + (int64_t)k * n] = v0;  // v stored in H[k+1:, k]; H[k+1,k] := alpha below
      tau[k] = s_sc[0];
    }
    __syncthreads();
    const double t = s_sc[0], alpha = s_sc[1];
    const double* v = H + (int64_t)k * n;  // v[i] for i >= k+1
    // left: H[k+1:, k+1:] -= t v (v^T H[k+1:, k+1:]); one warp per column
    {
      const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
      for (int j = k + 1 + wid; j < n; j += nw) {
        double a = 0;
        for (int i = k + 1 + lane; i < n; i += 32) a += v[i] * H[i + (int64_t)j * n];
        a = warp_sum(a);
        if (lane == 0) w[j] = a * t;
      }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < (n - k - 1) * (n - k - 1); q += blockDim.x) {
      const int j = k + 1 + q / (n - k - 1), i = k + 1 + q % (n - k - 1);
      H[i + (int64_t)j * n] -= v[i] * w[j];
    }
    __syncthreads();
    // right: H[:, k+1:] -= t (H[:, k+1:] v) v^T
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      double a[4] = {0, 0, 0, 0};  // four independent chains (FP64 FMA latency ~64 cycles)
      int j = k + 1;
      for (; j + 3 < n; j += 4) {
#pragma unroll
        for (int u = 0; u < 4; ++u) a[u] += H[i + (int64_t)(j + u) * n] * v[j + u];
      }
      for (; j < n; ++j) a[0] += H[i + (int64_t)j * n] * v[j];
      w[i] = ((a[0] + a[1]) + (a[2] + a[3])) * t;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < n * (n - k - 1); q += blockDim.x) {
      const int j = k + 1 + q / n, i = q % n;
      H[i + (int64_t)j * n] -= w[i] * v[j];
    }
    __syncthreads();
    if (threadIdx.x == 0) tau[n + k] = alpha;  // subdiagonal entry H[k+1, k]
    __syncthreads();
  }
}

// ---- 2. Francis double-shift QR, eigenvalues only ------------------------------------
struct Band {
  double* a;
  const int* off;
  __device__ __forceinline__ double& at(int i, int j) const { return a[off[i] + j - max(0, i - 3)]; }
};

__global__ void __launch_bounds__(kEigThreads)
hqr_kernel(const double* __restrict__ Hg, const double* __restrict__ tau, int n, double* __restrict__ wr,
           double* __restrict__ wi, int* __restrict__ status) {
  extern __shared__ double sm[];
  __shared__ int off[kEigMaxN + 1];
  __shared__ double sh[32];
  __shared__ int s_l, s_m;
  __shared__ double s_shift[3];  // x, y, w of the shift polynomial
  __shared__ double s_ref[6];    // the current 3x3 reflector (vx, vy, vz, q2, r2) and a non-zero flag
  if (threadIdx.x == 0) {
    int o = 0;
    for (int i = 0; i < n; ++i) { off[i] = o; o += n - max(0, i - 3); }
    off[n] = o;
  }
  __syncthreads();
  Band A{sm, off};
  // copy the Hessenberg part (subdiagonal from tau[n+k]); zeros below it
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    for (int j = max(0, i - 3); j < n; ++j) {
      double v = 0;
      if (j >= i) v = Hg[i + (int64_t)j * n];
      else if (j == i - 1) v = (j + 2 < n) ? tau[n + j] : Hg[i + (int64_t)j * n];
      A.at(i, j) = v;
    }
  }
  __syncthreads();
  double anorm_part = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    for (int j = max(0, i - 1); j < n; ++j) anorm_part += fabs(A.at(i, j));
  const double anorm = block_sum_d(anorm_part, sh);
  int nn = n - 1;
  double tsum = 0;  // accumulated exceptional shifts
  int fail = 0;
  while (nn >= 0) {
    int its = 0;
    int l;
    for (;;) {
      // look for a single small subdiagonal element
      __syncthreads();
      if (threadIdx.x == 0) {
        int ll;
        for (ll = nn; ll >= 1; --ll) {
          double s = fabs(A.at(ll - 1, ll - 1)) + fabs(A.at(ll, ll));
          if (s == 0.0) s = anorm;
          if (fabs(A.at(ll, ll - 1)) + s == s) { A.at(ll, ll - 1) = 0.0; break; }
        }
        s_l = ll;
      }
      __syncthreads();
      l = s_l;
      const double x = A.at(nn, nn);
      if (l == nn) {  // one eigenvalue
        if (threadIdx.x == 0) { wr[nn] = x + tsum; wi[nn] = 0.0; }
        nn -= 1;
        break;
      }
      const double y = A.at(nn - 1, nn - 1);
      const double w = A.at(nn, nn - 1) * A.at(nn - 1, nn);
      if (l == nn - 1) {  // a 2x2 block: two eigenvalues
        if (threadIdx.x == 0) {
          const double p = 0.5 * (y - x);
          const double q = p * p + w;
          const double z = sqrt(fabs(q));
          const double xs = x + tsum;
          if (q >= 0.0) {
            const double zz = p + copysign(z, p);
            wr[nn - 1] = wr[nn] = xs + zz;
            if (zz != 0.0) wr[nn] = xs - w / zz;
            wi[nn - 1] = wi[nn] = 0.0;
          } else {
            wr[nn - 1] = wr[nn] = xs + p;
            wi[nn - 1] = z;
            wi[nn] = -z;
          }
        }
        nn -= 2;
        break;
      }
      if (its == 60) { fail = 1; nn = -1; break; }
      // shifts: the eigenvalues of the trailing 2x2 block, or exceptional
      if (threadIdx.x == 0) {
        double xs = x, ys = y, ws = w;
        if (its == 10 || its == 20 || its == 30 || its == 40 || its == 50) {
          tsum += x;  // thread 0's copy; broadcast below
          for (int i = 0; i <= nn; ++i) A.at(i, i) -= x;
          const double s = fabs(A.at(nn, nn - 1)) + fabs(A.at(nn - 1, nn - 2));
          xs = ys = 0.75 * s;
          ws = -0.4375 * s * s;
        }
        s_shift[0] = xs; s_shift[1] = ys; s_shift[2] = ws;
        sh[31] = tsum;
        // find m: the first double-shift vector that is negligibly coupled above
        int m;
        for (m = nn - 2; m >= l; --m) {
          const double zm = A.at(m, m);
          const double r = xs - zm, s = ys - zm;
          double p = (r * s - ws) / A.at(m + 1, m) + A.at(m, m + 1);
          double q = A.at(m + 1, m + 1) - zm - r - s;
          double rr = A.at(m + 2, m + 1);
          const double sc = fabs(p) + fabs(q) + fabs(rr);
          p /= sc; q /= sc; rr /= sc;
          if (m == l) break;
          const double u = fabs(A.at(m, m - 1)) * (fabs(q) + fabs(rr));
          const double v = fabs(p) * (fabs(A.at(m - 1, m - 1)) + fabs(zm) + fabs(A.at(m + 1, m + 1)));
          if (u + v == v) break;
        }
        s_m = m;
        for (int i = m + 2; i <= nn; ++i) {
          A.at(i, i - 2) = 0.0;
          if (i != m + 2) A.at(i, i - 3) = 0.0;
        }
      }
      __syncthreads();
      tsum = sh[31];
      const int m = s_m;
      ++its;
      const double xs = s_shift[0], ys = s_shift[1], ws = s_shift[2];
      // double-shift QR step on rows l..nn, columns m..nn (bulge chase).  Thread
      // 0 forms each 3x3 reflector once and broadcasts it (FP64 divide and sqrt
      // take ~600 cycles each here; every thread computing them would also
      // saturate the FP64 pipe).
      for (int k = m; k <= nn - 1; ++k) {
        if (threadIdx.x == 0) {
          double p, q, r = 0.0, xk = 0.0;
          if (k == m) {
            const double zm = A.at(m, m);
            const double rr0 = xs - zm, ss0 = ys - zm;
            p = (rr0 * ss0 - ws) / A.at(m + 1, m) + A.at(m, m + 1);
            q = A.at(m + 1, m + 1) - zm - rr0 - ss0;
            r = A.at(m + 2, m + 1);
            xk = fabs(p) + fabs(q) + fabs(r);
            const double ix = 1.0 / xk;
            p *= ix; q *= ix; r *= ix;
          } else {
            p = A.at(k, k - 1);
            q = A.at(k + 1, k - 1);
            if (k != nn - 1) r = A.at(k + 2, k - 1);
            xk = fabs(p) + fabs(q) + fabs(r);
            if (xk != 0.0) {
              const double ix = 1.0 / xk;
              p *= ix; q *= ix; r *= ix;
            }
          }
          const double sg = copysign(sqrt(p * p + q * q + r * r), p);
          s_ref[5] = (sg == 0.0) ? 0.0 : 1.0;
          if (sg != 0.0) {
            if (k == m) {
              if (l != m) A.at(k, k - 1) = -A.at(k, k - 1);
            } else {
              A.at(k, k - 1) = -sg * xk;
              A.at(k + 1, k - 1) = 0.0;
              if (k != nn - 1) A.at(k + 2, k - 1) = 0.0;
            }
            const double pp = p + sg;
            const double is = 1.0 / sg, ip = 1.0 / pp;
            s_ref[0] = pp * is;  // vx
            s_ref[1] = q * is;   // vy
            s_ref[2] = r * is;   // vz
            s_ref[3] = q * ip;   // q2
            s_ref[4] = r * ip;   // r2
          }
        }
        __syncthreads();
        if (s_ref[5] == 0.0) {
          __syncthreads();  // all threads have read the flag before thread 0 forms the next reflector
          continue;
        }
        const double vx = s_ref[0], vy = s_ref[1], vz = s_ref[2], q2 = s_ref[3], r2 = s_ref[4];
        // rows k..k+2, columns k..nn
        for (int j = k + threadIdx.x; j <= nn; j += blockDim.x) {
          double t = A.at(k, j) + q2 * A.at(k + 1, j);
          if (k != nn - 1) {
            t += r2 * A.at(k + 2, j);
            A.at(k + 2, j) -= t * vz;
          }
          A.at(k + 1, j) -= t * vy;
          A.at(k, j) -= t * vx;
        }
        __syncthreads();
        // columns k..k+2, rows l..min(nn, k+3)
        const int mmin = nn < k + 3 ? nn : k + 3;
        for (int i = l + threadIdx.x; i <= mmin; i += blockDim.x) {
          double t = vx * A.at(i, k) + vy * A.at(i, k + 1);
          if (k != nn - 1) {
            t += vz * A.at(i, k + 2);
            A.at(i, k + 2) -= t * r2;
          }
          A.at(i, k + 1) -= t * q2;
          A.at(i, k) -= t;
        }
        __syncthreads();
      }
    }
  }
  if (threadIdx.x == 0) *status = fail;
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
  for (int i = threadIdx.x; i < n; i += blockDim.x) { yr[i] = 1.0; yi[i] = 0.0; }
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

size_t eig_smem_bytes(int n) {
  size_t o = 0;
  for (int i = 0; i < n; ++i) o += (size_t)(n - (i > 3 ? i - 3 : 0));
  return o * sizeof(double);
}

// M (n x n, col-major, overwritten), outputs: wr, wi (n), sel (nev), Yre/Yim
// (n x nev col-major), status (device int; 1 = QR iteration did not converge).
sk_status enqueue_eig(double* M, int n, int nev, double* tau, double* wr, double* wi, int* sel, double* Wre,
                      double* Wim, double* Yre, double* Yim, int* status, cudaStream_t st) {
  if (n > kEigMaxN || n < 3) { set_error("eigensolver supports 3 <= d <= %d", kEigMaxN); return SK_EINVAL; }
  hessenberg_kernel<<<1, kEigThreads, 0, st>>>(M, n, tau);
  SK_CUDA(cudaGetLastError());
  const size_t smem = eig_smem_bytes(n);
  if (smem > (size_t)kDynSmemLimit) { set_error("eigensolver: d too large for shared memory"); return SK_EINVAL; }
  SK_CUDA(cudaFuncSetAttribute(hqr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kDynSmemLimit));
  hqr_kernel<<<1, kEigThreads, smem, st>>>(M, tau, n, wr, wi, status);
  SK_CUDA(cudaGetLastError());
  select_kernel<<<1, 1, 0, st>>>(wr, wi, n, nev, sel);
  SK_CUDA(cudaGetLastError());
  invit_kernel<<<nev, kEigThreads, 0, st>>>(M, tau, n, wr, wi, sel, Wre, Wim, Yre, Yim);
  SK_CUDA(cudaGetLastError());
  return SK_OK;
}

}  // namespace sk
