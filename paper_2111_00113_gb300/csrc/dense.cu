// Small dense FP64 algebra of the sketched problems (s x d, d <= a few
// hundred): C = (S B_{d+1}) Hbar, blocked Householder QR, the sketched
// least-squares solve (§3.3 eqs. (sgmres-yhat), (sgmres-rhat)) and the
// kappa(T) truncation (§5.3).
//
// The QR works in place on an augmented s x ncols matrix: the first nq
// columns are factored, the remaining columns (the sketched right-hand side
// g for sGMRES, S A B for sRR) receive Q^T through the trailing updates.
// Panel p is factored by one CTA (reflectors stored below the diagonal,
// v_0 on the diagonal, R's diagonal in rdiag, tau = 2 / v^T v) together with
// its compact-WY factor T_p (Q_p = I - V T_p V^T); the trailing update
// A <- A - V T_p^T (V^T A) runs one CTA per column.
#include <cmath>

#include "common.cuh"
#include "dense.cuh"

namespace sk {

// Aug[:, j] = sum_i SB[:, i] Hbar[i, j] over the k+1 nonzeros of column j,
// for j < du (du = min(stop, d)); zero for du <= j < d.
__global__ void hbar_product_kernel(const double* __restrict__ SB, const double* __restrict__ Hbar, int s, int d,
                                    int k, const int* __restrict__ stop, double* __restrict__ Aug) {
  const int du = min(*stop, d);
  const int64_t total = (int64_t)s * d;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(q % s), j = (int)(q / s);
    double a = 0;
    if (j < du) {
      const int i0 = max(0, j - k + 1);
      for (int i = i0; i <= j + 1; ++i) {
        if (i >= *stop) continue;  // columns past a breakdown were never formed
        a += SB[(int64_t)i * s + r] * Hbar[(int64_t)j * (d + 1) + i];
      }
    }
    Aug[q] = a;
  }
}

// Copy SB columns [0, du) into Aug (zero beyond du): the sketched basis for sRR.
__global__ void copy_sb_kernel(const double* __restrict__ SB, int s, int d, const int* __restrict__ stop,
                               double* __restrict__ Aug) {
  const int du = min(*stop, d);
  const int64_t total = (int64_t)s * d;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(q / s);
    Aug[q] = (j < du) ? SB[q] : 0.0;
  }
}

__device__ __forceinline__ double block_sum1(double v, double* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double a = 0;
  for (int w = 0; w < nw; ++w) a += sh[w];
  return a;
}

// One CTA factors panel columns [p0, p0+nbc) of Aug (s rows, ld s) in place
// in global memory (fallback for panels too tall for shared memory).
__global__ void __launch_bounds__(kQrPanelThreads)
qr_panel_global_kernel(double* __restrict__ Aug, int s, int p0, int nbc, double* __restrict__ rdiag,
                double* __restrict__ tau, double* __restrict__ Tws) {
  __shared__ double sh[32];
  __shared__ double s_tau[kQrNb];
  __shared__ double s_T[kQrNb * kQrNb];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int jj = 0; jj < nbc; ++jj) {
    const int col = p0 + jj;
    double* x = Aug + (int64_t)col * s;
    double part = 0;
    for (int r = col + threadIdx.x; r < s; r += blockDim.x) part += x[r] * x[r];
    const double nrm2 = block_sum1(part, sh);
    const double x0 = (col < s) ? x[col] : 0.0;
    const double nrm = sqrt(nrm2);
    const double alpha = (x0 >= 0) ? -nrm : nrm;
    const double v0 = x0 - alpha;
    const double vtv = nrm2 - x0 * x0 + v0 * v0;
    const double t = (vtv > 0) ? 2.0 / vtv : 0.0;
    __syncthreads();
    if (threadIdx.x == 0) {
      if (col < s) x[col] = v0;
      rdiag[col] = (vtv > 0) ? alpha : x0;
      tau[col] = t;
      s_tau[jj] = t;
    }
    __syncthreads();
    // apply H = I - t v v^T to the remaining panel columns (one warp each)
    for (int c = col + 1 + wid; c < p0 + nbc; c += nw) {
      double* y = Aug + (int64_t)c * s;
      double dot = 0;
      for (int r = col + lane; r < s; r += 32) dot += x[r] * y[r];
      dot = warp_sum(dot) * t;
      for (int r = col + lane; r < s; r += 32) y[r] -= dot * x[r];
    }
    __syncthreads();
  }
  // compact WY: T[jj,jj] = tau_jj, T[:jj, jj] = -tau_jj T[:jj,:jj] (V[:, :jj]^T v_jj)
  for (int q = threadIdx.x; q < kQrNb * kQrNb; q += blockDim.x) s_T[q] = 0;
  __syncthreads();
  for (int jj = 0; jj < nbc; ++jj) {
    // z_i = v_i^T v_jj for i < jj, one warp per i; v_jj starts at row p0+jj
    const int cj = p0 + jj;
    const double* vj = Aug + (int64_t)cj * s;
    for (int i = wid; i < jj; i += nw) {
      const double* vi = Aug + (int64_t)(p0 + i) * s;
      double dot = 0;
      for (int r = cj + lane; r < s; r += 32) dot += vi[r] * vj[r];
      dot = warp_sum(dot);
      if (lane == 0) sh[i] = dot;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int i = 0; i < jj; ++i) {
        double a = 0;
        for (int l = i; l < jj; ++l) a += s_T[i * kQrNb + l] * sh[l];
        s_T[i * kQrNb + jj] = -s_tau[jj] * a;
      }
      s_T[jj * kQrNb + jj] = s_tau[jj];
    }
    __syncthreads();
  }
  for (int q = threadIdx.x; q < kQrNb * kQrNb; q += blockDim.x) Tws[q] = s_T[q];
}

// One CTA factors panel columns [p0, p0+nbc) of Aug: the panel's rows p0..s-1
// are staged in shared memory, factored column by column (norm, reflector,
// dots of all remaining panel columns in parallel, rank-1 update by the
// whole block), and written back with the compact-WY factor T.
__global__ void __launch_bounds__(kQrPanelThreads)
qr_panel_kernel(double* __restrict__ Aug, int s, int p0, int nbc, double* __restrict__ rdiag,
                double* __restrict__ tau, double* __restrict__ Tws) {
  extern __shared__ double P[];  // len x nbc, column-major, ld = len
  __shared__ double sh[32];
  __shared__ double s_tau[kQrNb];
  __shared__ double s_dot[kQrNb];
  __shared__ double s_T[kQrNb * kQrNb];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int len = s - p0;
  for (int q = threadIdx.x; q < len * nbc; q += blockDim.x) {
    const int c = q / len, r = q - c * len;
    P[q] = Aug[(int64_t)(p0 + c) * s + p0 + r];
  }
  __syncthreads();
  for (int jj = 0; jj < nbc; ++jj) {
    double* v = P + (int64_t)jj * len;
    double part = 0;
    for (int r = jj + threadIdx.x; r < len; r += blockDim.x) part += v[r] * v[r];
    const double nrm2 = block_sum1(part, sh);
    const double x0 = v[jj];
    const double nrm = sqrt(nrm2);
    const double alpha = (x0 >= 0) ? -nrm : nrm;
    const double v0 = x0 - alpha;
    const double vtv = nrm2 - x0 * x0 + v0 * v0;
    const double t = (vtv > 0) ? 2.0 / vtv : 0.0;
    __syncthreads();
    if (threadIdx.x == 0) {
      v[jj] = v0;
      rdiag[p0 + jj] = (vtv > 0) ? alpha : x0;
      tau[p0 + jj] = t;
      s_tau[jj] = t;
    }
    __syncthreads();
    for (int c = jj + 1 + wid; c < nbc; c += nw) {
      const double* y = P + (int64_t)c * len;
      double dot = 0;
      for (int r = jj + lane; r < len; r += 32) dot += v[r] * y[r];
      dot = warp_sum(dot);
      if (lane == 0) s_dot[c] = dot * t;
    }
    __syncthreads();
    const int rows = len - jj, cols = nbc - jj - 1;
    for (int q = threadIdx.x; q < rows * cols; q += blockDim.x) {
      const int c = jj + 1 + q / rows, r = jj + q % rows;
      P[(int64_t)c * len + r] -= s_dot[c] * v[r];
    }
    __syncthreads();
  }
  for (int q = threadIdx.x; q < kQrNb * kQrNb; q += blockDim.x) s_T[q] = 0;
  __syncthreads();
  for (int jj = 0; jj < nbc; ++jj) {
    const double* vj = P + (int64_t)jj * len;
    for (int i = wid; i < jj; i += nw) {
      const double* vi = P + (int64_t)i * len;
      double dot = 0;
      for (int r = jj + lane; r < len; r += 32) dot += vi[r] * vj[r];
      dot = warp_sum(dot);
      if (lane == 0) sh[i] = dot;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int i = 0; i < jj; ++i) {
        double a = 0;
        for (int l = i; l < jj; ++l) a += s_T[i * kQrNb + l] * sh[l];
        s_T[i * kQrNb + jj] = -s_tau[jj] * a;
      }
      s_T[jj * kQrNb + jj] = s_tau[jj];
    }
    __syncthreads();
  }
  for (int q = threadIdx.x; q < kQrNb * kQrNb; q += blockDim.x) Tws[q] = s_T[q];
  for (int q = threadIdx.x; q < len * nbc; q += blockDim.x) {
    const int c = q / len, r = q - c * len;
    Aug[(int64_t)(p0 + c) * s + p0 + r] = P[q];
  }
}

// Column c = c0 + blockIdx.x of Aug gets Q_p^T: a <- a - V T^T (V^T a).
__global__ void __launch_bounds__(kQrTrailThreads)
qr_trailing_kernel(double* __restrict__ Aug, int s, int p0, int nbc, int c0, const double* __restrict__ Tws) {
  __shared__ double red[kQrNb * (kQrTrailThreads / 32)];
  __shared__ double w[kQrNb];
  const int c = c0 + blockIdx.x;
  double* a = Aug + (int64_t)c * s;
  const double* V = Aug + (int64_t)p0 * s;
  double acc[kQrNb];
#pragma unroll
  for (int i = 0; i < kQrNb; ++i) acc[i] = 0;
  for (int r = p0 + threadIdx.x; r < s; r += blockDim.x) {
    const double ar = a[r];
#pragma unroll
    for (int i = 0; i < kQrNb; ++i) {
      if (i < nbc && r >= p0 + i) acc[i] += V[(int64_t)i * s + r] * ar;
    }
  }
  block_sum_k<kQrNb>(acc, red);
  if (threadIdx.x == 0) {
    for (int i = 0; i < nbc; ++i) {
      double t = 0;
      for (int l = 0; l <= i; ++l) t += Tws[l * kQrNb + i] * acc[l];  // (T^T w)_i
      w[i] = t;
    }
  }
  __syncthreads();
  for (int r = p0 + threadIdx.x; r < s; r += blockDim.x) {
    double u = 0;
#pragma unroll
    for (int i = 0; i < kQrNb; ++i) {
      if (i < nbc && r >= p0 + i) u += V[(int64_t)i * s + r] * w[i];
    }
    a[r] -= u;
  }
}

sk_status enqueue_qr(double* Aug, int s, int nq, int ncols, double* rdiag, double* tau, double* Tws,
                     cudaStream_t st) {
  for (int p0 = 0; p0 < nq; p0 += kQrNb) {
    const int nbc = (nq - p0) < kQrNb ? (nq - p0) : kQrNb;
    double* T = Tws + (int64_t)(p0 / kQrNb) * kQrNb * kQrNb;
    const size_t smem = (size_t)(s - p0) * nbc * sizeof(double);
    if (smem <= 200 * 1024) {
      SK_CUDA(cudaFuncSetAttribute(qr_panel_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kDynSmemLimit));
      qr_panel_kernel<<<1, kQrPanelThreads, smem, st>>>(Aug, s, p0, nbc, rdiag, tau, T);
    } else {
      qr_panel_global_kernel<<<1, kQrPanelThreads, 0, st>>>(Aug, s, p0, nbc, rdiag, tau, T);
    }
    const int c0 = p0 + nbc;
    if (ncols > c0) qr_trailing_kernel<<<ncols - c0, kQrTrailThreads, 0, st>>>(Aug, s, p0, nbc, c0, T);
  }
  SK_CUDA(cudaGetLastError());
  return SK_OK;
}

// Back substitution for the sketched LS with the kappa truncation.
// Aug: R above the diagonal of columns [0, d), rdiag its diagonal; column d
// holds Q^T g.  Writes y (d, zero past width) and diag = {rhat, kappa, width}.
// Blocked from the bottom: for each block of 32 unknowns, warp 0 solves the
// 32 x 32 triangle from shared memory with shuffles, then the whole CTA
// subtracts the block's contribution from the rows above it.
__global__ void __launch_bounds__(1024)
ls_solve_kernel(const double* __restrict__ Aug, const double* __restrict__ rdiag, int s, int d, double stab_tol,
                double* __restrict__ y, double* __restrict__ diag) {
  extern __shared__ double zz[];  // d right-hand side entries, then the 32 x d block of R
  double* Rb = zz + d;             // Rb[c * d + t] = R[t, i0 + c]
  __shared__ double sh[32];
  __shared__ int s_width;
  __shared__ double s_kappa;
  const double* z = Aug + (int64_t)d * s;
  if (threadIdx.x == 0) {
    double mx = 0, mn = INFINITY, kap = 1.0;
    int width = 0;
    for (int j = 0; j < d; ++j) {
      const double a = fabs(rdiag[j]);
      if (!(a > 0) || !isfinite(a)) break;
      mx = fmax(mx, a);
      mn = fmin(mn, a);
      kap = mx / mn;
      if (kap > stab_tol) break;
      width = j + 1;
    }
    double mxa = 0, mna = INFINITY;
    for (int j = 0; j < d; ++j) { const double a = fabs(rdiag[j]); mxa = fmax(mxa, a); mna = fmin(mna, a); }
    s_kappa = (mna > 0) ? mxa / mna : INFINITY;
    s_width = width;
  }
  __syncthreads();
  const int width = s_width;
  for (int i = threadIdx.x; i < d; i += blockDim.x) zz[i] = (i < width) ? z[i] : 0.0;
  double part = 0;
  for (int i = width + threadIdx.x; i < s; i += blockDim.x) part += z[i] * z[i];
  const double rh2 = block_sum1(part, sh);
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int i1 = width; i1 > 0; i1 -= 32) {
    const int i0 = max(0, i1 - 32);
    const int nb = i1 - i0;
    // stage R[0:i1, i0:i1]
    for (int q = threadIdx.x; q < nb * i1; q += blockDim.x) {
      const int c = q / i1, t = q - c * i1;
      Rb[c * d + t] = (t == i0 + c) ? rdiag[i0 + c] : Aug[(int64_t)(i0 + c) * s + t];
    }
    __syncthreads();
    if (wid == 0) {
      // lane l holds unknown i0 + l; solve bottom-up within the block
      double zl = (lane < nb) ? zz[i0 + lane] : 0.0;
      double yl = 0.0;
      for (int c = nb - 1; c >= 0; --c) {
        const double yc = __shfl_sync(0xffffffffu, zl, c) / Rb[c * d + i0 + c];
        if (lane == c) yl = yc;
        if (lane < c) zl -= yc * Rb[c * d + i0 + lane];
      }
      if (lane < nb) zz[i0 + lane] = yl;
    }
    __syncthreads();
    // rows above the block: zz[t] -= sum_c R[t, i0+c] y[i0+c]
    for (int t = threadIdx.x; t < i0; t += blockDim.x) {
      double a = zz[t];
      for (int c = 0; c < nb; ++c) a -= Rb[c * d + t] * zz[i0 + c];
      zz[t] = a;
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < d; i += blockDim.x) y[i] = (i < width) ? zz[i] : 0.0;
  if (threadIdx.x == 0) {
    diag[0] = sqrt(rh2);
    diag[1] = s_kappa;
    diag[2] = (double)width;
  }
}

sk_status enqueue_ls_solve(const double* Aug, const double* rdiag, int s, int d, double stab_tol, double* y,
                           double* diag, cudaStream_t st) {
  const size_t smem = (size_t)d * 33 * sizeof(double);
  if (smem > (size_t)kDynSmemLimit) { set_error("ls_solve: d too large"); return SK_EINVAL; }
  SK_CUDA(cudaFuncSetAttribute(ls_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kDynSmemLimit));
  ls_solve_kernel<<<1, 1024, smem, st>>>(Aug, rdiag, s, d, stab_tol, y, diag);
  SK_CUDA(cudaGetLastError());
  return SK_OK;
}

sk_status enqueue_hbar_product(const double* SB, const double* Hbar, int s, int d, int k, const int* stop,
                               double* Aug, cudaStream_t st) {
  int blocks = (int)(((int64_t)s * d + 255) / 256);
  if (blocks > 4 * num_sms()) blocks = 4 * num_sms();
  hbar_product_kernel<<<blocks, 256, 0, st>>>(SB, Hbar, s, d, k, stop, Aug);
  SK_CUDA(cudaGetLastError());
  return SK_OK;
}

sk_status enqueue_copy_sb(const double* SB, int s, int d, const int* stop, double* Aug, cudaStream_t st) {
  int blocks = (int)(((int64_t)s * d + 255) / 256);
  if (blocks > 4 * num_sms()) blocks = 4 * num_sms();
  copy_sb_kernel<<<blocks, 256, 0, st>>>(SB, s, d, stop, Aug);
  SK_CUDA(cudaGetLastError());
  return SK_OK;
}

}  // namespace sk
