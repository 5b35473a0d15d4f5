// Small dense FP64 algebra of the sketched problems (s x d, d <= a few
// hundred): C = (S B_{d+1}) Hbar, blocked Householder QR, the sketched
// least-squares solve (§3.3 eqs. (sgmres-yhat), (sgmres-rhat)) and the
// kappa(T) truncation (§5.3).
//
// The QR works in place on an augmented s x ncols matrix: the first nq
// columns are factored, the remaining columns (the sketched right-hand side
// g for sGMRES, S A B for sRR) receive Q^T through the trailing updates.
// Panel p is factored (reflectors stored below the diagonal, v_0 on the
// diagonal, R's diagonal in rdiag, tau = 2 / v^T v) together with its
// compact-WY factor T_p (Q_p = I - V T_p V^T); the trailing update
// A <- A - V T_p^T (V^T A) runs one 8-CTA cluster per column.
#include <cmath>
#include <cooperative_groups.h>

#include "common.cuh"
#include "dense.cuh"

namespace cg = cooperative_groups;

namespace sk {

// Aug[:, j] = sum_i SB[:, i] Hbar[i, j] over the k+1 nonzeros of column j,
// for columns c0 <= j < c1 (0 <= c0 < c1 <= d): the product for j < du
// (du = min(stop, d)), zero for du <= j.
__global__ void hbar_product_kernel(const double* __restrict__ SB, const double* __restrict__ Hbar, int s, int d,
                                    int k, const int* __restrict__ stop, int c0, int c1, double* __restrict__ Aug,
                                    JobSlab js) {
  SB = at_job(SB, js);
  Hbar = at_job(Hbar, js);
  stop = at_job(stop, js);
  Aug = at_job(Aug, js);
  const int du = min(*stop, d);
  const int64_t total = (int64_t)s * (c1 - c0);
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(q % s), j = c0 + (int)(q / s);
    double a = 0;
    if (j < du) {
      const int i0 = max(0, j - k + 1);
      for (int i = i0; i <= j + 1; ++i) {
        if (i >= *stop) continue;  // columns past a breakdown were never formed
        a += SB[(int64_t)i * s + r] * Hbar[(int64_t)j * (d + 1) + i];
      }
    }
    Aug[(int64_t)j * s + r] = a;
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
                double* __restrict__ tau, double* __restrict__ Tws, JobSlab js) {
  Aug = at_job(Aug, js);
  rdiag = at_job(rdiag, js);
  tau = at_job(tau, js);
  Tws = at_job(Tws, js);
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
                double* __restrict__ tau, double* __restrict__ Tws, JobSlab js) {
  Aug = at_job(Aug, js);
  rdiag = at_job(rdiag, js);
  tau = at_job(tau, js);
  Tws = at_job(Tws, js);
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

// Reduce-scatter of 16 per-lane values over a warp: on return lanes 2c and
// 2c+1 hold the warp-wide sum of value c.  16 FP64 adds per lane instead of
// the 80 of sixteen independent butterflies.
__device__ __forceinline__ double warp_reduce_scatter16(double (&v)[16]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int h = 8, off = 16; h >= 1; h >>= 1, off >>= 1) {
    const bool hi = (lane & off) != 0;
#pragma unroll
    for (int i = 0; i < h; ++i) {
      const double send = hi ? v[i] : v[i + h];
      const double keep = hi ? v[i + h] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
    }
  }
  return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

// Panel factorization spread over a cluster of kQrCluster CTAs.  CTA q holds
// a contiguous block of the panel's rows in shared memory, one row per
// thread of the row warps.  Step j needs, over the panel rows >= j and with x
// the current column j,
//   tot_c = sum_r P[r, c] x_r   for every panel column c,   row_c = P[j, c];
// then with alpha = -sign(x_0) ||x|| (||x||^2 = tot_j, x_0 = row_j) and the
// reflector v = x - alpha e_j:
//   v^T y_c  = tot_c - alpha row_c   (c > j, applied to the later columns)
//   v_c^T v  = tot_c - alpha row_c   (c < j, the compact-WY coupling z_c).
// A thread folds the update of step j and the partial sums of step j+1 into
// one pass over its own row; partials go through a warp reduce-scatter, then
// the control warp pushes them into every CTA of the cluster (remote shared
// stores) and a single cluster barrier per column publishes them.  All CTAs
// sum the pushed partials in rank order, so they hold identical reflectors.
// The control warp also extends T (Q_p = I - V T V^T) by one column per step
// while the row warps update.  Partial slots are double-buffered by column
// parity: a slot is rewritten two barriers after it was read.
static constexpr int kQrCluster = 8;
static constexpr int kQrClusterThreads = 256;
static constexpr int kQrRowWarps = kQrClusterThreads / 32 - 1;

__global__ void __launch_bounds__(kQrClusterThreads)
qr_panel_cluster_kernel(double* __restrict__ Aug, int s, int p0, int nbc, double* __restrict__ rdiag,
                        double* __restrict__ tau, double* __restrict__ Tws, JobSlab js) {
  Aug = at_job(Aug, js);
  rdiag = at_job(rdiag, js);
  tau = at_job(tau, js);
  Tws = at_job(Tws, js);
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ double P[];                           // rows x kQrNb, column-major (ld = per)
  __shared__ double slot[2][kQrCluster][kQrNb];            // tot partials of every rank
  __shared__ double rowslot[2][kQrNb];                     // row j, posted by its owner
  __shared__ double wpart[kQrRowWarps][kQrNb];
  __shared__ double s_T[kQrNb * kQrNb];
  __shared__ double s_dot[kQrNb];                          // tau * v^T y_c
  __shared__ double s_z[kQrNb];
  __shared__ double s_v0;
  const int q = (int)cluster.block_rank();
  const int len = s - p0;
  const int per = (len + kQrCluster - 1) / kQrCluster;
  const int r0 = q * per;                                  // first panel row held by this CTA
  const int rows = max(0, min(len, r0 + per) - r0);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const bool ctrl = (wid == kQrRowWarps);
  const int nrt = kQrRowWarps * 32;                        // row threads
  for (int t = threadIdx.x; t < rows * kQrNb; t += blockDim.x) {
    const int c = t / rows, r = t - c * rows;
    P[c * per + r] = (c < nbc) ? Aug[(int64_t)(p0 + c) * s + p0 + r0 + r] : 0.0;
  }
  for (int e = threadIdx.x; e < kQrNb * kQrNb; e += blockDim.x) s_T[e] = 0;
  cluster.sync();  // every CTA of the cluster has started before the first remote store
  for (int jj = 0; jj < nbc; ++jj) {
    const int buf = jj & 1;
    if (!ctrl) {
      // update by reflector jj-1 (s_dot, s_v0 from the previous step), then partials of step jj
      double acc[kQrNb];
#pragma unroll
      for (int c = 0; c < kQrNb; ++c) acc[c] = 0;
      if (wid * 32 < rows) {
        for (int r = threadIdx.x; r < rows; r += nrt) {
          const int g = r0 + r;
          if (jj > 0 && g >= jj - 1) {
            double x = P[(jj - 1) * per + r];
            if (g == jj - 1) {
              x = s_v0;
              P[(jj - 1) * per + r] = x;
            }
#pragma unroll
            for (int c = 0; c < kQrNb; ++c)
              if (c >= jj) P[c * per + r] -= s_dot[c] * x;
          }
          if (g >= jj) {
            const double x = P[jj * per + r];
#pragma unroll
            for (int c = 0; c < kQrNb; ++c) acc[c] += P[c * per + r] * x;
          }
        }
        const double w = warp_reduce_scatter16(acc);
        if ((lane & 1) == 0) wpart[wid][lane >> 1] = w;
      } else if (lane < 2 * kQrNb && (lane & 1) == 0) {
        wpart[wid][lane >> 1] = 0.0;
      }
    }
    __syncthreads();
    if (ctrl) {
      // this CTA's partial, pushed to every rank; the owner of row jj posts that row
      if (lane < kQrNb) {
        double a = 0;
#pragma unroll
        for (int w = 0; w < kQrRowWarps; ++w) a += wpart[w][lane];
        for (int k = 0; k < kQrCluster; ++k) cluster.map_shared_rank(&slot[buf][q][0], k)[lane] = a;
      } else if (jj >= r0 && jj < r0 + rows) {
        const double v = P[(lane - kQrNb) * per + (jj - r0)];
        for (int k = 0; k < kQrCluster; ++k) cluster.map_shared_rank(&rowslot[buf][0], k)[lane - kQrNb] = v;
      }
    }
    cluster.sync();
    if (ctrl) {
      const int c = lane & (kQrNb - 1);
      double tot = 0;
#pragma unroll
      for (int k = 0; k < kQrCluster; ++k) tot += slot[buf][k][c];
      const double row = rowslot[buf][c];
      const double nrm2 = __shfl_sync(0xffffffffu, tot, jj);
      const double x0 = __shfl_sync(0xffffffffu, row, jj);
      const double nrm = sqrt(nrm2);
      const double alpha = (x0 >= 0) ? -nrm : nrm;
      const double v0 = x0 - alpha;
      const double vtv = nrm2 - x0 * x0 + v0 * v0;
      const double t = (vtv > 0) ? 2.0 / vtv : 0.0;
      const double qv = tot - alpha * row;
      if (lane < kQrNb) {
        s_dot[c] = (c > jj) ? t * qv : 0.0;
        s_z[c] = (c < jj) ? qv : 0.0;
      }
      if (lane == 0) {
        s_v0 = v0;
        if (q == 0) {
          rdiag[p0 + jj] = (vtv > 0) ? alpha : x0;
          tau[p0 + jj] = t;
        }
      }
      __syncwarp();
      // T[:jj, jj] = -t T[:jj, :jj] z, T[jj, jj] = t (runs while the row warps update)
      if (lane < jj) {
        double a = 0;
        for (int l = lane; l < jj; ++l) a += s_T[lane * kQrNb + l] * s_z[l];
        s_T[lane * kQrNb + jj] = -t * a;
      } else if (lane == jj) {
        s_T[jj * kQrNb + jj] = t;
      }
      __syncwarp();
    }
    __syncthreads();
  }
  // the last reflector's update of the panel (only its own diagonal entry changes)
  for (int r = threadIdx.x; r < rows; r += blockDim.x)
    if (r0 + r == nbc - 1) P[(nbc - 1) * per + r] = s_v0;
  __syncthreads();
  if (q == 0)
    for (int e = threadIdx.x; e < kQrNb * kQrNb; e += blockDim.x) Tws[e] = s_T[e];
  for (int e = threadIdx.x; e < rows * nbc; e += blockDim.x) {
    const int c = e / rows, r = e - c * rows;
    Aug[(int64_t)(p0 + c) * s + p0 + r0 + r] = P[c * per + r];
  }
}

// Q_p^T of panels p_first .. p_last - 1, in order, applied to column
// c = c0 + blockIdx.x / kWyCluster by a cluster of kWyCluster CTAs: CTA q
// always owns rows [q per, (q+1) per) of the column (per = ceil(s / 8)), so a
// row is only ever read and written by its owner.  For each panel the CTAs'
// partial sums of u = V^T a (over their rows at or below the panel's
// diagonal) are pushed into every CTA's shared memory, one cluster barrier
// publishes them, every CTA sums them in rank order (identical u
// everywhere), forms w = T^T u and updates its rows: a <- a - V w.  The same
// kernel serves the right-looking trailing update (one panel, many columns)
// and the left-looking one (all earlier panels, the new columns), so the
// sequential and the pipelined QR give identical columns.  The FP64 work of
// one column is spread over 8 SMs (one SM's FP64 rate made the one-CTA
// left-looking update, 16 columns x up to 18 panels, take ~240 us).
static constexpr int kWyCluster = 8;
static constexpr int kWyThreads = 128;

__global__ void __launch_bounds__(kWyThreads)
qr_apply_cluster_kernel(double* __restrict__ Aug, int s, int p_first, int p_last, int last_nbc, int c0,
                        const double* __restrict__ Tws, JobSlab js) {
  Aug = at_job(Aug, js);
  Tws = at_job(Tws, js);
  cg::cluster_group cluster = cg::this_cluster();
  __shared__ double slot[2][kWyCluster][kQrNb];
  __shared__ double red[kWyThreads / 32][kQrNb];
  __shared__ double uu[kQrNb];
  __shared__ double w[kQrNb];
  const int q = (int)cluster.block_rank();
  const int c = c0 + (int)(blockIdx.x / kWyCluster);
  double* a = Aug + (int64_t)c * s;
  const int per = (s + kWyCluster - 1) / kWyCluster;
  const int r_lo = q * per, r_hi = min(s, r_lo + per);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  cluster.sync();  // every CTA of the cluster has started before the first remote store
  for (int p = p_first; p < p_last; ++p) {
    const int buf = (p - p_first) & 1;
    const int p0 = p * kQrNb;
    const int nbc = (p == p_last - 1) ? last_nbc : kQrNb;
    const double* V = Aug + (int64_t)p0 * s;
    const double* T = Tws + (int64_t)p * kQrNb * kQrNb;
    __syncthreads();  // the previous panel's row updates (by other threads of this CTA) are visible
    double acc[kQrNb];
#pragma unroll
    for (int i = 0; i < kQrNb; ++i) acc[i] = 0;
    for (int r = max(r_lo, p0) + threadIdx.x; r < r_hi; r += blockDim.x) {
      const double ar = a[r];
#pragma unroll
      for (int i = 0; i < kQrNb; ++i)
        if (i < nbc && r >= p0 + i) acc[i] += V[(int64_t)i * s + r] * ar;
    }
    const double part = warp_reduce_scatter16(acc);
    if ((lane & 1) == 0) red[wid][lane >> 1] = part;
    __syncthreads();
    if (wid == 0 && lane < kQrNb) {
      double t = 0;
      for (int k = 0; k < nw; ++k) t += red[k][lane];
      for (int k = 0; k < kWyCluster; ++k) cluster.map_shared_rank(&slot[buf][q][0], k)[lane] = t;
    }
    cluster.sync();
    if (wid == 0) {
      if (lane < kQrNb) {
        double t = 0;
        for (int k = 0; k < kWyCluster; ++k) t += slot[buf][k][lane];
        uu[lane] = t;
      }
      __syncwarp();
      if (lane < kQrNb) {
        double t = 0;
        for (int l = 0; l <= lane && l < nbc; ++l) t += T[l * kQrNb + lane] * uu[l];
        w[lane] = (lane < nbc) ? t : 0.0;
      }
    }
    __syncthreads();
    for (int r = max(r_lo, p0) + threadIdx.x; r < r_hi; r += blockDim.x) {
      double d = 0;
#pragma unroll
      for (int i = 0; i < kQrNb; ++i)
        if (i < nbc && r >= p0 + i) d += V[(int64_t)i * s + r] * w[i];
      a[r] -= d;
    }
  }
  cluster.sync();  // no CTA leaves while another may still store into its shared memory
}

// Panels p_first .. p_last - 1 (the last with last_nbc columns) applied to
// columns [c0, c0 + ncols).
static sk_status launch_wy_apply(double* Aug, int s, int p_first, int p_last, int last_nbc, int c0, int ncols,
                                 const double* Tws, cudaStream_t st, const JobSlab& js = JobSlab(), int nj = 1) {
  if (ncols <= 0 || p_last <= p_first) return SK_OK;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)ncols * kWyCluster, (unsigned)nj);
  cfg.blockDim = dim3(kWyThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kWyCluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  SK_CUDA(cudaLaunchKernelEx(&cfg, qr_apply_cluster_kernel, Aug, s, p_first, p_last, last_nbc, c0, Tws, js));
  return SK_OK;
}

// Factor panel [p0, p0+nbc) of Aug in place: the 8-CTA cluster kernel when
// the panel is tall enough, else one CTA (shared or global memory).  (One
// CTA holding a 600 x 16 panel in registers was tried: slower, 2.9 against
// 2.0 ms of QR per cycle, because one SM's FP64 pipe issues one warp
// instruction per 16 cycles and the per-column products and reductions of
// the whole panel then queue on it.)
static sk_status factor_panel(double* Aug, int s, int p0, int nbc, double* rdiag, double* tau, double* T,
                              cudaStream_t st, const JobSlab& js = JobSlab(), int nj = 1) {
  const int per = (s - p0 + kQrCluster - 1) / kQrCluster;
  if (s - p0 >= 4 * kQrCluster && (size_t)per * kQrNb * sizeof(double) <= (size_t)kDynSmemLimit) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kQrCluster, (unsigned)nj);
    cfg.blockDim = dim3(kQrClusterThreads);
    cfg.dynamicSmemBytes = (size_t)per * kQrNb * sizeof(double);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kQrCluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    SK_CUDA(cudaFuncSetAttribute(qr_panel_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kDynSmemLimit));
    SK_CUDA(cudaLaunchKernelEx(&cfg, qr_panel_cluster_kernel, Aug, s, p0, nbc, rdiag, tau, T, js));
    return SK_OK;
  }
  const size_t smem = (size_t)(s - p0) * nbc * sizeof(double);
  if (smem <= 200 * 1024) {
    SK_CUDA(cudaFuncSetAttribute(qr_panel_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kDynSmemLimit));
    qr_panel_kernel<<<dim3(1, nj), kQrPanelThreads, smem, st>>>(Aug, s, p0, nbc, rdiag, tau, T, js);
  } else {
    qr_panel_global_kernel<<<dim3(1, nj), kQrPanelThreads, 0, st>>>(Aug, s, p0, nbc, rdiag, tau, T, js);
  }
  return SK_OK;
}

sk_status enqueue_qr(double* Aug, int s, int nq, int ncols, double* rdiag, double* tau, double* Tws,
                     cudaStream_t st, const JobSlab& js, int nj) {
  for (int p0 = 0; p0 < nq; p0 += kQrNb) {
    const int nbc = (nq - p0) < kQrNb ? (nq - p0) : kQrNb;
    double* T = Tws + (int64_t)(p0 / kQrNb) * kQrNb * kQrNb;
    SK_TRY(factor_panel(Aug, s, p0, nbc, rdiag, tau, T, st, js, nj));
    const int c0 = p0 + nbc;
    SK_TRY(launch_wy_apply(Aug, s, p0 / kQrNb, p0 / kQrNb + 1, nbc, c0, ncols - c0, Tws, st, js, nj));
  }
  SK_CUDA(cudaGetLastError());
  return SK_OK;
}

// Columns [c0, c1) joined a QR whose columns [0, c0) are factored (c0 a
// multiple of the panel width) and whose column zc has received those
// panels' reflectors.  Every earlier panel is applied to the new columns in
// order (left-looking, one launch), then the new panels are factored, each
// applied to the new columns right of it and to column zc.  Column by
// column this is the arithmetic of enqueue_qr: the same reflectors, in the
// same order, through the same per-column update.  Returns the launch count
// through *launches.
sk_status enqueue_qr_append(double* Aug, int s, int c0, int c1, int zc, double* rdiag, double* tau, double* Tws,
                            long long* launches, cudaStream_t st) {
  if (c0 < 0 || c0 % kQrNb != 0 || c1 <= c0 || zc < c1 || s <= c1) {
    set_error("qr_append: bad column range");
    return SK_EINVAL;
  }
  long long nl = 0;
  if (c0 > 0) {
    SK_TRY(launch_wy_apply(Aug, s, 0, c0 / kQrNb, kQrNb, c0, c1 - c0, Tws, st));
    ++nl;
  }
  for (int p0 = c0; p0 < c1; p0 += kQrNb) {
    const int nbc = (c1 - p0) < kQrNb ? (c1 - p0) : kQrNb;
    double* T = Tws + (int64_t)(p0 / kQrNb) * kQrNb * kQrNb;
    SK_TRY(factor_panel(Aug, s, p0, nbc, rdiag, tau, T, st));
    const int cn = p0 + nbc;
    if (c1 > cn) {
      SK_TRY(launch_wy_apply(Aug, s, p0 / kQrNb, p0 / kQrNb + 1, nbc, cn, c1 - cn, Tws, st));
      ++nl;
    }
    SK_TRY(launch_wy_apply(Aug, s, p0 / kQrNb, p0 / kQrNb + 1, nbc, zc, 1, Tws, st));
    nl += 2;
  }
  SK_CUDA(cudaGetLastError());
  if (launches) *launches += nl;
  return SK_OK;
}

// Early stop of the iterative cycle (§5.2 eq. (sgmres-iterative-soln)), run
// after the QR covers columns [0, c1) and z = Q^T g.  For every prefix j in
// (c0, c1] the estimate is rhat_j^2 = sum_{i >= j} z_i^2 (the reflectors past
// j leave that tail's norm unchanged).  out[0] = the first j with
// rhat_j <= tau ||z|| (||z|| = ||g||), or 0; out[1] = 1 when the kappa
// estimate of the solve (max/min |r_jj| over [0, c1)) exceeds stab_tol or a
// diagonal entry is zero or not finite (§5.3), or when the basis broke down
// before column c1 (stop <= c1).  One CTA of kCheckThreads threads; the chunk
// c1 - c0 is at most kCheckThreads.
static constexpr int kCheckThreads = 1024;

__global__ void __launch_bounds__(kCheckThreads)
prefix_check_kernel(const double* __restrict__ z, const double* __restrict__ rdiag, const int* __restrict__ stop,
                    int s, int c0, int c1, const double* __restrict__ tau_p, double stab_tol, int* __restrict__ out) {
  const double tau = *tau_p;
  __shared__ double red[kCheckThreads / 32][2];
  __shared__ double wsum[kCheckThreads / 32];
  __shared__ long long wmx[kCheckThreads / 32], wmn[kCheckThreads / 32];
  __shared__ int s_first;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const long long kAbs = 0x7fffffffffffffffLL;
  const long long kInf = 0x7ff0000000000000LL;
  if (threadIdx.x == 0) s_first = 0x7fffffff;
  // ||z||^2 and the tail past the chunk, sum_{i >= c1} z_i^2
  double all = 0, tail = 0;
  for (int i = threadIdx.x; i < s; i += blockDim.x) {
    const double q = z[i] * z[i];
    all += q;
    if (i >= c1) tail += q;
  }
  // max / min |r_jj| over [0, c1) on the IEEE bit patterns
  long long mx = 0, mn = kInf;
  for (int j = threadIdx.x; j < c1; j += blockDim.x) {
    const long long b = __double_as_longlong(rdiag[j]) & kAbs;
    mx = max(mx, b);
    mn = min(mn, b);
  }
  all = warp_sum(all);
  tail = warp_sum(tail);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
  }
  // inclusive suffix sums of v_t = z_{c0+t}^2 within the chunk, t < m
  const int m = c1 - c0;
  const int t = threadIdx.x;
  double v = (t < m) ? z[c0 + t] * z[c0 + t] : 0.0;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double u = __shfl_down_sync(0xffffffffu, v, o);
    if (lane + o < 32) v += u;
  }
  if (lane == 0) {
    red[wid][0] = all;
    red[wid][1] = tail;
    wsum[wid] = v;  // lane 0 holds its warp's total
    wmx[wid] = mx;
    wmn[wid] = mn;
  }
  __syncthreads();
  double tot = 0, tl = 0, later = 0;
  long long gmx = 0, gmn = kInf;
  for (int w = 0; w < nw; ++w) {
    tot += red[w][0];
    tl += red[w][1];
    if (w > wid) later += wsum[w];
    gmx = max(gmx, wmx[w]);
    gmn = min(gmn, wmn[w]);
  }
  // thread t in [1, m) tests prefix j = c0 + t: rhat_j^2 = sum_{u >= t} v_u
  // + tail; thread 0 tests j = c1 (the tail alone)
  if (t < m) {
    const double r2 = (t == 0 ? 0.0 : v + later) + tl;
    if (r2 <= tau * tau * tot) atomicMin(&s_first, t == 0 ? c1 : c0 + t);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double dmx = __longlong_as_double(gmx), dmn = __longlong_as_double(gmn);
    const bool bad = gmn == 0 || gmx >= kInf || dmx > stab_tol * dmn || *stop <= c1;
    out[0] = (s_first == 0x7fffffff) ? 0 : s_first;
    out[1] = bad ? 1 : 0;
  }
}

sk_status enqueue_prefix_check(const double* z, const double* rdiag, const int* stop, int s, int c0, int c1,
                               const double* tau, double stab_tol, int* out, cudaStream_t st) {
  if (c0 < 0 || c1 <= c0 || c1 - c0 > kCheckThreads || c1 > s) {
    set_error("prefix_check: bad column range");
    return SK_EINVAL;
  }
  prefix_check_kernel<<<1, kCheckThreads, 0, st>>>(z, rdiag, stop, s, c0, c1, tau, stab_tol, out);
  SK_CUDA(cudaGetLastError());
  return SK_OK;
}

// Back substitution for the sketched LS with the kappa truncation.
// Aug: R above the diagonal of columns [0, d), rdiag its diagonal; column d
// holds Q^T g.  Writes y (d, zero past width) and diag = {rhat, kappa, width}.
//
// width is the longest leading block whose diagonal is finite, nonzero and
// has max|r_jj| <= stab_tol * min|r_jj|: a block-wide prefix max/min of the
// |r_jj| taken on their IEEE bit patterns (ordered like the values for
// non-negative doubles), so no FP64 division or compare chain runs serially.
// The solve is blocked from the bottom: for each block of 32 unknowns warp 0
// forms the 32 reciprocals of the diagonal in parallel and solves the
// triangle with shuffles; then four threads per row subtract the block's
// contribution from the rows above it.
static constexpr int kLsThreads = 1024;

__device__ __forceinline__ long long warp_scan_max(long long v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v = max(v, u);
  }
  return v;
}
__device__ __forceinline__ long long warp_scan_min(long long v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v = min(v, u);
  }
  return v;
}

__global__ void __launch_bounds__(kLsThreads)
ls_solve_kernel(const double* __restrict__ Aug, const double* __restrict__ rdiag, const double* __restrict__ z,
                int s, int d, double stab_tol, double* __restrict__ y, double* __restrict__ diag, JobSlab js) {
  Aug = at_job(Aug, js);
  rdiag = at_job(rdiag, js);
  z = at_job(z, js);
  y = at_job(y, js);
  diag = at_job(diag, js);
  extern __shared__ double zz[];  // d right-hand side entries, then the 32 x d block of R
  double* Rb = zz + d;             // Rb[c * d + t] = R[t, i0 + c]
  __shared__ long long wmax[kLsThreads / 32], wmin[kLsThreads / 32];
  __shared__ long long s_cmax, s_cmin;
  __shared__ int s_width;
  __shared__ double sh[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const long long kAbs = 0x7fffffffffffffffLL;
  const long long kInf = 0x7ff0000000000000LL;
  if (threadIdx.x == 0) {
    s_cmax = 0;
    s_cmin = kInf;
    s_width = d;
  }
  __syncthreads();
  long long amax = 0, amin = kInf;  // over all d entries (the kappa estimate reported in diag[1])
  for (int base = 0; base < d; base += blockDim.x) {
    const int j = base + threadIdx.x;
    const long long bits = (j < d) ? (__double_as_longlong(rdiag[j]) & kAbs) : 0;
    const bool valid = (j < d);
    long long vmax = valid ? bits : 0, vmin = valid ? bits : kInf;
    amax = max(amax, vmax);
    amin = min(amin, vmin);
    vmax = warp_scan_max(vmax);
    vmin = warp_scan_min(vmin);
    if (lane == 31) {
      wmax[wid] = vmax;
      wmin[wid] = vmin;
    }
    __syncthreads();
    long long cmax = s_cmax, cmin = s_cmin;
    for (int w = 0; w < wid; ++w) {
      cmax = max(cmax, wmax[w]);
      cmin = min(cmin, wmin[w]);
    }
    vmax = max(vmax, cmax);
    vmin = min(vmin, cmin);
    // entry j fails if it is zero or not finite, or if the prefix ratio exceeds stab_tol
    const bool bad = valid && (bits == 0 || bits >= kInf ||
                               __longlong_as_double(vmax) > stab_tol * __longlong_as_double(vmin));
    if (bad) atomicMin(&s_width, j);
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) {
      s_cmax = vmax;
      s_cmin = vmin;
    }
    __syncthreads();
  }
  // kappa over all d entries (zero entries give infinity)
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    amax = max(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    amin = min(amin, __shfl_xor_sync(0xffffffffu, amin, o));
  }
  if (lane == 0) {
    wmax[wid] = amax;
    wmin[wid] = amin;
  }
  __syncthreads();
  const int width = s_width;
  for (int i = threadIdx.x; i < d; i += blockDim.x) zz[i] = (i < width) ? z[i] : 0.0;
  // rhat^2 = ||(Q^T g)[width:s]||^2 over the first four warps
  if (wid < 4) {
    double part = 0;
    for (int i = width + threadIdx.x; i < s; i += 128) part += z[i] * z[i];
    part = warp_sum(part);
    if (lane == 0) sh[wid] = part;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    long long mx = 0, mn = kInf;
    for (int w = 0; w < nw; ++w) {
      mx = max(mx, wmax[w]);
      mn = min(mn, wmin[w]);
    }
    const double mna = __longlong_as_double(mn);
    diag[0] = sqrt((sh[0] + sh[1]) + (sh[2] + sh[3]));
    diag[1] = (mna > 0) ? __longlong_as_double(mx) / mna : INFINITY;
    diag[2] = (double)width;
  }
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
      const double rinv = (lane < nb) ? 1.0 / Rb[lane * d + i0 + lane] : 0.0;
      double zl = (lane < nb) ? zz[i0 + lane] : 0.0;
      double yl = 0.0;
      for (int c = nb - 1; c >= 0; --c) {
        if (lane == c) yl = zl * rinv;
        const double yc = __shfl_sync(0xffffffffu, yl, c);
        if (lane < c) zl -= yc * Rb[c * d + i0 + lane];
      }
      if (lane < nb) zz[i0 + lane] = yl;
    }
    __syncthreads();
    // rows above the block: zz[t] -= sum_c R[t, i0+c] y[i0+c], four threads per row
    {
      const int part = threadIdx.x & 3;
      for (int t0 = 0; t0 < i0; t0 += blockDim.x / 4) {
        const int t = t0 + (threadIdx.x >> 2);
        double a = 0;
        if (t < i0)
          for (int c = part; c < nb; c += 4) a += Rb[c * d + t] * zz[i0 + c];
        a += __shfl_xor_sync(0xffffffffu, a, 1);
        a += __shfl_xor_sync(0xffffffffu, a, 2);
        if (t < i0 && part == 0) zz[t] -= a;
      }
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < d; i += blockDim.x) y[i] = (i < width) ? zz[i] : 0.0;
}

sk_status enqueue_ls_solve(const double* Aug, const double* rdiag, int s, int d, double stab_tol, double* y,
                           double* diag, cudaStream_t st, const JobSlab& js, int nj) {
  return enqueue_ls_solve_z(Aug, rdiag, Aug + (size_t)d * s, s, d, stab_tol, y, diag, st, js, nj);
}

sk_status enqueue_ls_solve_z(const double* Aug, const double* rdiag, const double* z, int s, int d, double stab_tol,
                             double* y, double* diag, cudaStream_t st, const JobSlab& js, int nj) {
  const size_t smem = (size_t)d * 33 * sizeof(double);
  if (d < 1 || smem > (size_t)kDynSmemLimit) { set_error("ls_solve: d out of range"); return SK_EINVAL; }
  SK_CUDA(cudaFuncSetAttribute(ls_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kDynSmemLimit));
  ls_solve_kernel<<<dim3(1, nj), kLsThreads, smem, st>>>(Aug, rdiag, z, s, d, stab_tol, y, diag, js);
  SK_CUDA(cudaGetLastError());
  return SK_OK;
}

sk_status enqueue_hbar_product(const double* SB, const double* Hbar, int s, int d, int k, const int* stop,
                               double* Aug, cudaStream_t st, const JobSlab& js, int nj) {
  return enqueue_hbar_product_cols(SB, Hbar, s, d, k, stop, 0, d, Aug, st, js, nj);
}

sk_status enqueue_hbar_product_cols(const double* SB, const double* Hbar, int s, int d, int k, const int* stop,
                                    int c0, int c1, double* Aug, cudaStream_t st, const JobSlab& js, int nj) {
  if (c0 < 0 || c1 > d || c0 >= c1) { set_error("hbar_product: bad column range"); return SK_EINVAL; }
  int blocks = (int)(((int64_t)s * (c1 - c0) + 255) / 256);
  if (blocks > 4 * num_sms()) blocks = 4 * num_sms();
  hbar_product_kernel<<<dim3(blocks, nj), 256, 0, st>>>(SB, Hbar, s, d, k, stop, c0, c1, Aug, js);
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
