// Persistent k-truncated Arnoldi (§1.2.2 eq. (partorth), Algorithm 1 loop,
// double Gram-Schmidt) for grid operators: one cooperative launch builds the
// whole basis of a cycle.
//
// Each CTA owns a contiguous range [c0, c1) of unknowns.  It keeps b_j on
// its range plus one grid row on each side (the 5-point halo) in shared
// memory and m = A b_j for its own unknowns in registers.  One Arnoldi step:
//   phase 1: m = A b_j (from shared memory); partial W^T m, ||m||^2
//            -> grid barrier -> every CTA sums all partials (same order)
//   phase 2: w = m - W h1; partial W^T w, ||w||^2 -> barrier -> h2, nu
//   phase 3: b_{j+1} = (m - W(h1+h2))/nu on its range (written to B), and on
//            its two halo rows recomputed from b_j read back from B (written
//            by the neighbours two barriers earlier), so the next phase 1
//            needs no barrier.  Halo values are computed by the same
//            function, in the same order, as the owner computes them, so
//            they are bit-identical.
// HBM traffic per step: one basis vector written, plus halo and window reads
// that hit L2.  Grid barriers spin on a generation counter with a bounded
// iteration count; a CTA that gives up sets the error word and returns, and
// the others give up at their next barrier.
#include <cmath>

#include "basis.cuh"
#include "common.cuh"

namespace sk {

static constexpr int kPThreads = 512;

__device__ __forceinline__ float fmac(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmac(double a, double b, double c) { return __fma_rn(a, b, c); }

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

struct PersistCtl {
  unsigned* bar_count;  // zeroed before the launch
  unsigned* bar_gen;    // zeroed before the launch
  int* err;             // SK_ETIMEOUT on a barrier timeout
  long long spin_limit;
};

// Grid barrier with acquire/release ordering; false if this CTA gave up.
__device__ bool grid_sync(const PersistCtl& c, unsigned& gen) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned target = gen + 1;
    bool ok = true;
    __threadfence();
    const unsigned prev = atomicAdd(c.bar_count, 1u);
    if (prev == gridDim.x - 1) {
      atomicExch(c.bar_count, 0u);
      __threadfence();
      atomicExch(c.bar_gen, target);
    } else {
      long long it = 0;
      while (ld_acquire(c.bar_gen) != target) {
        if (++it > c.spin_limit) { atomicExch(c.err, (int)SK_ETIMEOUT); ok = false; break; }
        if (*((volatile int*)c.err) != 0) { ok = false; break; }
        __nanosleep(20);
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  gen += 1;
  return s_ok != 0;
}

template <typename C>
struct GridOp {
  int kind;  // OP_STENCIL5 or OP_DIFFUSION
  int nx, ny;
  C cP, cE, cW, cN, cS;
  const C* shift;  // global, may be NULL
  const C* theta;  // global (diffusion)
};

// (A x)_i with x and theta fetched through the given functors; one fixed
// evaluation order with explicit FMAs so that every caller rounds the same way.
template <typename C, typename FX, typename FT>
__device__ __forceinline__ C op_point(const GridOp<C>& A, int i, FX fx, FT ft) {
  const int iy = i / A.nx;
  const int ix = i - iy * A.nx;
  const C xP = fx(i);
  if (A.kind == OP_STENCIL5) {
    C acc = A.cP * xP;
    if (ix + 1 < A.nx) acc = fmac(A.cE, fx(i + 1), acc);
    if (ix > 0) acc = fmac(A.cW, fx(i - 1), acc);
    if (iy + 1 < A.ny) acc = fmac(A.cN, fx(i + A.nx), acc);
    if (iy > 0) acc = fmac(A.cS, fx(i - A.nx), acc);
    if (A.shift) acc = fmac(A.shift[i], xP, acc);
    return acc;
  } else {
    const C tP = ft(i);
    const C h = (C)0.5;
    C acc = 0;
    acc = (ix + 1 < A.nx) ? fmac(h * (tP + ft(i + 1)), xP - fx(i + 1), acc) : fmac(tP, xP, acc);
    acc = (ix > 0) ? fmac(h * (tP + ft(i - 1)), xP - fx(i - 1), acc) : fmac(tP, xP, acc);
    acc = (iy + 1 < A.ny) ? fmac(h * (tP + ft(i + A.nx)), xP - fx(i + A.nx), acc) : fmac(tP, xP, acc);
    acc = (iy > 0) ? fmac(h * (tP + ft(i - A.nx)), xP - fx(i - A.nx), acc) : fmac(tP, xP, acc);
    return acc;
  }
}

// b_{j+1} = round((m - sum_q h_q b_{j-q}) * inv): one formula for owners and halos.
template <typename T, typename C, int KM>
__device__ __forceinline__ C next_vec(C m, const C (&h)[KM], const C (&bw)[KM], int kw, C inv) {
  C v = m;
#pragma unroll
  for (int q = 0; q < KM; ++q)
    if (q < kw) v = fmac(-h[q], bw[q], v);
  return to_c(from_c<T>(v * inv));
}

struct PersistParams {
  BasisParams bp;
  PersistCtl ctl;
  double* part1;  // 2 x grid x (kMaxK+1): pass-1 partials, alternating by step parity (the
                  // reads of step j and the writes of step j+1 are separated by a grid sync)
  double* part2;  // grid x (kMaxK+1): pass-2 partials (and ||r||^2 before step 0)
};

// Sum K per-CTA partials of every CTA (fixed order, same in all CTAs);
// result broadcast to all threads.
template <int K, typename V>
__device__ __forceinline__ void all_partials(const V* part, int nblk, V (&tot)[K], V* sh, V* bc) {
  V v[K];
#pragma unroll
  for (int q = 0; q < K; ++q) v[q] = 0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
#pragma unroll
    for (int q = 0; q < K; ++q) v[q] += __ldcg(part + b * K + q);
  }
  block_sum_k<K>(v, sh);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < K; ++q) bc[q] = v[q];
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < K; ++q) tot[q] = bc[q];
  __syncthreads();
}

template <typename T, int KM, int EPT>
__global__ void __launch_bounds__(kPThreads, 1)
arnoldi_persistent_kernel(PersistParams pp, GridOp<typename Compute<T>::type> A) {
  using C = typename Compute<T>::type;
  constexpr int K1 = KM + 1;
  const BasisParams& p = pp.bp;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double shr[K1 * (kPThreads / 32)];
  __shared__ double bc[K1];
  __shared__ C s_red[K1 * (kPThreads / 32)];
  __shared__ C s_bc[K1];
  __shared__ C s_h[KM + 2];  // step coefficients h (KM), 1/nu, breakdown flag
  const int n = (int)p.n;
  const int nx = A.nx;
  const int chunk = (n + gridDim.x - 1) / gridDim.x;
  const int c0 = min(n, (int)blockIdx.x * chunk);
  const int c1 = min(n, c0 + chunk);
  const int lo = max(0, c0 - nx), hi = min(n, c1 + nx);  // staged range [lo, hi)
  const int span = chunk + 2 * nx;
  C* X = (C*)smem_raw;            // b_j on [lo, hi)
  C* Xn = X + span;               // b_{j+1} being formed (double buffer)
  C* TH = Xn + span;              // theta on [lo, hi) (diffusion)
  auto fx_s = [&](int i) -> C { return X[i - lo]; };
  auto ft_s = [&](int i) -> C { return TH[i - lo]; };
  auto ft_g = [&](int i) -> C { return A.theta[i]; };
  unsigned gen = 0;

  if (A.kind == OP_DIFFUSION)
    for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) TH[i - lo] = A.theta[i];

  // ---- b_0 = r / ||r|| ---------------------------------------------------------
  {
    double a[K1];
#pragma unroll
    for (int q = 0; q < K1; ++q) a[q] = 0;
    for (int e = 0; e < EPT; ++e) {
      const int i = c0 + threadIdx.x + e * kPThreads;
      if (i < c1) a[KM] += p.r[i] * p.r[i];
    }
    block_sum_k<K1>(a, shr);
    if (threadIdx.x == 0) {
#pragma unroll
      for (int q = 0; q < K1; ++q) pp.part2[blockIdx.x * K1 + q] = a[q];
    }
    if (!grid_sync(pp.ctl, gen)) return;
    double tot[K1];
    all_partials<K1>(pp.part2, gridDim.x, tot, shr, bc);
    if (threadIdx.x == 0) bc[0] = 1.0 / sqrt(tot[KM]);  // once per CTA: FP64 sqrt and divide are slow
    __syncthreads();
    const double inv = bc[0];
    T* b0 = (T*)p.B;
    for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) {
      const C v = to_c(from_c<T>((C)(p.r[i] * inv)));
      X[i - lo] = v;
      if (i >= c0 && i < c1) b0[i] = from_c<T>(v);
    }
    __syncthreads();
  }

  C cur[EPT], m[EPT];
#pragma unroll
  for (int e = 0; e < EPT; ++e) {
    const int i = c0 + threadIdx.x + e * kPThreads;
    cur[e] = (i < c1) ? X[i - lo] : (C)0;
  }

  for (int j = 0; j < p.d; ++j) {
    const int kw = min(p.k, j + 1);
    // ---- phase 1 ----------------------------------------------------------------
    C acc[K1];
#pragma unroll
    for (int q = 0; q < K1; ++q) acc[q] = 0;
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
      const int i = c0 + threadIdx.x + e * kPThreads;
      if (i < c1) {
        m[e] = op_point<C>(A, i, fx_s, ft_s);
        acc[0] = fmac(cur[e], m[e], acc[0]);
#pragma unroll
        for (int q = 1; q < KM; ++q)
          if (q < kw) acc[q] = fmac(to_c(__ldcg((const T*)p.B + (int64_t)(j - q) * p.ldb + i)), m[e], acc[q]);
        acc[KM] = fmac(m[e], m[e], acc[KM]);
      } else {
        m[e] = 0;
      }
    }
    block_sum_k<K1>(acc, s_red);
    C* part1 = reinterpret_cast<C*>(pp.part1 + (j & 1) * (int64_t)gridDim.x * (kMaxK + 1));
    C* part2 = reinterpret_cast<C*>(pp.part2);
    if (threadIdx.x == 0) {
#pragma unroll
      for (int q = 0; q < K1; ++q) part1[blockIdx.x * K1 + q] = acc[q];
    }
    if (!grid_sync(pp.ctl, gen)) return;
    // sums in the compute type (the per-CTA partials carry its precision)
    C h1c[K1];
    all_partials<K1>(part1, gridDim.x, h1c, s_red, s_bc);
    C h2c[K1];
#pragma unroll
    for (int q = 0; q < K1; ++q) h2c[q] = 0;
    C h[KM];
    if (p.passes == 2) {
      // ---- phase 2 --------------------------------------------------------------
      C h1[KM];
#pragma unroll
      for (int q = 0; q < KM; ++q) h1[q] = (q < kw) ? h1c[q] : (C)0;
#pragma unroll
      for (int q = 0; q < K1; ++q) acc[q] = 0;
#pragma unroll
      for (int e = 0; e < EPT; ++e) {
        const int i = c0 + threadIdx.x + e * kPThreads;
        if (i < c1) {
          C bw[KM];
          bw[0] = cur[e];
#pragma unroll
          for (int q = 1; q < KM; ++q)
            bw[q] = (q < kw) ? to_c(__ldcg((const T*)p.B + (int64_t)(j - q) * p.ldb + i)) : (C)0;
          C w = m[e];
#pragma unroll
          for (int q = 0; q < KM; ++q) w = fmac(-h1[q], bw[q], w);
#pragma unroll
          for (int q = 0; q < KM; ++q) acc[q] = fmac(bw[q], w, acc[q]);
          acc[KM] = fmac(w, w, acc[KM]);
        }
      }
      block_sum_k<K1>(acc, s_red);
      if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < K1; ++q) part2[blockIdx.x * K1 + q] = acc[q];
      }
      if (!grid_sync(pp.ctl, gen)) return;
      all_partials<K1>(part2, gridDim.x, h2c, s_red, s_bc);
    }
    // ---- finalise step j: thread 0 of every CTA (identical arithmetic), broadcast ----
    if (threadIdx.x == 0) {
      double h1d[KM], h2d[KM];
      double ww;
      for (int q = 0; q < KM; ++q) {
        h1d[q] = (q < kw) ? (double)h1c[q] : 0.0;
        h2d[q] = (q < kw && p.passes == 2) ? (double)h2c[q] : 0.0;
      }
      const double mn2 = (double)h1c[KM];
      if (p.passes == 2) {
        ww = (double)h2c[KM];
      } else {
        // one classical pass: ||w||^2 = ||m||^2 - ||h1||^2 (W_j orthonormal)
        ww = mn2;
        for (int q = 0; q < kw; ++q) ww -= h1d[q] * h1d[q];
      }
      double h2sq = 0;
      for (int q = 0; q < kw; ++q) h2sq += h2d[q] * h2d[q];
      const double nu2 = ww - h2sq;
      const bool brk = !(nu2 > p.bd * p.bd * mn2) || !(mn2 > 0) || !isfinite(nu2);
      const C nuc = brk ? (C)0 : sqrt((C)nu2);
      for (int q = 0; q < KM; ++q) s_h[q] = (q < kw) ? (C)(h1d[q] + h2d[q]) : (C)0;
      s_h[KM] = brk ? (C)0 : (C)1 / nuc;
      s_h[KM + 1] = brk ? (C)1 : (C)0;
      if (blockIdx.x == 0) {
        const double nu = (double)nuc;
        for (int q = 0; q < kw; ++q) {
          p.h1[j * p.k + q] = h1d[q];
          p.h2[j * p.k + q] = h2d[q];
        }
        p.mn2[j] = mn2;
        p.nu[j] = nu;
        if (!isfinite(nu2) || !isfinite(mn2)) *p.nanflag = 1;
        if (p.Hbar) {
          double* col = p.Hbar + (int64_t)j * (p.d + 1);
          for (int q = 0; q < kw; ++q) col[j - q] = h1d[q] + h2d[q];
          col[j + 1] = nu;
        }
        if (brk) *p.stop = j + 1;
      }
    }
    __syncthreads();
    if (s_h[KM + 1] != (C)0) return;
#pragma unroll
    for (int q = 0; q < KM; ++q) h[q] = s_h[q];
    const C inv = s_h[KM];
    // ---- phase 3: b_{j+1} on the owned range and on the halo rows ----------------------
    T* bnext = (T*)p.B + (int64_t)(j + 1) * p.ldb;
    const T* bj = (const T*)p.B + (int64_t)j * p.ldb;
    auto fx_g = [&](int i) -> C { return to_c(__ldcg(bj + i)); };
    C nb[EPT];
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
      const int i = c0 + threadIdx.x + e * kPThreads;
      if (i < c1) {
        C bw[KM];
        bw[0] = cur[e];
#pragma unroll
        for (int q = 1; q < KM; ++q)
          bw[q] = (q < kw) ? to_c(__ldcg((const T*)p.B + (int64_t)(j - q) * p.ldb + i)) : (C)0;
        nb[e] = next_vec<T, C, KM>(m[e], h, bw, kw, inv);
        bnext[i] = from_c<T>(nb[e]);
      } else {
        nb[e] = 0;
      }
    }
    // halo rows [lo, c0) and [c1, hi), from b_j in global memory
    const int nlo = c0 - lo, nhi = hi - c1;
    for (int t = threadIdx.x; t < nlo + nhi; t += blockDim.x) {
      const int i = t < nlo ? lo + t : c1 + (t - nlo);
      C bw[KM];
#pragma unroll
      for (int q = 0; q < KM; ++q)
        bw[q] = (q < kw) ? to_c(__ldcg((const T*)p.B + (int64_t)(j - q) * p.ldb + i)) : (C)0;
      const C mh = op_point<C>(A, i, fx_g, ft_g);
      Xn[i - lo] = next_vec<T, C, KM>(mh, h, bw, kw, inv);
    }
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
      const int i = c0 + threadIdx.x + e * kPThreads;
      if (i < c1) Xn[i - lo] = nb[e];
      cur[e] = nb[e];
    }
    __syncthreads();
    C* tmp = X;
    X = Xn;
    Xn = tmp;
  }
}

// ---- host side ---------------------------------------------------------------------
template <typename T, int KM, int EPT>
static sk_status launch_persist_t(const PersistParams& pp, const GridOp<typename Compute<T>::type>& A, int grid,
                                  size_t smem, cudaStream_t st) {
  auto kern = arnoldi_persistent_kernel<T, KM, EPT>;
  SK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kDynSmemLimit));
  int per_sm = 0;
  SK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kPThreads, smem));
  if (per_sm * num_sms() < grid) {
    set_error("persistent basis: %d CTAs cannot be co-resident", grid);
    return SK_EINVAL;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kPThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  SK_CUDA(cudaLaunchKernelEx(&cfg, kern, pp, A));
  return SK_OK;
}

template <typename T, int EPT>
static sk_status launch_persist_k(const PersistParams& pp, const GridOp<typename Compute<T>::type>& A, int grid,
                                  size_t smem, cudaStream_t st) {
  if (pp.bp.k <= 2) return launch_persist_t<T, 2, EPT>(pp, A, grid, smem, st);
  return launch_persist_t<T, 4, EPT>(pp, A, grid, smem, st);  // persist_shape admits k <= 4
}

template <typename T>
static sk_status launch_persist_e(const PersistParams& pp, const GridOp<typename Compute<T>::type>& A, int grid,
                                  int ept, size_t smem, cudaStream_t st) {
  switch (ept) {
    case 1: return launch_persist_k<T, 1>(pp, A, grid, smem, st);
    case 2: return launch_persist_k<T, 2>(pp, A, grid, smem, st);
    case 4: return launch_persist_k<T, 4>(pp, A, grid, smem, st);
    case 8: return launch_persist_k<T, 8>(pp, A, grid, smem, st);
    default: return launch_persist_k<T, 16>(pp, A, grid, smem, st);
  }
}

// Geometry of the persistent launch; false if the problem does not fit.  The
// opt-in persistent path covers k <= 4 with FP32 or FP64 storage (other
// cases use the three-launch path), which keeps its instantiations few.
bool persist_shape(const sk_op* op, sk_dtype dt, int k, int* grid, int* ept, size_t* smem) {
  if (!(op->kind == OP_STENCIL5 || op->kind == OP_DIFFUSION)) return false;
  if (k > 4 || dt == SK_BF16) return false;
  if (op->n >= (1ll << 30)) return false;
  const int64_t n = op->n;
  int g = num_sms();
  const int64_t per = (n + g - 1) / g;
  if (per < 2 * kPThreads && g > 1) {
    // small problems: fewer CTAs, about 2 elements per thread
    g = (int)((n + 2 * kPThreads - 1) / (2 * kPThreads));
    if (g < 1) g = 1;
  }
  const int64_t chunk = (n + g - 1) / g;
  int e = 1;
  while ((int64_t)e * kPThreads < chunk) e *= 2;
  if (e > 16) return false;
  const size_t csize = dt == SK_F64 ? 8 : 4;
  const size_t words = (size_t)(chunk + 2 * op->nx) * (op->kind == OP_DIFFUSION ? 3 : 2);
  const size_t sm = words * csize;
  if (sm > 200 * 1024) return false;
  *grid = g;
  *ept = e;
  *smem = sm;
  return true;
}

sk_status enqueue_basis_persistent(const BasisParams& bp, const sk_op* op, PersistWork& w, cudaStream_t st) {
  int grid = 0, ept = 0;
  size_t smem = 0;
  if (!persist_shape(op, bp.dtype, bp.k, &grid, &ept, &smem)) { set_error("persistent basis: shape"); return SK_EINVAL; }
  PersistParams pp;
  pp.bp = bp;
  pp.ctl.bar_count = w.bar;
  pp.ctl.bar_gen = w.bar + 1;
  pp.ctl.err = w.err;
  pp.ctl.spin_limit = w.spin_limit;
  pp.part1 = w.part;
  pp.part2 = w.part + (size_t)2 * grid * (kMaxK + 1);
  SK_CUDA(cudaMemsetAsync(w.bar, 0, 2 * sizeof(unsigned), st));
  if (bp.dtype == SK_F64) {
    OpView<double> v;
    make_view(op, &v);
    GridOp<double> A{v.kind, v.nx, v.ny, v.cP, v.cE, v.cW, v.cN, v.cS, v.shift, v.theta};
    return launch_persist_e<double>(pp, A, grid, ept, smem, st);
  }
  OpView<float> v;
  SK_TRY(make_view(op, &v, st));
  GridOp<float> A{v.kind, v.nx, v.ny, v.cP, v.cE, v.cW, v.cN, v.cS, v.shift, v.theta};
  return launch_persist_e<float>(pp, A, grid, ept, smem, st);
}

}  // namespace sk
