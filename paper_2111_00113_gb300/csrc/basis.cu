// k-truncated Arnoldi basis (§1.2.2 eq. (partorth); Algorithm 1 loop with
// "double Gram-Schmidt"; §4.2).
//
// One Arnoldi step j (0-based; window W_j = {b_j, ..., b_{j-kw+1}},
// kw = min(k, j+1)) is three grid-wide passes, each ending in a deterministic
// last-block reduction of per-CTA partials:
//   dots1(j):  m = A b_j;      h1 = W_j^T m,  ||m||^2
//   dots2(j):  m = A b_j;  w = m - W_j h1;  h2 = W_j^T w,  ||w||^2
//              nu_j = sqrt(||w||^2 - ||h2||^2)   (W_j is orthonormal: its
//              vectors were orthogonalised against each other, |i-j| < k)
//   form(j+1): b_{j+1} = (A b_j - W_j (h1 + h2)) / nu_j
// With an FP32/BF16 basis, m = A b_j is recomputed from the stored b_j in
// each pass (a 5-point product costs less than writing and re-reading a
// vector).  With an FP64 basis the FP64 pipe is the bound on this part, so
// dots1 stores m once (FP64) and the other passes read it.
// The Arnoldi coefficients are kept: A b_j = sum_q (h1+h2)_q b_{j-q} +
// nu_j b_{j+1}, i.e. AB_d = B_{d+1} Hbar with Hbar (d+1) x d, k+1 diagonals.
//
// Constant-coefficient stencils take a vector path: each thread handles
// groups of 4 consecutive cells with 16-byte loads.  When nx % 4 == 0 the
// group lies in one grid row and its north and south neighbours are aligned
// groups too; otherwise those are single loads, a group may wrap into the
// next row, and when n % 4 != 0 the last group reads zeros past n and writes
// nothing there.  Other operators take the scalar path.
#include <cmath>

#include "basis.cuh"
#include "common.cuh"
#include "grouped.cuh"

namespace sk {

template <typename T>
__device__ __forceinline__ T* bcol(void* B, int64_t ldb, int c) {
  return (T*)B + (int64_t)c * ldb;
}

// ---- groups of G consecutive elements ---------------------------------------
template <typename C>
__device__ __forceinline__ void ld4(const float* p, C (&v)[4]) {
  const float4 t = *reinterpret_cast<const float4*>(p);
  v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
template <typename C>
__device__ __forceinline__ void ld4(const double* p, C (&v)[4]) {
  const double2 a = *reinterpret_cast<const double2*>(p);
  const double2 b = *reinterpret_cast<const double2*>(p + 2);
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
template <typename C>
__device__ __forceinline__ void ld4(const __nv_bfloat16* p, C (&v)[4]) {
  const uint2 u = *reinterpret_cast<const uint2*>(p);
  const __nv_bfloat162 a = *reinterpret_cast<const __nv_bfloat162*>(&u.x);
  const __nv_bfloat162 b = *reinterpret_cast<const __nv_bfloat162*>(&u.y);
  const float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
  v[0] = fa.x; v[1] = fa.y; v[2] = fb.x; v[3] = fb.y;
}
__device__ __forceinline__ void st4(float* p, const float (&v)[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void st4(double* p, const double (&v)[4]) {
  *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
  *reinterpret_cast<double2*>(p + 2) = make_double2(v[2], v[3]);
}
__device__ __forceinline__ void st4(__nv_bfloat16* p, const float (&v)[4]) {
  uint2 u;
  *reinterpret_cast<__nv_bfloat162*>(&u.x) = __floats2bfloat162_rn(v[0], v[1]);
  *reinterpret_cast<__nv_bfloat162*>(&u.y) = __floats2bfloat162_rn(v[2], v[3]);
  *reinterpret_cast<uint2*>(p) = u;
}

template <int G, typename T, typename C>
__device__ __forceinline__ void gload(const T* p, int64_t i, C (&v)[G]) {
  if constexpr (G == 4) ld4(p + i, v);
  else v[0] = to_c(p[i]);
}
template <int G, typename T, typename C>
__device__ __forceinline__ void gstore(T* p, int64_t i, const C (&v)[G]) {
  if constexpr (G == 4) st4(p + i, v);
  else p[i] = from_c<T>(v[0]);
}

// GUARD: the vector path across rows also serves n % 4 != 0; its last group
// (the one holding n - 1) reads zeros and writes nothing past n.
template <int G, bool GUARD, typename T, typename C>
__device__ __forceinline__ void gload_n(const T* p, int64_t i, int64_t n, C (&v)[G]) {
  if constexpr (GUARD) {
    if (i + G > n) {
#pragma unroll
      for (int e = 0; e < G; ++e) v[e] = (i + e < n) ? to_c(p[i + e]) : (C)0;
      return;
    }
  }
  gload<G>(p, i, v);
}
template <int G, bool GUARD, typename T, typename C>
__device__ __forceinline__ void gstore_n(T* p, int64_t i, int64_t n, const C (&v)[G]) {
  if constexpr (GUARD) {
    if (i + G > n) {
#pragma unroll
      for (int e = 0; e < G; ++e)
        if (i + e < n) p[i + e] = from_c<T>(v[e]);
      return;
    }
  }
  gstore<G>(p, i, v);
}

// m[0..G) = (A x)[i0..i0+G); G = 4 only for constant-coefficient stencils
// (see the vector path above).
template <int G, bool ROWS, typename T, typename C>
__device__ __forceinline__ void op_apply(const OpView<C>& A, const T* __restrict__ x, int64_t i0, C (&m)[G]) {
  if constexpr (G == 4) {
    int ix0;
    int64_t iy64;
    A.grid_pos(i0, ix0, iy64);
    const int iy = (int)iy64;
    C xc[4], up[4], dn[4];
    ld4(x + i0, xc);
    // explicit fused multiply-adds, left to right: the rounding does not
    // depend on how the compiler contracts the sum in a given kernel
    const C cP = A.cP, cE = A.cE, cW = A.cW, cN = A.cN, cS = A.cS;
    if constexpr (ROWS) {
      // the four cells share one grid row; north and south are aligned groups
      const C w = ix0 > 0 ? to_c(x[i0 - 1]) : (C)0;
      const C e = ix0 + 4 < A.nx ? to_c(x[i0 + 4]) : (C)0;
      if (iy + 1 < A.ny) ld4(x + i0 + A.nx, up);
      else up[0] = up[1] = up[2] = up[3] = 0;
      if (iy > 0) ld4(x + i0 - A.nx, dn);
      else dn[0] = dn[1] = dn[2] = dn[3] = 0;
      m[0] = fma(cS, dn[0], fma(cN, up[0], fma(cW, w, fma(cE, xc[1], cP * xc[0]))));
      m[1] = fma(cS, dn[1], fma(cN, up[1], fma(cW, xc[0], fma(cE, xc[2], cP * xc[1]))));
      m[2] = fma(cS, dn[2], fma(cN, up[2], fma(cW, xc[1], fma(cE, xc[3], cP * xc[2]))));
      m[3] = fma(cS, dn[3], fma(cN, up[3], fma(cW, xc[2], fma(cE, e, cP * xc[3]))));
    } else {
      // any other width: the group may run into the next grid
      // row; cell q sits at (ix0 + q, iy) or, past the row's end, at
      // (ix0 + q - nx, iy + 1); north and south are unaligned single loads,
      // and a neighbour outside the grid contributes zero
      const int64_t n = A.n;
      const C w = i0 > 0 ? to_c(x[i0 - 1]) : (C)0;
      const C e = i0 + 4 < n ? to_c(x[i0 + 4]) : (C)0;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        int cx = ix0 + q, cy = iy;
        if (cx >= A.nx) {
          cx -= A.nx;
          cy += 1;
        }
        const int64_t i = i0 + q;
        const C xe = (cx + 1 < A.nx) ? (q < 3 ? xc[q + 1] : e) : (C)0;
        const C xw = (cx > 0) ? (q > 0 ? xc[q - 1] : w) : (C)0;
        const C xn = (cy + 1 < A.ny) ? to_c(x[i + A.nx]) : (C)0;
        const C xs = (cy > 0) ? to_c(x[i - A.nx]) : (C)0;
        m[q] = fma(cS, xs, fma(cN, xn, fma(cW, xw, fma(cE, xe, cP * xc[q]))));
      }
    }
    if (A.shift) {
      C sh[4];
      if constexpr (ROWS) ld4(A.shift + i0, sh);
      else gload_n<4, true>(A.shift, i0, A.n, sh);
#pragma unroll
      for (int q = 0; q < 4; ++q) m[q] = fma(sh[q], xc[q], m[q]);
    }
    if constexpr (!ROWS) {
      // cells past n (the last group when n % 4 != 0) contribute nothing; x's
      // column padding read there is never used
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (i0 + q >= A.n) m[q] = 0;
    }
  } else {
    m[0] = A.apply(x, i0);
  }
}

// Final reduction in the last block: thread t sums blocks t, t+T, ... (fixed
// assignment), then a fixed-order block reduction, all in the compute type C
// (the per-block partials already carry C's precision; on this GPU FP64
// shuffles and adds cost 64+ cycles each).  Result in thread 0.
template <int K, typename C>
__device__ __forceinline__ void reduce_partials(const C* part, int nblocks, C (&tot)[K], C* sh) {
#pragma unroll
  for (int q = 0; q < K; ++q) tot[q] = 0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
#pragma unroll
    for (int q = 0; q < K; ++q) tot[q] += __ldcg(part + b * K + q);
  }
  block_sum_k<K>(tot, sh);
}

// Step j's coefficients in the compute type (see BasisParams::coef).
template <typename C>
__device__ __forceinline__ C* coef_row(const BasisParams& p, int j) {
  return static_cast<C*>(p.coef) + (int64_t)j * (kMaxK + 1);
}

// ---- kernels ------------------------------------------------------------------
// Each thread handles IterOf<G> groups of G elements.  The passes are launched
// with programmatic dependent launch: a kernel loads every operand that its
// immediate predecessor does not write (b_j is written by form(j), the
// predecessor of dots1(j); the older window vectors and, for dots2 and form,
// b_j itself are older), then waits for the predecessor's results (h1, h2,
// nu, stop; m for FP64) and only then lets its own successor launch, so a
// successor's early loads only ever read what completed kernels wrote.
// kIter<G> groups per thread: 2 groups of 4 cells (vector path) or 8 single
// cells, so every CTA covers 2048 unknowns on either path (fewer, longer
// CTAs: each pass is latency bound, one block reduction per CTA).
template <int G>
struct IterOf {
  static constexpr int value = G == 4 ? 2 : 8;
};

__device__ __forceinline__ void pdl_trigger() {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 900
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
#endif
}
__device__ __forceinline__ void pdl_wait() {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 900
  asm volatile("griddepcontrol.wait;" ::: "memory");
#endif
}

// The passes' bodies take the block index `bid` of `nb` blocks that cover
// the vector: the whole grid of a single-system launch, or one job's blocks
// of a grouped launch.
template <typename T, int KM, int G, bool STORE_M, bool ROWS>
__device__ __forceinline__ void form_body(const BasisParams& p, const OpView<typename Compute<T>::type>& A, int c,
                                          int bid, int nb) {
  constexpr int kIter = IterOf<G>::value;
  constexpr bool GUARD = G == 4 && !ROWS;
  using C = typename Compute<T>::type;
  T* out = bcol<T>(p.B, p.ldb, c);
  const int64_t n = p.n;
  const int64_t stride = (int64_t)nb * blockDim.x * G;
  const int64_t i_begin = ((int64_t)bid * blockDim.x + threadIdx.x) * G;
  if (c == 0) {
    pdl_wait();
    pdl_trigger();
    if (c >= *p.stop) return;
    __shared__ double s_inv;
    if (threadIdx.x == 0) s_inv = 1.0 / sqrt(*p.rho2);  // once per CTA: FP64 sqrt and divide are slow here
    __syncthreads();
    const double inv = s_inv;
    for (int64_t i = i_begin; i < n; i += stride) {
      C v[G];
#pragma unroll
      for (int q = 0; q < G; ++q) v[q] = (!GUARD || i + q < n) ? (C)(p.r[i + q] * inv) : (C)0;
      gstore_n<G, GUARD>(out, i, n, v);
    }
    return;
  }
  const int j = c - 1;
  const int kw = min(p.k, j + 1);
  const T* bj = bcol<T>(p.B, p.ldb, j);
  // prologue: b_j and the window are older than the predecessor (dots2(j));
  // with one Gram-Schmidt pass the predecessor is dots1(j), which writes m
  const bool m_late = STORE_M && p.passes == 1;
  C m[kIter][G];
  C bw[kIter][KM][G];
#pragma unroll
  for (int it = 0; it < kIter; ++it) {
    const int64_t i = i_begin + it * stride;
    if (i < n) {
      if constexpr (STORE_M) {
        if (!m_late) gload_n<G, GUARD>(p.M, i, n, m[it]);
      } else {
        op_apply<G, ROWS>(A, bj, i, m[it]);
      }
#pragma unroll
      for (int q = 0; q < KM; ++q)
        if (q < kw) gload_n<G, GUARD>(bcol<T>(p.B, p.ldb, j - q), i, n, bw[it][q]);
    }
  }
  pdl_wait();
  pdl_trigger();
  if (c >= *p.stop) return;
  if (m_late) {
#pragma unroll
    for (int it = 0; it < kIter; ++it) {
      const int64_t i = i_begin + it * stride;
      if (i < n) gload_n<G, GUARD>(p.M, i, n, m[it]);
    }
  }
  const C* cf = coef_row<C>(p, j);
  C h[KM];
#pragma unroll
  for (int q = 0; q < KM; ++q) h[q] = (q < kw) ? cf[q] : (C)0;
  const C inv = cf[kMaxK];
#pragma unroll
  for (int it = 0; it < kIter; ++it) {
    const int64_t i = i_begin + it * stride;
    if (i < n) {
#pragma unroll
      for (int q = 0; q < KM; ++q) {
        if (q < kw) {
#pragma unroll
          for (int e = 0; e < G; ++e) m[it][e] = fma(-h[q], bw[it][q][e], m[it][e]);
        }
      }
#pragma unroll
      for (int e = 0; e < G; ++e) m[it][e] *= inv;
      gstore_n<G, GUARD>(out, i, n, m[it]);
    }
  }
}

template <typename T, int KM, int G, bool STORE_M, bool ROWS>
__global__ void __launch_bounds__(kBasisThreads)
form_kernel(BasisParams p, OpView<typename Compute<T>::type> A, int c) {
  form_body<T, KM, G, STORE_M, ROWS>(p, A, c, blockIdx.x, gridDim.x);
}

// PASS = 1: dots with m (and m stored if STORE_M);  PASS = 2: dots with
// w = m - W h1.
template <typename T, int KM, int G, bool STORE_M, int PASS, bool ROWS>
__device__ __forceinline__ void dots_body(const BasisParams& p, const OpView<typename Compute<T>::type>& A, int j,
                                          int bid, int nb) {
  constexpr int kIter = IterOf<G>::value;
  constexpr bool GUARD = G == 4 && !ROWS;
  using C = typename Compute<T>::type;
  __shared__ C red[(KM + 1) * (kBasisThreads / 32)];
  const int kw = min(p.k, j + 1);
  const int64_t n = p.n;
  const T* bj = bcol<T>(p.B, p.ldb, j);
  const int64_t stride = (int64_t)nb * blockDim.x * G;
  const int64_t i_begin = ((int64_t)bid * blockDim.x + threadIdx.x) * G;
  C m[kIter][G];
  C bw[kIter][KM][G];
  // prologue: the window b_{j-1..} is old; b_j is old for pass 2 only
#pragma unroll
  for (int it = 0; it < kIter; ++it) {
    const int64_t i = i_begin + it * stride;
#pragma unroll
    for (int q = 0; q < KM; ++q) {
#pragma unroll
      for (int e = 0; e < G; ++e) bw[it][q][e] = 0;
    }
    if (i < n) {
#pragma unroll
      for (int q = (PASS == 1 ? 1 : 0); q < KM; ++q)
        if (q < kw) gload_n<G, GUARD>(bcol<T>(p.B, p.ldb, j - q), i, n, bw[it][q]);
      if (PASS == 2 && !STORE_M) op_apply<G, ROWS>(A, bj, i, m[it]);
    }
  }
  pdl_wait();
  pdl_trigger();
  if (j >= *p.stop) return;
  C h[KM];
  if (PASS == 2) {
    const C* cf = coef_row<C>(p, j);  // h1 in the compute type, written by pass 1
#pragma unroll
    for (int q = 0; q < KM; ++q) h[q] = (q < kw) ? cf[q] : (C)0;
  }
  C acc[KM + 1];
#pragma unroll
  for (int q = 0; q <= KM; ++q) acc[q] = 0;
#pragma unroll
  for (int it = 0; it < kIter; ++it) {
    const int64_t i = i_begin + it * stride;
    if (i < n) {
      if (PASS == 1) {
        gload_n<G, GUARD>(bj, i, n, bw[it][0]);
        op_apply<G, ROWS>(A, bj, i, m[it]);
        if (STORE_M) {
          double md[G];
#pragma unroll
          for (int e = 0; e < G; ++e) md[e] = (double)m[it][e];
          gstore_n<G, GUARD>(p.M, i, n, md);
        }
      } else if (STORE_M) {
        gload_n<G, GUARD>(p.M, i, n, m[it]);
      }
      if (PASS == 2) {
#pragma unroll
        for (int q = 0; q < KM; ++q) {
#pragma unroll
          for (int e = 0; e < G; ++e) m[it][e] = fma(-h[q], bw[it][q][e], m[it][e]);
        }
      }
#pragma unroll
      for (int q = 0; q < KM; ++q) {
#pragma unroll
        for (int e = 0; e < G; ++e) acc[q] = fma(bw[it][q][e], m[it][e], acc[q]);
      }
#pragma unroll
      for (int e = 0; e < G; ++e) acc[KM] = fma(m[it][e], m[it][e], acc[KM]);
    }
  }
  block_sum_k<KM + 1>(acc, red);
  C* part = reinterpret_cast<C*>(p.partial);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q <= KM; ++q) part[bid * (KM + 1) + q] = acc[q];
  }
  if (!last_block_arrived_n(p.counters + (PASS - 1), (unsigned)nb)) return;
  C tc[KM + 1];
  reduce_partials<KM + 1>(part, nb, tc, red);
  if (threadIdx.x != 0) return;
  C* cf = coef_row<C>(p, j);
  double tot[KM + 1];
#pragma unroll
  for (int q = 0; q <= KM; ++q) tot[q] = (double)tc[q];
  if (PASS == 1) {
    for (int q = 0; q < kw; ++q) {
      p.h1[j * p.k + q] = tot[q];
      cf[q] = tc[q];
    }
    p.mn2[j] = tot[KM];
    if (!isfinite(tot[KM])) *p.nanflag = 1;
    if (p.passes == 2) return;
    // single classical pass: ||w||^2 = ||m||^2 - ||h1||^2 (W_j orthonormal)
    for (int q = 0; q < kw; ++q) p.h2[j * p.k + q] = 0;
    double hh = 0;
    for (int q = 0; q < kw; ++q) hh += tot[q] * tot[q];
    tot[KM] = tot[KM] - hh;
    for (int q = 0; q < kw; ++q) tot[q] = 0;
  } else {
    for (int q = 0; q < kw; ++q) p.h2[j * p.k + q] = tot[q];
  }
  // finalise step j: nu_j, the Hessenberg column and the form pass's coefficients
  double h2sq = 0;
  for (int q = 0; q < kw; ++q) h2sq += tot[q] * tot[q];
  const double nu2 = tot[KM] - h2sq;
  const double mn2 = p.mn2[j];
  bool brk = !(nu2 > p.bd * p.bd * mn2) || !(mn2 > 0);
  if (!isfinite(nu2)) { *p.nanflag = 1; brk = true; }
  const C nuc = brk ? (C)0 : sqrt((C)nu2);
  const double nu = (double)nuc;
  p.nu[j] = nu;
  for (int q = 0; q < kw; ++q) {
    const double hs = p.h1[j * p.k + q] + p.h2[j * p.k + q];
    cf[q] = (C)hs;
    if (p.Hbar) p.Hbar[(int64_t)j * (p.d + 1) + j - q] = hs;
  }
  cf[kMaxK] = brk ? (C)0 : (C)1 / nuc;
  if (p.Hbar) p.Hbar[(int64_t)j * (p.d + 1) + j + 1] = nu;
  if (brk) *p.stop = j + 1;
}

template <typename T, int KM, int G, bool STORE_M, int PASS, bool ROWS>
__global__ void __launch_bounds__(kBasisThreads)
dots_kernel(BasisParams p, OpView<typename Compute<T>::type> A, int j) {
  dots_body<T, KM, G, STORE_M, PASS, ROWS>(p, A, j, blockIdx.x, gridDim.x);
}

// ---- grouped passes (batched solver) -------------------------------------------
// map[blockIdx.x] = {slot, block of that job}; the job's vector path picks
// the body instantiation (the branch is uniform over the CTA).  The map and
// the job array are written before the cycle, so the prologue may read them
// before the programmatic wait.
template <typename T, int KM, bool STORE_M>
__global__ void __launch_bounds__(kBasisThreads)
g_form_kernel(const GJob* __restrict__ jobs, const int2* __restrict__ map, int c) {
  using C = typename Compute<T>::type;
  const int2 m = map[blockIdx.x];
  const GJob& J = jobs[m.x];
  const BasisParams& p = J.bp;
  const OpView<C>& A = job_view<C>(J);
  if (J.vec == 1) form_body<T, KM, 4, STORE_M, true>(p, A, c, m.y, p.nblk);
  else if (J.vec == 2) form_body<T, KM, 4, STORE_M, false>(p, A, c, m.y, p.nblk);
  else form_body<T, KM, 1, STORE_M, true>(p, A, c, m.y, p.nblk);
}

template <typename T, int KM, bool STORE_M, int PASS>
__global__ void __launch_bounds__(kBasisThreads)
g_dots_kernel(const GJob* __restrict__ jobs, const int2* __restrict__ map, int j) {
  using C = typename Compute<T>::type;
  const int2 m = map[blockIdx.x];
  const GJob& J = jobs[m.x];
  const BasisParams& p = J.bp;
  const OpView<C>& A = job_view<C>(J);
  if (J.vec == 1) dots_body<T, KM, 4, STORE_M, PASS, true>(p, A, j, m.y, p.nblk);
  else if (J.vec == 2) dots_body<T, KM, 4, STORE_M, PASS, false>(p, A, j, m.y, p.nblk);
  else dots_body<T, KM, 1, STORE_M, PASS, true>(p, A, j, m.y, p.nblk);
}

// prio != 0 gives the launch that priority (the pipelined cycle raises the
// basis passes above the sketch and QR work that runs beside them).
template <typename K, typename... Args>
static cudaError_t launch_pdl(K kernel, int grid, cudaStream_t st, bool pdl, int prio, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kBasisThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  int na = 0;
  if (pdl) {
    attr[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[na].val.programmaticStreamSerializationAllowed = 1;
    ++na;
  }
  if (prio != 0) {
    attr[na].id = cudaLaunchAttributePriority;
    attr[na].val.priority = prio;
    ++na;
  }
  cfg.attrs = attr;
  cfg.numAttrs = na;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// ---- Chebyshev basis (§4.3, eq. (Chebrecurse)) -------------------------------
// With rho = max(dx, dy) and gamma = (dx^2 - dy^2)/(4 rho), the paper's
// recurrence u_2 = (A - c) u_1 / (2 rho), u_{j+1} = ((A - c) u_j - gamma
// u_{j-1}) / rho shrinks like 2^-j; B stores v_j = 2^j u_j (0-based), the
// same vectors scaled by exact powers of two (so FP32 storage neither
// underflows nor differs from the paper's recurrence by more than rounding):
//   v_1 = (A - c) v_0 / rho,   v_{j+1} = ((A - c) v_j - 2 gamma v_{j-1}) * 2 / rho.
// Hence A v_0 = c v_0 + rho v_1 and A v_j = c v_j + (rho/2) v_{j+1} + 2 gamma
// v_{j-1}.  No inner products: one launch per vector, which also leaves its
// per-CTA partial sums of ||v_j||^2 for the unit rescaling (done once per
// basis by cheb_finalize_kernel, and applied through Hbar and the update
// coefficients instead of rewriting B).
template <typename T, int G>
__global__ void __launch_bounds__(kBasisThreads)
cheb_kernel(BasisParams p, OpView<typename Compute<T>::type> A, int c) {
  constexpr int kIter = IterOf<G>::value;
  constexpr bool ROWS = true;  // the Chebyshev basis takes the vector path only when nx % 4 == 0
  using C = typename Compute<T>::type;
  __shared__ C red[2 * (kBasisThreads / 32)];
  const int64_t n = p.n;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x * G;
  const int64_t i_begin = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * G;
  const T* v1 = bcol<T>(p.B, p.ldb, c - 1);
  const T* v2 = bcol<T>(p.B, p.ldb, c >= 2 ? c - 2 : 0);
  T* out = bcol<T>(p.B, p.ldb, c);
  // prologue: v_{c-2} is older than the predecessor, which writes v_{c-1}
  C x2[kIter][G];
#pragma unroll
  for (int it = 0; it < kIter; ++it) {
    const int64_t i = i_begin + it * stride;
#pragma unroll
    for (int e = 0; e < G; ++e) x2[it][e] = 0;
    if (i < n && c >= 2) gload<G>(v2, i, x2[it]);
  }
  pdl_wait();
  pdl_trigger();
  if (c >= *p.stop) return;
  const C cc = (C)p.cheb_c;
  const C al = (C)(c == 1 ? 1.0 / p.cheb_rho : 2.0 / p.cheb_rho);
  const C be = (C)(c == 1 ? 0.0 : 2.0 * p.cheb_gamma);
  C acc[2] = {0, 0};  // ||v_c||^2 and, for c = 1, ||v_0||^2
#pragma unroll
  for (int it = 0; it < kIter; ++it) {
    const int64_t i = i_begin + it * stride;
    if (i < n) {
      C m[G], x1[G], v[G];
      op_apply<G, ROWS>(A, v1, i, m);
      gload<G>(v1, i, x1);
#pragma unroll
      for (int e = 0; e < G; ++e) v[e] = ((m[e] - cc * x1[e]) - be * x2[it][e]) * al;
      gstore<G>(out, i, v);
#pragma unroll
      for (int e = 0; e < G; ++e) {
        const C vs = to_c(from_c<T>(v[e]));  // the value B holds
        acc[0] += vs * vs;
        acc[1] += x1[e] * x1[e];
      }
    }
  }
  block_sum_k<2>(acc, red);
  if (threadIdx.x == 0) {
    C* part = reinterpret_cast<C*>(p.cheb_part);
    part[(int64_t)c * p.nblk_cap + blockIdx.x] = acc[0];
    if (c == 1) part[blockIdx.x] = acc[1];
  }
}

// One CTA per column j = 0..d: sigma_j = ||v_j|| from the partials (fixed
// order), column j of Hbar = H_v[:, j] / sigma_j.  A zero or non-finite norm
// ends the basis at j columns.
template <typename C>
__global__ void __launch_bounds__(kBasisThreads) cheb_finalize_kernel(BasisParams p, int nblk, int j0) {
  __shared__ C red[kBasisThreads / 32];
  const int j = j0 + blockIdx.x;
  const C* part = reinterpret_cast<const C*>(p.cheb_part) + (int64_t)j * p.nblk_cap;
  C t[1] = {0};
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) t[0] += part[b];
  block_sum_k<1>(t, red);
  if (threadIdx.x != 0) return;
  const double sig = sqrt((double)t[0]);
  p.sigma[j] = sig;
  const bool ok = sig > 0 && isfinite(sig);
  if (!isfinite(sig)) *p.nanflag = 1;
  if (!ok) atomicMin(p.stop, j);
  if (j < p.d && p.Hbar) {
    double* col = p.Hbar + (int64_t)j * (p.d + 1);
    const double inv = ok ? 1.0 / sig : 0.0;
    col[j] = p.cheb_c * inv;
    col[j + 1] = (j == 0 ? p.cheb_rho : 0.5 * p.cheb_rho) * inv;
    if (j >= 1) col[j - 1] = 2.0 * p.cheb_gamma * inv;
  }
}

template <typename T, int G>
static sk_status enqueue_cheb_t(const BasisParams& p, const OpView<typename Compute<T>::type>& A, cudaStream_t st) {
  using C = typename Compute<T>::type;
  const int g = p.nblk;
  // steps [j_begin, j_end) form v_{j_begin+1} .. v_{j_end} (j_end = 0: all d;
  // then the norms are finalised here too, else by enqueue_cheb_finalize)
  const int jb = p.j_begin, je = p.j_end > 0 ? p.j_end : p.d;
  if (jb == 0)
    SK_CUDA(launch_pdl(form_kernel<T, 2, G, false, true>, g, st, false, p.prio, p, A, 0));  // v_0 = r/||r||
  for (int c = jb + 1; c <= je; ++c)
    SK_CUDA(launch_pdl(cheb_kernel<T, G>, g, st, jb == 0 || c > jb + 1 || p.pdl_resume, p.prio, p, A, c));
  if (p.j_end == 0) {
    cheb_finalize_kernel<C><<<p.d + 1, kBasisThreads, 0, st>>>(p, g, 0);
    SK_CUDA(cudaGetLastError());
  }
  return SK_OK;
}


// Unit columns for callers of the basis itself: B[:, j] /= sigma_j and
// Hbar[i, j] *= sigma_i (Hbar then relates the unit columns).
template <typename T>
__global__ void cheb_scale_cols_kernel(BasisParams p) {
  using C = typename Compute<T>::type;
  T* B = static_cast<T*>(p.B);
  const int64_t total = p.n * (int64_t)(p.d + 1);
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(q / p.n);
    const int64_t i = q - (int64_t)j * p.n;
    if (j >= *p.stop) continue;
    T* e = B + (int64_t)j * p.ldb + i;
    *e = from_c<T>((C)((double)to_c(*e) / p.sigma[j]));
  }
}
__global__ void cheb_scale_hbar_kernel(BasisParams p) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < (p.d + 1) * p.d; q += gridDim.x * blockDim.x) {
    const int i = q % (p.d + 1);
    if (i < *p.stop) p.Hbar[q] *= p.sigma[i];
  }
}

sk_status enqueue_cheb_finalize(const BasisParams& p, const sk_op* op, int j0, int j1, cudaStream_t st) {
  if (j1 <= j0) return SK_OK;
  const bool cvec = basis_vector_path(op, p.ldb, p.B) && (p.r == nullptr || ((uintptr_t)p.r % 16) == 0) &&
                    op->nx % 4 == 0;
  const int g = basis_grid(p.n, cvec ? 4 : 1);
  if (p.dtype == SK_F64) cheb_finalize_kernel<double><<<j1 - j0, kBasisThreads, 0, st>>>(p, g, j0);
  else cheb_finalize_kernel<float><<<j1 - j0, kBasisThreads, 0, st>>>(p, g, j0);
  SK_CUDA(cudaGetLastError());
  return SK_OK;
}

sk_status enqueue_cheb_normalize(const BasisParams& p, cudaStream_t st) {
  const int blocks = 4 * num_sms();
  if (p.dtype == SK_F64) cheb_scale_cols_kernel<double><<<blocks, 256, 0, st>>>(p);
  else if (p.dtype == SK_F32) cheb_scale_cols_kernel<float><<<blocks, 256, 0, st>>>(p);
  else cheb_scale_cols_kernel<__nv_bfloat16><<<blocks, 256, 0, st>>>(p);
  if (p.Hbar) cheb_scale_hbar_kernel<<<(p.d + 256) / 256, 256, 0, st>>>(p);
  SK_CUDA(cudaGetLastError());
  return SK_OK;
}

template <typename T, int KM, int G, bool SM, bool ROWS>
static sk_status enqueue_basis_t(const BasisParams& p, const OpView<typename Compute<T>::type>& A, cudaStream_t st) {
  const int g = p.nblk;
  // steps [j_begin, j_end) (j_end = 0: all d); the first launch follows
  // memset/plain nodes or other kernels: no programmatic edge
  const int jb = p.j_begin, je = p.j_end > 0 ? p.j_end : p.d;
  if (jb == 0) SK_CUDA(launch_pdl(form_kernel<T, KM, G, SM, ROWS>, g, st, false, p.prio, p, A, 0));
  for (int j = jb; j < je; ++j) {
    SK_CUDA(launch_pdl(dots_kernel<T, KM, G, SM, 1, ROWS>, g, st, jb == 0 || j > jb || p.pdl_resume, p.prio, p, A,
                       j));
    if (p.passes == 2) SK_CUDA(launch_pdl(dots_kernel<T, KM, G, SM, 2, ROWS>, g, st, true, p.prio, p, A, j));
    SK_CUDA(launch_pdl(form_kernel<T, KM, G, SM, ROWS>, g, st, true, p.prio, p, A, j + 1));
  }
  return SK_OK;
}

template <typename T, int G, bool SM, bool ROWS, typename C>
static sk_status enqueue_basis_k(const BasisParams& p, const OpView<C>& A, cudaStream_t st) {
  if (p.k <= 2) return enqueue_basis_t<T, 2, G, SM, ROWS>(p, A, st);
  if (p.k <= 4) return enqueue_basis_t<T, 4, G, SM, ROWS>(p, A, st);
  if (p.k <= 8) return enqueue_basis_t<T, 8, G, SM, ROWS>(p, A, st);
  return enqueue_basis_t<T, 16, G, SM, ROWS>(p, A, st);
}

// vector path with cells in one row (nx % 4 == 0), vector path across rows,
// or the scalar path
template <typename T, bool SM, typename C>
static sk_status enqueue_basis_v(const BasisParams& p, const OpView<C>& A, bool vec, bool rows, cudaStream_t st) {
  if (vec && rows) return enqueue_basis_k<T, 4, SM, true>(p, A, st);
  if (vec) return enqueue_basis_k<T, 4, SM, false>(p, A, st);
  return enqueue_basis_k<T, 1, SM, true>(p, A, st);
}

bool basis_vector_path(const sk_op* op, int64_t ldb, const void* B) {
  return op->kind == OP_STENCIL5 && ldb % 8 == 0 && op->n < (1ll << 31) &&
         ((uintptr_t)B % 16) == 0;
}

int basis_grid(int64_t n, int G) {
  // every thread handles exactly IterOf<G> groups of G elements (registers hold
  // the prefetched operands); the grid grows with n
  const int64_t per = (int64_t)kBasisThreads * G * (G == 4 ? IterOf<4>::value : IterOf<1>::value);
  int64_t g = (n + per - 1) / per;
  if (g < 1) g = 1;
  return (int)g;
}

template <typename T, int KM, bool SM>
static sk_status enqueue_basis_grouped_t(const GJob* jobs, const int2* map, int nmap, int passes, int d,
                                         cudaStream_t st) {
  SK_CUDA(launch_pdl(g_form_kernel<T, KM, SM>, nmap, st, false, 0, jobs, map, 0));
  for (int j = 0; j < d; ++j) {
    SK_CUDA(launch_pdl(g_dots_kernel<T, KM, SM, 1>, nmap, st, true, 0, jobs, map, j));
    if (passes == 2) SK_CUDA(launch_pdl(g_dots_kernel<T, KM, SM, 2>, nmap, st, true, 0, jobs, map, j));
    SK_CUDA(launch_pdl(g_form_kernel<T, KM, SM>, nmap, st, true, 0, jobs, map, j + 1));
  }
  return SK_OK;
}

template <typename T, bool SM>
static sk_status enqueue_basis_grouped_k(const GJob* jobs, const int2* map, int nmap, int k, int passes, int d,
                                         cudaStream_t st) {
  if (k <= 2) return enqueue_basis_grouped_t<T, 2, SM>(jobs, map, nmap, passes, d, st);
  if (k <= 4) return enqueue_basis_grouped_t<T, 4, SM>(jobs, map, nmap, passes, d, st);
  if (k <= 8) return enqueue_basis_grouped_t<T, 8, SM>(jobs, map, nmap, passes, d, st);
  return enqueue_basis_grouped_t<T, 16, SM>(jobs, map, nmap, passes, d, st);
}

sk_status enqueue_basis_grouped(const GJob* jobs, const int2* map, int nmap, sk_dtype dt, int k, int passes, int d,
                                cudaStream_t st) {
  if (k > kMaxK) { set_error("k <= %d supported", kMaxK); return SK_EINVAL; }
  if (nmap <= 0) return SK_OK;
  if (dt == SK_F64) return enqueue_basis_grouped_k<double, true>(jobs, map, nmap, k, passes, d, st);
  if (dt == SK_F32) return enqueue_basis_grouped_k<float, false>(jobs, map, nmap, k, passes, d, st);
  return enqueue_basis_grouped_k<__nv_bfloat16, false>(jobs, map, nmap, k, passes, d, st);
}

sk_status enqueue_basis(const BasisParams& p, const sk_op* op, cudaStream_t st) {
  if (p.k > kMaxK) { set_error("k <= %d supported", kMaxK); return SK_EINVAL; }
  const bool vec = basis_vector_path(op, p.ldb, p.B) && (p.r == nullptr || ((uintptr_t)p.r % 16) == 0);
  const bool rows = op->nx % 4 == 0;
  BasisParams q = p;
  q.nblk = basis_grid(p.n, vec ? 4 : 1);
  if (q.nblk > p.nblk_cap) { set_error("basis: partial buffer too small"); return SK_EINVAL; }
  const BasisParams& pp = q;
  if (p.kind == SK_BASIS_CHEBYSHEV) {
    if (!p.sigma || !p.cheb_part || !(p.cheb_rho > 0)) { set_error("Chebyshev basis: workspace or rho missing"); return SK_EINVAL; }
    const bool cvec = vec && rows;
    q.nblk = basis_grid(p.n, cvec ? 4 : 1);
    if (p.dtype == SK_F64) {
      OpView<double> A;
      make_view(op, &A);
      return cvec ? enqueue_cheb_t<double, 4>(pp, A, st) : enqueue_cheb_t<double, 1>(pp, A, st);
    }
    OpView<float> A;
    SK_TRY(make_view(op, &A, st));
    if (p.dtype == SK_F32) return cvec ? enqueue_cheb_t<float, 4>(pp, A, st) : enqueue_cheb_t<float, 1>(pp, A, st);
    return cvec ? enqueue_cheb_t<__nv_bfloat16, 4>(pp, A, st) : enqueue_cheb_t<__nv_bfloat16, 1>(pp, A, st);
  }
  if (p.dtype == SK_F64) {
    OpView<double> A;
    make_view(op, &A);
    if (!p.M) { set_error("FP64 basis needs the m workspace"); return SK_EINVAL; }
    return enqueue_basis_v<double, true>(pp, A, vec, rows, st);
  }
  OpView<float> A;
  SK_TRY(make_view(op, &A, st));
  if (p.dtype == SK_F32) return enqueue_basis_v<float, false>(pp, A, vec, rows, st);
  return enqueue_basis_v<__nv_bfloat16, false>(pp, A, vec, rows, st);
}

}  // namespace sk
