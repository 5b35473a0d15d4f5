// Drivers: trunc_arnoldi_basis, sgmres_solve (Algorithm 1 with restarts,
// §3.5) and the residual / solution-update kernels.
//
// One sGMRES cycle (captured once as a CUDA graph and replayed):
//   g = S r                                   (sketch of the FP64 residual)
//   B_{d+1}, Hbar = truncated Arnoldi(r)      (basis.cu, basis precision)
//   S B_{d+1}; C = (S B_{d+1}) Hbar = S [A b_1 .. A b_d]
//   [C | g] -> Householder QR; y = T^{-1} (U^T g), rhat, kappa (dense.cu)
//   x += B y                                  (FP64 solution update)
//   r = b - A x, ||r||^2                      (FP64 outer residual)
// The host reads ||r|| once per cycle to decide whether to restart.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>
#include <type_traits>
#include <vector>

#include "basis.cuh"
#include "common.cuh"
#include "dense.cuh"
#include "grouped.cuh"
#include "srr.cuh"

namespace sk {

static constexpr int kVecThreads = 256;

// G consecutive entries of one column, converted to the compute type.
template <int G, typename T, typename C>
__device__ __forceinline__ void gload_rows(const T* __restrict__ col, int64_t i, C (&v)[G]) {
  if constexpr (G == 4 && std::is_same<T, float>::value) {
    const float4 t = __ldg(reinterpret_cast<const float4*>(col + i));
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
  } else if constexpr (G == 8 && std::is_same<T, float>::value) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(col + i));
    const float4 b = __ldg(reinterpret_cast<const float4*>(col + i + 4));
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
  } else if constexpr (G == 4 && std::is_same<T, double>::value) {
    const double2 a = __ldg(reinterpret_cast<const double2*>(col + i));
    const double2 b = __ldg(reinterpret_cast<const double2*>(col + i + 2));
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
  } else if constexpr (G == 4) {
    const uint2 u = __ldg(reinterpret_cast<const uint2*>(col + i));
    const float2 fa = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.x));
    const float2 fb = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.y));
    v[0] = fa.x; v[1] = fa.y; v[2] = fb.x; v[3] = fb.y;
  } else {
#pragma unroll
    for (int e = 0; e < G; ++e) v[e] = to_c(col[i + e]);
  }
}

int vec_grid(int64_t n) {
  int64_t g = (n + kVecThreads * 4 - 1) / (kVecThreads * 4);
  const int64_t gmax = 2 * num_sms();
  if (g > gmax) g = gmax;
  if (g < 1) g = 1;
  return (int)g;
}

// r = b - A x and ||r||^2 (last-block reduction into *rho2).  Block `bid`
// of `nb` (the grid, or one job's blocks of a grouped launch).
__device__ __forceinline__ void residual_body(const OpView<double>& A, const double* __restrict__ b,
                                              const double* __restrict__ x, double* __restrict__ r,
                                              double* __restrict__ partial, unsigned* __restrict__ counter,
                                              double* __restrict__ rho2, int bid, int nb) {
  __shared__ double red[kVecThreads / 32];
  double acc[1] = {0.0};
  for (int64_t i = bid * (int64_t)blockDim.x + threadIdx.x; i < A.n; i += (int64_t)nb * blockDim.x) {
    const double v = b[i] - A.apply(x, i);
    r[i] = v;
    acc[0] += v * v;
  }
  block_sum_k<1>(acc, red);
  if (threadIdx.x == 0) partial[bid] = acc[0];
  if (!last_block_arrived_n(counter, (unsigned)nb)) return;
  if (threadIdx.x == 0) {
    double t = 0;
    for (int q = 0; q < nb; ++q) t += __ldcg(partial + q);
    *rho2 = t;
  }
}

__global__ void __launch_bounds__(kVecThreads)
residual_kernel(OpView<double> A, const double* __restrict__ b, const double* __restrict__ x, double* __restrict__ r,
                double* __restrict__ partial, unsigned* __restrict__ counter, double* __restrict__ rho2) {
  residual_body(A, b, x, r, partial, counter, rho2, blockIdx.x, gridDim.x);
}

__device__ __forceinline__ void norm2_body(const double* __restrict__ v, int64_t n, double* __restrict__ partial,
                                           unsigned* __restrict__ counter, double* __restrict__ out, int bid, int nb) {
  __shared__ double red[kVecThreads / 32];
  double acc[1] = {0.0};
  for (int64_t i = bid * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)nb * blockDim.x)
    acc[0] += v[i] * v[i];
  block_sum_k<1>(acc, red);
  if (threadIdx.x == 0) partial[bid] = acc[0];
  if (!last_block_arrived_n(counter, (unsigned)nb)) return;
  if (threadIdx.x == 0) {
    double t = 0;
    for (int q = 0; q < nb; ++q) t += __ldcg(partial + q);
    *out = t;
  }
}

__global__ void __launch_bounds__(kVecThreads)
norm2_kernel(const double* __restrict__ v, int64_t n, double* __restrict__ partial, unsigned* __restrict__ counter,
             double* __restrict__ out) {
  norm2_body(v, n, partial, counter, out, blockIdx.x, gridDim.x);
}

__global__ void init_stop_kernel(int* stop, int value, int* nanflag) {
  *stop = value;
  *nanflag = 0;
}

// x += B y over the first `width` columns (width = diag[2]).  FP64 basis:
// FP64 FMAs.  FP32/BF16 basis: products and sums in pairs of floats
// (exact product error by FMA, two-sum accumulation), about 48 significant
// bits, added to x in FP64.  G = 4 consecutive rows per thread (16-byte
// loads) when the leading dimension and n allow it.
template <typename T, int G>
__device__ __forceinline__ void update_body(double* __restrict__ x, const T* __restrict__ B, int64_t ldb, int64_t n,
                                            int d, const double* __restrict__ y, const double* __restrict__ diag,
                                            int bid, int nb) {
  extern __shared__ double ys[];  // d doubles (+ 2d floats for the pair path)
  const int width = (int)diag[2];
  for (int j = threadIdx.x; j < width; j += blockDim.x) ys[j] = y[j];
  const int64_t stride = (int64_t)nb * blockDim.x * G;
  const int64_t i_begin = ((int64_t)bid * blockDim.x + threadIdx.x) * G;
  if constexpr (!std::is_same<T, double>::value) {
    float* yh = (float*)(ys + d);
    float* yl = yh + d;
    __syncthreads();
    for (int j = threadIdx.x; j < width; j += blockDim.x) {
      const float hi = (float)ys[j];
      yh[j] = hi;
      yl[j] = (float)(ys[j] - (double)hi);
    }
    __syncthreads();
    for (int64_t i = i_begin; i < n; i += stride) {
      float s_hi[G], s_lo[G];
#pragma unroll
      for (int e = 0; e < G; ++e) { s_hi[e] = 0.f; s_lo[e] = 0.f; }
#pragma unroll 4
      for (int j = 0; j < width; ++j) {
        float bv[G];
        gload_rows<G>(B + (int64_t)j * ldb, i, bv);
        const float yhj = yh[j], ylj = yl[j];
#pragma unroll
        for (int e = 0; e < G; ++e) {
          const float p = bv[e] * yhj;
          const float pe = fmaf(bv[e], yhj, -p);
          const float t = s_hi[e] + p;
          const float bp = t - s_hi[e];
          const float err = (s_hi[e] - (t - bp)) + (p - bp);
          s_hi[e] = t;
          s_lo[e] += err + pe + bv[e] * ylj;
        }
      }
#pragma unroll
      for (int e = 0; e < G; ++e) x[i + e] += (double)s_hi[e] + (double)s_lo[e];
    }
  } else {
    __syncthreads();
    for (int64_t i = i_begin; i < n; i += stride) {
      double acc[G];
#pragma unroll
      for (int e = 0; e < G; ++e) acc[e] = 0;
#pragma unroll 4
      for (int j = 0; j < width; ++j) {
        double bv[G];
        gload_rows<G>(B + (int64_t)j * ldb, i, bv);
#pragma unroll
        for (int e = 0; e < G; ++e) acc[e] += bv[e] * ys[j];
      }
#pragma unroll
      for (int e = 0; e < G; ++e) x[i + e] += acc[e];
    }
  }
}

template <typename T, int G>
__global__ void __launch_bounds__(kVecThreads)
update_kernel(double* __restrict__ x, const T* __restrict__ B, int64_t ldb, int64_t n, int d,
              const double* __restrict__ y, const double* __restrict__ diag) {
  update_body<T, G>(x, B, ldb, n, d, y, diag, blockIdx.x, gridDim.x);
}

// ---- grouped vector kernels (batched solver): map[blockIdx.x] = {slot, block} --
__global__ void __launch_bounds__(kVecThreads)
g_residual_kernel(const GJob* __restrict__ jobs, const int2* __restrict__ map) {
  const int2 m = map[blockIdx.x];
  const GJob& J = jobs[m.x];
  residual_body(J.Ad, J.b, J.x, const_cast<double*>(J.bp.r), J.vpart, J.vcnt, const_cast<double*>(J.bp.rho2), m.y, J.vgrid);
}

__global__ void __launch_bounds__(kVecThreads)
g_norm2_kernel(const GJob* __restrict__ jobs, const int2* __restrict__ map) {
  const int2 m = map[blockIdx.x];
  const GJob& J = jobs[m.x];
  norm2_body(J.b, J.bp.n, J.vpart, J.vcnt + 1, J.bn2, m.y, J.vgrid);
}

template <typename T>
__global__ void __launch_bounds__(kVecThreads)
g_update_kernel(const GJob* __restrict__ jobs, const int2* __restrict__ map, int d) {
  const int2 m = map[blockIdx.x];
  const GJob& J = jobs[m.x];
  const T* B = static_cast<const T*>(J.bp.B);
  if (J.uvec) update_body<T, 4>(J.x, B, J.bp.ldb, J.bp.n, d, J.y, J.out + 1, m.y, J.ugrid);
  else update_body<T, 1>(J.x, B, J.bp.ldb, J.bp.n, d, J.y, J.out + 1, m.y, J.ugrid);
}

int update_grid(int64_t n, int G) {
  int64_t g = (n + (int64_t)kVecThreads * G - 1) / ((int64_t)kVecThreads * G);
  if (g > 16 * num_sms()) g = 16 * num_sms();
  if (g < 1) g = 1;
  return (int)g;
}

sk_status enqueue_vec_grouped(GroupedVec which, const GJob* jobs, const int2* map, int nmap, sk_dtype dt, int d,
                              cudaStream_t st) {
  if (nmap <= 0) return SK_OK;
  if (which == GV_RESIDUAL) {
    g_residual_kernel<<<nmap, kVecThreads, 0, st>>>(jobs, map);
  } else if (which == GV_NORM_B) {
    g_norm2_kernel<<<nmap, kVecThreads, 0, st>>>(jobs, map);
  } else {
    const size_t smem = (size_t)d * sizeof(double) + (size_t)2 * d * sizeof(float);
    if (dt == SK_F64) {
      SK_CUDA(cudaFuncSetAttribute(g_update_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, kDynSmemLimit));
      g_update_kernel<double><<<nmap, kVecThreads, smem, st>>>(jobs, map, d);
    } else if (dt == SK_F32) {
      SK_CUDA(cudaFuncSetAttribute(g_update_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, kDynSmemLimit));
      g_update_kernel<float><<<nmap, kVecThreads, smem, st>>>(jobs, map, d);
    } else {
      SK_CUDA(cudaFuncSetAttribute(g_update_kernel<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   kDynSmemLimit));
      g_update_kernel<__nv_bfloat16><<<nmap, kVecThreads, smem, st>>>(jobs, map, d);
    }
  }
  SK_CUDA(cudaGetLastError());
  return SK_OK;
}

template <typename T, int G>
static sk_status launch_update(double* x, const T* B, int64_t ldb, int64_t n, int d, const double* y,
                               const double* diag, cudaStream_t st) {
  const size_t smem = (size_t)d * sizeof(double) + (size_t)2 * d * sizeof(float);
  const int g = update_grid(n, G);
  SK_CUDA(cudaFuncSetAttribute(update_kernel<T, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, kDynSmemLimit));
  update_kernel<T, G><<<g, kVecThreads, smem, st>>>(x, B, ldb, n, d, y, diag);
  SK_CUDA(cudaGetLastError());
  return SK_OK;
}

static sk_status enqueue_update(double* x, const void* B, int64_t ldb, int64_t n, int d, sk_dtype dt, const double* y,
                                const double* diag, cudaStream_t st) {
  const bool vec = (n % 4 == 0) && (ldb % 8 == 0) && ((uintptr_t)B % 16 == 0) && ((uintptr_t)x % 32 == 0);
  if (dt == SK_F64)
    return vec ? launch_update<double, 4>(x, (const double*)B, ldb, n, d, y, diag, st)
               : launch_update<double, 1>(x, (const double*)B, ldb, n, d, y, diag, st);
  // FP32: 8 consecutive rows per thread (two 16-byte loads per column) keep
  // the 2^20-row grid to one wave of resident CTAs
  if (dt == SK_F32 && vec && n % 8 == 0) return launch_update<float, 8>(x, (const float*)B, ldb, n, d, y, diag, st);
  if (dt == SK_F32)
    return vec ? launch_update<float, 4>(x, (const float*)B, ldb, n, d, y, diag, st)
               : launch_update<float, 1>(x, (const float*)B, ldb, n, d, y, diag, st);
  return vec ? launch_update<__nv_bfloat16, 4>(x, (const __nv_bfloat16*)B, ldb, n, d, y, diag, st)
             : launch_update<__nv_bfloat16, 1>(x, (const __nv_bfloat16*)B, ldb, n, d, y, diag, st);
}

void resolve_opts(const sk_opts* in, sk_opts* o, int d) {
  if (in) *o = *in;
  else sk_opts_default(o);
  if (o->zeta <= 0) o->zeta = default_zeta_for(d);
  if (o->stab_tol <= 0) o->stab_tol = o->basis == SK_F64 ? 1e14 : (o->basis == SK_F32 ? 2e6 : 1e2);
  if (o->breakdown <= 0) o->breakdown = o->basis == SK_F64 ? 1e-13 : 1e-6;
  if (o->cgs_passes != 1) o->cgs_passes = 2;
  if (o->maxit <= 0) o->maxit = 10000;
}

// A single classical Gram-Schmidt pass takes nu_j from ||m||^2 - ||h||^2,
// which needs the window orthonormal to the working precision: fine with an
// FP64 basis, unstable with FP32/BF16 (columns blow up after ~20 steps).
sk_status check_passes(const sk_opts& o) {
  if (o.basis_kind == SK_BASIS_CHEBYSHEV) {
    const double rho = o.cheb_dx > o.cheb_dy ? o.cheb_dx : o.cheb_dy;
    if (!(rho > 0) || !std::isfinite(rho) || !std::isfinite(o.cheb_c) || o.cheb_dx < 0 || o.cheb_dy < 0) {
      set_error("invalid argument: the Chebyshev basis needs cheb_dx, cheb_dy >= 0 with max(cheb_dx, cheb_dy) > 0");
      return SK_EINVAL;
    }
    return SK_OK;
  }
  if (o.basis_kind != SK_BASIS_ARNOLDI) {
    set_error("invalid argument: unknown basis_kind %d", (int)o.basis_kind);
    return SK_EINVAL;
  }
  if (o.cgs_passes == 1 && o.basis != SK_F64) {
    set_error("invalid argument: cgs_passes = 1 needs an FP64 basis (use 2 passes with FP32/BF16)");
    return SK_EINVAL;
  }
  return SK_OK;
}

static constexpr long long kBarrierSpinLimit = 1ll << 22;

// Device workspace of one basis build.
struct BasisBuffers {
  BasisParams bp;
  PersistWork pw;
  bool persistent = false;
  sk_status alloc(int64_t n, int d, int k, sk_dtype dt, int passes, double bd, Scratch& sc, void* Bext,
                  const sk_op* op = nullptr, bool want_persistent = false) {
    std::memset(&bp, 0, sizeof(bp));
    bp.n = n;
    bp.d = d;
    bp.k = k;
    bp.passes = passes;
    bp.dtype = dt;
    // internal bases pad the leading dimension to 8 elements (16-byte
    // aligned columns for every storage type); a caller's basis has ld = n
    bp.ldb = Bext ? n : ((n + 7) / 8) * 8;
    bp.bd = bd;
    bp.nblk = basis_grid(n, 1);  // the scalar path needs the most CTAs
    bp.nblk_cap = bp.nblk;
    if (Bext) bp.B = Bext;
    else {
      unsigned char* Bp = nullptr;
      SK_TRY(sc.alloc(&Bp, (size_t)bp.ldb * (d + 1) * dtype_size(dt)));
      bp.B = Bp;
    }
    if (dt == SK_F64) SK_TRY(sc.alloc(&bp.M, (size_t)n));
    int pg = 0, pe = 0;
    size_t psm = 0;
    persistent = want_persistent && op != nullptr && persist_shape(op, dt, k, &pg, &pe, &psm);
    std::memset(&pw, 0, sizeof(pw));
    if (persistent) {
      SK_TRY(sc.alloc(&pw.bar, 2));
      SK_TRY(sc.alloc(&pw.err, 1));
      SK_CUDA(cudaMemsetAsync(pw.err, 0, sizeof(int), sc.st));
      SK_TRY(sc.alloc(&pw.part, (size_t)3 * pg * (kMaxK + 1)));
      pw.spin_limit = kBarrierSpinLimit;
    }
    double* dd = nullptr;
    const size_t nd = (size_t)2 * d * k + 2 * (size_t)d + (size_t)(d + 1) * d + (size_t)bp.nblk_cap * (kMaxK + 1) + 2 +
                      (size_t)d * (kMaxK + 1);
    SK_TRY(sc.alloc(&dd, nd));
    bp.h1 = dd;
    bp.h2 = bp.h1 + (size_t)d * k;
    bp.nu = bp.h2 + (size_t)d * k;
    bp.mn2 = bp.nu + d;
    bp.Hbar = bp.mn2 + d;
    bp.partial = bp.Hbar + (size_t)(d + 1) * d;
    double* rho2 = bp.partial + (size_t)bp.nblk_cap * (kMaxK + 1);
    bp.rho2 = rho2;
    bp.coef = rho2 + 2;
    unsigned* cnt = nullptr;
    SK_TRY(sc.alloc(&cnt, 8));
    SK_CUDA(cudaMemsetAsync(cnt, 0, 8 * sizeof(unsigned), sc.st));
    bp.counters = cnt;
    int* flags = nullptr;
    SK_TRY(sc.alloc(&flags, 2));
    bp.stop = flags;
    bp.nanflag = flags + 1;
    return SK_OK;
  }
  double* rho2_mut() const { return const_cast<double*>(bp.rho2); }
  // Chebyshev basis: recurrence parameters and its workspace (call after alloc)
  sk_status set_kind(const sk_opts& o, Scratch& sc) {
    if (o.barrier_spins > 0) pw.spin_limit = o.barrier_spins;
    else if (o.barrier_spins < 0) pw.spin_limit = 0;
    bp.kind = o.basis_kind;
    if (o.basis_kind != SK_BASIS_CHEBYSHEV) return SK_OK;
    persistent = false;
    bp.cheb_c = o.cheb_c;
    bp.cheb_rho = o.cheb_dx > o.cheb_dy ? o.cheb_dx : o.cheb_dy;
    bp.cheb_gamma = (o.cheb_dx * o.cheb_dx - o.cheb_dy * o.cheb_dy) / (4.0 * bp.cheb_rho);
    SK_TRY(sc.alloc(&bp.sigma, (size_t)bp.d + 1));
    SK_TRY(sc.alloc(&bp.cheb_part, (size_t)(bp.d + 1) * bp.nblk_cap));
    return SK_OK;
  }
  bool cheb() const { return bp.kind == SK_BASIS_CHEBYSHEV; }
  int hbar_k() const { return cheb() && bp.k < 2 ? 2 : bp.k; }  // Chebyshev Hbar is tridiagonal
};

// y[j] /= sigma[j]: the sketched problem is posed in the unit columns
// b_j = v_j / sigma_j, the update uses the stored v_j.
__global__ void scale_y_kernel(double* __restrict__ y, const double* __restrict__ sigma, int d) {
  for (int j = threadIdx.x; j < d; j += blockDim.x) {
    const double sg = sigma[j];
    y[j] = (sg > 0) ? y[j] / sg : 0.0;
  }
}

// Enqueue one basis build: stop = d+1, Hbar = 0, then the kernels.
static sk_status enqueue_basis_build(BasisBuffers& bb, const sk_op* A, cudaStream_t st) {
  const BasisParams& bp = bb.bp;
  init_stop_kernel<<<1, 1, 0, st>>>(bp.stop, bp.d + 1, bp.nanflag);
  SK_CUDA(cudaMemsetAsync(bp.Hbar, 0, sizeof(double) * (size_t)(bp.d + 1) * bp.d, st));
  if (bb.persistent) return enqueue_basis_persistent(bp, A, bb.pw, st);
  return enqueue_basis(bp, A, st);
}

}  // namespace sk

using namespace sk;

extern "C" sk_status trunc_arnoldi_basis(const sk_op* A, const double* r0, int d, int k, sk_dtype basis_dtype,
                                         void* B, double* Hbar, const sk_sketch* S, double* SB, double* SAB,
                                         const sk_opts* opts, int* d_used, void* stream) {
  SK_CHECK_ARG(A != nullptr && r0 != nullptr && B != nullptr && d_used != nullptr, "NULL argument");
  SK_CHECK_ARG(d >= 1 && k >= 1 && k <= d, "need d >= 1 and 1 <= k <= d");
  SK_CHECK_ARG(k <= kMaxK, "k <= 16 supported");
  SK_CHECK_ARG(basis_dtype == SK_F64 || basis_dtype == SK_F32 || basis_dtype == SK_BF16, "basis dtype");
  SK_CHECK_ARG((SB == nullptr && SAB == nullptr) || S != nullptr, "SB/SAB need a sketch");
  if (S) SK_CHECK_ARG(S->n == A->n, "sketch n must equal operator n");
  cudaStream_t st = (cudaStream_t)stream;
  sk_opts o;
  resolve_opts(opts, &o, d);
  o.basis = basis_dtype;
  if (!opts || opts->breakdown <= 0) o.breakdown = basis_dtype == SK_F64 ? 1e-13 : 1e-6;
  SK_TRY(check_passes(o));
  Scratch sc(st);
  BasisBuffers bb;
  SK_TRY(bb.alloc(A->n, d, k, basis_dtype, o.cgs_passes, o.breakdown, sc, B, A, o.persistent != 0));
  SK_TRY(bb.set_kind(o, sc));
  bb.bp.r = r0;
  {
    double* part = nullptr;
    unsigned* cnt = nullptr;
    const int g = vec_grid(A->n);
    SK_TRY(sc.alloc(&part, g));
    SK_TRY(sc.alloc(&cnt, 1));
    SK_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned), st));
    norm2_kernel<<<g, kVecThreads, 0, st>>>(r0, A->n, part, cnt, bb.rho2_mut());
    SK_CUDA(cudaGetLastError());
  }
  SK_TRY(enqueue_basis_build(bb, A, st));
  if (bb.cheb()) SK_TRY(enqueue_cheb_normalize(bb.bp, st));
  if (S) {
    Sketcher sk;
    SK_TRY(sk.create(*S, sc, st));
    double* SBfull = nullptr;
    double* ws = nullptr;
    SK_TRY(sc.alloc(&SBfull, (size_t)S->s * (d + 1)));
    SK_TRY(sc.alloc(&ws, sk.ws(d + 1, basis_dtype, true)));
    SK_TRY(sk.apply(B, A->n, d + 1, basis_dtype, SBfull, ws, st, true));
    if (SB) SK_TRY(enqueue_copy_sb(SBfull, S->s, d, bb.bp.stop, SB, st));
    if (SAB) SK_TRY(enqueue_hbar_product(SBfull, bb.bp.Hbar, S->s, d, bb.hbar_k(), bb.bp.stop, SAB, st));
  }
  if (Hbar) SK_CUDA(cudaMemcpyAsync(Hbar, bb.bp.Hbar, sizeof(double) * (size_t)(d + 1) * d, cudaMemcpyDeviceToDevice, st));
  int h[3] = {0, 0, 0};
  SK_CUDA(cudaMemcpyAsync(h, bb.bp.stop, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
  if (bb.persistent) SK_CUDA(cudaMemcpyAsync(h + 2, bb.pw.err, sizeof(int), cudaMemcpyDeviceToHost, st));
  SK_CUDA(cudaStreamSynchronize(st));
  *d_used = h[0] < d ? h[0] : d;
  if (h[2]) { set_error("persistent basis: a grid barrier timed out"); return SK_ETIMEOUT; }
  if (h[1]) { set_error("NaN/Inf in the basis recurrence"); return SK_ENAN; }
  return SK_OK;
}

namespace sk {

struct SolveState {
  int64_t n;
  int d, k, s;
  sk_opts o;
  BasisBuffers bb;
  Sketcher sketch;
  double* r;
  double* g;
  double* SB;
  double* Aug;
  double* rdiag;
  double* tau;
  double* Tws;
  double* y;
  double* ws_r;
  double* ws_B;
  double* vec_part;
  unsigned* vec_cnt;
  double* out;      // device: [rho2, rhat, kappa, width]
  double* h_out;    // pinned host copy, 8 doubles: [0..3] the cycle's scalars, [4] the persistent
                    // kernel's error word, [5] the iterative cycle's tau, [6..7] its chunk check
  int* h_err;
  // iterative cycles: one captured graph per chunk position (made on first
  // use, replayed every cycle), its kernel count, the device tau it reads
  cudaGraphExec_t* ig;
  long long* ig_kernels;
  int n_ig;
  double* tau_dev;
  // pipelined cycle: side stream for the sketch and QR of finished basis
  // blocks, its fork/join events, one event per block, the basis priority
  bool pipe;
  cudaStream_t side, qrs;   // block sketches; QR panels
  cudaEvent_t fork, join;
  cudaEvent_t* blk;         // per block: basis columns formed (main), then sketched (side)
  cudaEvent_t* skd;
  int prio_hi;
};

static sk_status enqueue_residual(const SolveState& S, const OpView<double>& Av, const double* b, const double* x,
                                  cudaStream_t st) {
  residual_kernel<<<vec_grid(S.n), kVecThreads, 0, st>>>(Av, b, x, S.r, S.vec_part, S.vec_cnt, S.bb.rho2_mut());
  SK_CUDA(cudaGetLastError());
  return SK_OK;
}

// Phase boundaries of a cycle, recorded as event nodes inside the graph.
enum { EV_START, EV_G, EV_BASIS, EV_SB, EV_SMALL, EV_UPDATE, EV_RES, EV_COUNT };

static sk_status mark(cudaEvent_t* ev, int which, cudaStream_t st, bool capturing) {
  if (!ev) return SK_OK;
  if (capturing) SK_CUDA(cudaEventRecordWithFlags(ev[which], st, cudaEventRecordExternal));
  else SK_CUDA(cudaEventRecord(ev[which], st));
  return SK_OK;
}

// One restart cycle, ending with the new residual and its norm.
static sk_status enqueue_cycle(SolveState& S, const sk_op* A, const OpView<double>& Av, const double* b, double* x,
                               cudaStream_t st, cudaEvent_t* ev, bool capturing) {
  SK_TRY(mark(ev, EV_START, st, capturing));
  SK_TRY(S.sketch.apply(S.r, S.n, 1, SK_F64, S.g, S.ws_r, st, false));
  SK_TRY(mark(ev, EV_G, st, capturing));
  SK_TRY(enqueue_basis_build(S.bb, A, st));
  SK_TRY(mark(ev, EV_BASIS, st, capturing));
  SK_TRY(S.sketch.apply(S.bb.bp.B, S.bb.bp.ldb, S.d + 1, S.o.basis, S.SB, S.ws_B, st, true));
  SK_TRY(mark(ev, EV_SB, st, capturing));
  SK_TRY(enqueue_hbar_product(S.SB, S.bb.bp.Hbar, S.s, S.d, S.bb.hbar_k(), S.bb.bp.stop, S.Aug, st));
  SK_CUDA(cudaMemcpyAsync(S.Aug + (size_t)S.d * S.s, S.g, sizeof(double) * S.s, cudaMemcpyDeviceToDevice, st));
  SK_TRY(enqueue_qr(S.Aug, S.s, S.d, S.d + 1, S.rdiag, S.tau, S.Tws, st));
  SK_TRY(enqueue_ls_solve(S.Aug, S.rdiag, S.s, S.d, S.o.stab_tol, S.y, S.out + 1, st));
  if (S.bb.cheb()) {
    scale_y_kernel<<<1, 256, 0, st>>>(S.y, S.bb.bp.sigma, S.d);
    SK_CUDA(cudaGetLastError());
  }
  SK_TRY(mark(ev, EV_SMALL, st, capturing));
  SK_TRY(enqueue_update(x, S.bb.bp.B, S.bb.bp.ldb, S.n, S.d, S.o.basis, S.y, S.out + 1, st));
  SK_TRY(mark(ev, EV_UPDATE, st, capturing));
  SK_TRY(enqueue_residual(S, Av, b, x, st));
  SK_CUDA(cudaMemcpyAsync(S.out, S.bb.bp.rho2, sizeof(double), cudaMemcpyDeviceToDevice, st));
  SK_TRY(mark(ev, EV_RES, st, capturing));
  SK_CUDA(cudaMemcpyAsync(S.h_out, S.out, 4 * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (S.bb.persistent) SK_CUDA(cudaMemcpyAsync(S.h_err, S.bb.pw.err, sizeof(int), cudaMemcpyDeviceToHost, st));
  return SK_OK;
}

// One restart cycle in pipelined form.  The truncated-Arnoldi passes run on
// `st` at raised priority, in blocks of kQrNb steps; after each block its
// basis columns (still partly in L2) are sketched on the side stream, and
// every panel of C = (S B_{d+1}) Hbar whose columns the sketched part of
// B_{d+1} completes (column j needs b_0 .. b_{j+1}) joins the Householder
// QR: the earlier panels' reflectors applied left-looking, the panel
// factored, its reflectors applied to g = S r in column d.  The side work
// overlaps the next blocks' basis passes, which are latency bound and leave
// most of the GPU idle.  After the last block the streams join for the LS
// solve, the update and the residual.  Column by column the arithmetic is
// that of enqueue_cycle (same kernels, same order per column), so the two
// forms give identical results.
static sk_status enqueue_cycle_pipelined(SolveState& S, const sk_op* A, const OpView<double>& Av, const double* b,
                                         double* x, cudaStream_t st, cudaEvent_t* ev, bool capturing) {
  const int d = S.d, s = S.s;
  const size_t esz = dtype_size(S.o.basis);
  BasisParams& bp = S.bb.bp;
  cudaStream_t sd = S.side, sq = S.qrs;
  SK_TRY(mark(ev, EV_START, st, capturing));
  SK_TRY(mark(ev, EV_G, st, capturing));
  SK_CUDA(cudaEventRecord(S.fork, st));
  SK_CUDA(cudaStreamWaitEvent(sq, S.fork, 0));
  SK_TRY(S.sketch.apply(S.r, S.n, 1, SK_F64, S.g, S.ws_r, sq, false));
  SK_CUDA(cudaMemcpyAsync(S.Aug + (size_t)d * s, S.g, sizeof(double) * s, cudaMemcpyDeviceToDevice, sq));
  init_stop_kernel<<<1, 1, 0, st>>>(bp.stop, d + 1, bp.nanflag);
  SK_CUDA(cudaMemsetAsync(bp.Hbar, 0, sizeof(double) * (size_t)(d + 1) * d, st));
  const int nb = (d + 1 + kQrNb - 1) / kQrNb;
  const int npanels = (d + kQrNb - 1) / kQrNb;
  int panels = 0, prev = 0;
  sk_status rs = SK_OK;
  for (int t = 0; t < nb && rs == SK_OK; ++t) {
    // main: steps [prev, je) form basis columns up to je
    const int je = std::min(kQrNb * t + kQrNb - 1, d);
    bp.j_begin = prev;
    bp.j_end = je;
    bp.pdl_resume = prev > 0;
    bp.prio = S.prio_hi;
    rs = enqueue_basis(bp, A, st);
    prev = je;
    if (rs != SK_OK) break;
    SK_CUDA(cudaEventRecord(S.blk[t], st));
    // side: (Chebyshev: the block's column norms and Hbar columns, then) the
    // sketch of the block's columns
    SK_CUDA(cudaStreamWaitEvent(sd, S.blk[t], 0));
    const int c0 = kQrNb * t, c1 = std::min(c0 + kQrNb, d + 1);
    if (S.bb.cheb()) {
      rs = enqueue_cheb_finalize(bp, A, c0, c1, sd);
      if (rs != SK_OK) break;
    }
    rs = S.sketch.apply((const unsigned char*)bp.B + (size_t)c0 * bp.ldb * esz, bp.ldb, c1 - c0, S.o.basis,
                        S.SB + (size_t)c0 * s, S.ws_B, sd, true);
    if (rs != SK_OK) break;
    SK_CUDA(cudaEventRecord(S.skd[t], sd));
    // QR stream: the panels this block completes
    bool waited = false;
    while (rs == SK_OK && panels < npanels && std::min(kQrNb * panels + kQrNb, d) <= c1 - 1) {
      if (!waited) SK_CUDA(cudaStreamWaitEvent(sq, S.skd[t], 0));
      waited = true;
      const int q0 = kQrNb * panels, q1 = std::min(q0 + kQrNb, d);
      rs = enqueue_hbar_product_cols(S.SB, bp.Hbar, s, d, S.bb.hbar_k(), bp.stop, q0, q1, S.Aug, sq);
      if (rs == SK_OK) rs = enqueue_qr_append(S.Aug, s, q0, q1, d, S.rdiag, S.tau, S.Tws, nullptr, sq);
      ++panels;
    }
  }
  bp.j_begin = bp.j_end = 0;
  bp.pdl_resume = 0;
  bp.prio = 0;
  SK_TRY(rs);
  SK_TRY(mark(ev, EV_BASIS, st, capturing));
  // the sketch stream's last block precedes the last panels on the QR stream
  SK_CUDA(cudaStreamWaitEvent(sq, S.skd[nb - 1], 0));
  SK_CUDA(cudaEventRecord(S.join, sq));
  SK_CUDA(cudaStreamWaitEvent(st, S.join, 0));
  SK_TRY(mark(ev, EV_SB, st, capturing));
  SK_TRY(enqueue_ls_solve(S.Aug, S.rdiag, s, d, S.o.stab_tol, S.y, S.out + 1, st));
  if (S.bb.cheb()) {
    scale_y_kernel<<<1, 256, 0, st>>>(S.y, bp.sigma, d);
    SK_CUDA(cudaGetLastError());
  }
  SK_TRY(mark(ev, EV_SMALL, st, capturing));
  SK_TRY(enqueue_update(x, bp.B, bp.ldb, S.n, d, S.o.basis, S.y, S.out + 1, st));
  SK_TRY(mark(ev, EV_UPDATE, st, capturing));
  SK_TRY(enqueue_residual(S, Av, b, x, st));
  SK_CUDA(cudaMemcpyAsync(S.out, bp.rho2, sizeof(double), cudaMemcpyDeviceToDevice, st));
  SK_TRY(mark(ev, EV_RES, st, capturing));
  SK_CUDA(cudaMemcpyAsync(S.h_out, S.out, 4 * sizeof(double), cudaMemcpyDeviceToHost, st));
  return SK_OK;
}

// One cycle of iterative sGMRES (§5.2; restart on kappa, §5.3).  The basis
// grows o.iter_chunk columns at a time; after each chunk its new columns are
// sketched, S A B's QR grows by them (enqueue_qr_append: the reflectors of
// enqueue_qr, applied left-looking) and prefix_check finds the first prefix
// j whose estimate ||z[j:]|| (z = Q^T g) meets tau_rel ||g||.  The host reads
// that one answer per chunk; the cycle ends there, or on the kappa estimate,
// a breakdown or j = d, and the solve and the update use that prefix.
// *used = the prefix solved, *built = the steps the basis ran.
static long long count_kernel_nodes(cudaGraph_t g);

static sk_status run_iterative_cycle(SolveState& S, const sk_op* A, const OpView<double>& Av, const double* b,
                                     double* x, double tau_rel, int* chk, cudaStream_t st, cudaEvent_t* ev,
                                     int* used, int* built, long long* launches) {
  const int d = S.d, s = S.s, chunk = S.o.iter_chunk;
  const size_t esz = dtype_size(S.o.basis);
  BasisParams& bp = S.bb.bp;
  long long nl = 0;
  SK_TRY(mark(ev, EV_START, st, false));
  S.h_out[5] = tau_rel;  // the captured checks read it from the device
  SK_CUDA(cudaMemcpyAsync(S.tau_dev, S.h_out + 5, sizeof(double), cudaMemcpyHostToDevice, st));
  SK_TRY(S.sketch.apply(S.r, S.n, 1, SK_F64, S.g, S.ws_r, st, false));
  nl += 2;
  SK_TRY(mark(ev, EV_G, st, false));
  init_stop_kernel<<<1, 1, 0, st>>>(bp.stop, d + 1, bp.nanflag);
  ++nl;
  SK_CUDA(cudaMemsetAsync(bp.Hbar, 0, sizeof(double) * (size_t)(d + 1) * d, st));
  double* z = S.Aug + (size_t)d * s;
  SK_CUDA(cudaMemcpyAsync(z, S.g, sizeof(double) * s, cudaMemcpyDeviceToDevice, st));
  int dp = d, c1 = 0;
  int* h = reinterpret_cast<int*>(S.h_out + 6);
  for (int ci = 0, c0 = 0; c0 < d; ++ci, c0 = c1) {
    c1 = c0 + chunk < d ? c0 + chunk : d;
    if (!S.ig[ci]) {
      // capture the chunk once: its basis steps, the sketch of its new
      // columns, their columns of C, the QR append, the stop test and the
      // copy of the test's word to the host
      SK_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
      auto body = [&]() -> sk_status {
        bp.j_begin = c0;
        bp.j_end = c1;
        const sk_status bs = enqueue_basis(bp, A, st);
        bp.j_begin = bp.j_end = 0;
        SK_TRY(bs);
        // the chunk's new basis columns: b_{c0+1} .. b_{c1} (0-based), and b_0 first
        const int s0 = c0 == 0 ? 0 : c0 + 1;
        SK_TRY(S.sketch.apply((const unsigned char*)bp.B + (size_t)s0 * bp.ldb * esz, bp.ldb, c1 + 1 - s0,
                              S.o.basis, S.SB + (size_t)s0 * s, S.ws_B, st, true));
        SK_TRY(enqueue_hbar_product_cols(S.SB, bp.Hbar, s, d, S.bb.hbar_k(), bp.stop, c0, c1, S.Aug, st));
        SK_TRY(enqueue_qr_append(S.Aug, s, c0, c1, d, S.rdiag, S.tau, S.Tws, nullptr, st));
        SK_TRY(enqueue_prefix_check(z, S.rdiag, bp.stop, s, c0, c1, S.tau_dev, S.o.stab_tol, chk, st));
        SK_CUDA(cudaMemcpyAsync(h, chk, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
        return SK_OK;
      };
      const sk_status bs = body();
      cudaGraph_t g = nullptr;
      const cudaError_t ce = cudaStreamEndCapture(st, &g);
      if (bs != SK_OK) {
        if (g) cudaGraphDestroy(g);
        return bs;
      }
      if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamEndCapture");
      const cudaError_t ie = cudaGraphInstantiate(&S.ig[ci], g, 0);
      S.ig_kernels[ci] = count_kernel_nodes(g);
      cudaGraphDestroy(g);
      if (ie != cudaSuccess) return cuda_fail(ie, "cudaGraphInstantiate");
    }
    SK_CUDA(cudaGraphLaunch(S.ig[ci], st));
    nl += S.ig_kernels[ci];
    SK_CUDA(cudaStreamSynchronize(st));
    if (h[0] > 0) {
      dp = h[0];
      break;
    }
    if (h[1] || c1 == d) {
      dp = c1;
      break;
    }
  }
  SK_TRY(mark(ev, EV_BASIS, st, false));
  SK_TRY(mark(ev, EV_SB, st, false));
  SK_TRY(enqueue_ls_solve_z(S.Aug, S.rdiag, z, s, dp, S.o.stab_tol, S.y, S.out + 1, st));
  ++nl;
  SK_TRY(mark(ev, EV_SMALL, st, false));
  SK_TRY(enqueue_update(x, bp.B, bp.ldb, S.n, dp, S.o.basis, S.y, S.out + 1, st));
  ++nl;
  SK_TRY(mark(ev, EV_UPDATE, st, false));
  SK_TRY(enqueue_residual(S, Av, b, x, st));
  ++nl;
  SK_CUDA(cudaMemcpyAsync(S.out, bp.rho2, sizeof(double), cudaMemcpyDeviceToDevice, st));
  SK_TRY(mark(ev, EV_RES, st, false));
  SK_CUDA(cudaMemcpyAsync(S.h_out, S.out, 4 * sizeof(double), cudaMemcpyDeviceToHost, st));
  *used = dp;
  *built = c1;
  *launches += nl;
  return SK_OK;
}

static long long count_kernel_nodes(cudaGraph_t g) {
  size_t nn = 0;
  if (cudaGraphGetNodes(g, nullptr, &nn) != cudaSuccess) return -1;
  cudaGraphNode_t* nodes = new cudaGraphNode_t[nn ? nn : 1];
  long long k = 0;
  if (cudaGraphGetNodes(g, nodes, &nn) == cudaSuccess) {
    for (size_t i = 0; i < nn; ++i) {
      cudaGraphNodeType t;
      if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++k;
    }
  }
  delete[] nodes;
  return k;
}

}  // namespace sk

namespace sk {

// One restarted-sGMRES configuration on one operator: its buffers, sketch
// plan, side streams and (once captured) the cycle's graph.  sgmres_solve
// builds one per call; sgmres_plan_create keeps one across calls.
struct Solver {
  SolveState S;
  const sk_op* A = nullptr;
  OpView<double> Av;
  Scratch* sc = nullptr;       // the state's buffers, freed on the creation stream
  cudaStream_t st0 = nullptr;  // creation stream
  cudaStream_t last = nullptr; // stream of the last solve
  bool iter = false;
  int* chk = nullptr;
  double* bn2d = nullptr;
  bool own_pinned = false;
  long long setup_launches = 0;  // plan build and FP32 operator copies
  cudaGraphExec_t gexec = nullptr;
  long long kernels_per_cycle = 0;
  const double* gb = nullptr;  // the b and x the captured cycle reads and writes
  double* gx = nullptr;
  cudaStream_t own = nullptr;  // capturable stream when the caller passes the legacy stream
  cudaEvent_t ev[EV_COUNT] = {};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  double* hb = nullptr;        // plan handles: private b and x (the graph's operands)
  double* hx = nullptr;

  Solver() { std::memset(&S, 0, sizeof(S)); }
  ~Solver();
  sk_status setup(const sk_op* A_, int d, int k, int s, const sk_opts* opts, cudaStream_t st, double* h_pinned);
  sk_status capture(const double* b, double* x, cudaStream_t cap);
  sk_status run(const double* b, double* x, double tol, sk_info* info, cudaStream_t st);
};

Solver::~Solver() {
  if (last) cudaStreamSynchronize(last);
  if (st0) cudaStreamSynchronize(st0);
  if (gexec) cudaGraphExecDestroy(gexec);
  for (int q = 0; q < EV_COUNT; ++q)
    if (ev[q]) cudaEventDestroy(ev[q]);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (own) cudaStreamDestroy(own);
  if (S.side) cudaStreamDestroy(S.side);
  if (S.qrs) cudaStreamDestroy(S.qrs);
  if (S.fork) cudaEventDestroy(S.fork);
  if (S.join) cudaEventDestroy(S.join);
  const int nb = (S.d + 1 + kQrNb - 1) / kQrNb;
  for (cudaEvent_t* e : {S.blk, S.skd}) {
    if (!e) continue;
    for (int t = 0; t < nb; ++t)
      if (e[t]) cudaEventDestroy(e[t]);
    delete[] e;
  }
  for (int q = 0; q < S.n_ig; ++q)
    if (S.ig[q]) cudaGraphExecDestroy(S.ig[q]);
  delete[] S.ig;
  delete[] S.ig_kernels;
  if (own_pinned && S.h_out) cudaFreeHost(S.h_out);
  delete sc;  // stream-ordered frees on st0, after the synchronisations above
}

sk_status Solver::setup(const sk_op* A_, int d, int k, int s, const sk_opts* opts, cudaStream_t st,
                        double* h_pinned) {
  A = A_;
  st0 = st;
  resolve_opts(opts, &S.o, d);
  SK_CHECK_ARG(S.o.basis == SK_F64 || S.o.basis == SK_F32 || S.o.basis == SK_BF16, "basis dtype");
  SK_TRY(check_passes(S.o));
  iter = S.o.iter_chunk != 0;
  if (iter) {
    SK_CHECK_ARG(S.o.iter_chunk > 0 && S.o.iter_chunk % kQrNb == 0 && S.o.iter_chunk <= 1024,
                 "iter_chunk must be a positive multiple of 16, at most 1024");
    SK_CHECK_ARG(S.o.basis_kind == SK_BASIS_ARNOLDI, "iter_chunk needs the truncated-Arnoldi basis");
    S.o.use_graph = 0;
    S.o.persistent = 0;
  }
  S.n = A->n;
  S.d = d;
  S.k = k;
  S.s = s;
  sc = new Scratch(st);
  Scratch& scr = *sc;
  SK_TRY(S.bb.alloc(S.n, d, k, S.o.basis, S.o.cgs_passes, S.o.breakdown, scr, nullptr, A, S.o.persistent != 0));
  SK_TRY(S.bb.set_kind(S.o, scr));
  // the pipelined cycle: captured cycles of the 3-launch Arnoldi basis or the Chebyshev basis
  S.pipe = S.o.pipeline != 0 && S.o.use_graph && !iter && !S.bb.persistent;
  if (S.pipe) {
    int least = 0, greatest = 0;
    SK_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    S.prio_hi = greatest;
    SK_CUDA(cudaStreamCreateWithPriority(&S.side, cudaStreamNonBlocking, least));
    SK_CUDA(cudaStreamCreateWithPriority(&S.qrs, cudaStreamNonBlocking, least));
    SK_CUDA(cudaEventCreateWithFlags(&S.fork, cudaEventDisableTiming));
    SK_CUDA(cudaEventCreateWithFlags(&S.join, cudaEventDisableTiming));
    const int nb = (d + 1 + kQrNb - 1) / kQrNb;
    S.blk = new cudaEvent_t[nb];
    S.skd = new cudaEvent_t[nb];
    for (int t = 0; t < nb; ++t) S.blk[t] = S.skd[t] = nullptr;
    for (int t = 0; t < nb; ++t) {
      SK_CUDA(cudaEventCreateWithFlags(&S.blk[t], cudaEventDisableTiming));
      SK_CUDA(cudaEventCreateWithFlags(&S.skd[t], cudaEventDisableTiming));
    }
  }
  sk_sketch sks;
  sks.kind = S.o.sketch;
  sks.n = S.n;
  sks.s = s;
  sks.zeta = S.o.zeta;
  sks.seed = S.o.seed;
  SK_TRY(S.sketch.create(sks, scr, st));
  SK_TRY(scr.alloc(&S.r, S.n));
  S.bb.bp.r = S.r;
  SK_TRY(scr.alloc(&S.g, s));
  SK_TRY(scr.alloc(&S.SB, (size_t)s * (d + 1)));
  SK_TRY(scr.alloc(&S.Aug, (size_t)s * (d + 1)));
  SK_TRY(scr.alloc(&S.rdiag, d));
  SK_TRY(scr.alloc(&S.tau, d));
  SK_TRY(scr.alloc(&S.Tws, (size_t)((d + kQrNb - 1) / kQrNb) * kQrNb * kQrNb));
  SK_TRY(scr.alloc(&S.y, d));
  SK_TRY(scr.alloc(&S.ws_r, S.sketch.ws(1, SK_F64, false)));
  {
    // iterative cycles sketch 1..iter_chunk+1 columns at a time: room for
    // the largest of those shapes too
    size_t wsb = S.sketch.ws(d + 1, S.o.basis, true);
    for (int c = 1; iter && c <= S.o.iter_chunk + 1 && c <= d + 1; ++c) {
      const size_t w = S.sketch.ws(c, S.o.basis, true);
      if (w > wsb) wsb = w;
    }
    SK_TRY(scr.alloc(&S.ws_B, wsb));
  }
  if (iter) {
    SK_TRY(scr.alloc(&chk, 2));
    SK_TRY(scr.alloc(&S.tau_dev, 1));
    S.n_ig = (d + S.o.iter_chunk - 1) / S.o.iter_chunk;
    S.ig = new cudaGraphExec_t[S.n_ig];
    S.ig_kernels = new long long[S.n_ig];
    for (int q = 0; q < S.n_ig; ++q) {
      S.ig[q] = nullptr;
      S.ig_kernels[q] = 0;
    }
  }
  SK_TRY(scr.alloc(&S.vec_part, vec_grid(S.n)));
  SK_TRY(scr.alloc(&S.vec_cnt, 2));
  SK_CUDA(cudaMemsetAsync(S.vec_cnt, 0, 2 * sizeof(unsigned), st));
  SK_TRY(scr.alloc(&S.out, 4));
  SK_CUDA(cudaMemsetAsync(S.out, 0, 4 * sizeof(double), st));
  SK_TRY(scr.alloc(&bn2d, 1));
  // pinned landing buffer for the per-cycle scalars (the caller's, or our own)
  if (h_pinned) S.h_out = h_pinned;
  else {
    SK_CUDA(cudaMallocHost((void**)&S.h_out, 8 * sizeof(double)));
    own_pinned = true;
  }
  S.h_err = (int*)(S.h_out + 4);
  *S.h_err = 0;
  make_view(A, &Av);
  if (S.o.basis != SK_F64) {
    // the op's FP32 parameter copies are allocated here, before any capture
    OpView<float> Af;
    SK_TRY(make_view(A, &Af, st));
  }
  // kernels launched here: the sketch plan (1, or 1 for SRHT signs) and the
  // FP32 operator copies
  setup_launches = 1;
  if (S.o.basis != SK_F64) setup_launches += (A->shift ? 1 : 0) + (A->theta ? 1 : 0) + (A->val ? 1 : 0);
  for (int q = 0; q < EV_COUNT; ++q) SK_CUDA(cudaEventCreate(&ev[q]));
  SK_CUDA(cudaEventCreate(&e0));
  SK_CUDA(cudaEventCreate(&e1));
  // the legacy default stream cannot be captured: a private stream then
  if ((iter || S.o.use_graph) && (st == nullptr || st == cudaStreamLegacy))
    SK_CUDA(cudaStreamCreateWithFlags(&own, cudaStreamNonBlocking));
  if (!iter && !S.o.use_graph) {
    const long long basis_kernels = S.bb.cheb() ? (long long)d + 2 : (long long)d * (S.o.cgs_passes + 1);
    kernels_per_cycle = 5 + 3 + basis_kernels + 2 + 1 + 2 * ((d + kQrNb - 1) / kQrNb) + 1 + 1 + 1 + (S.bb.cheb() ? 1 : 0);
  }
  return SK_OK;
}

// Capture one cycle reading b and writing x (replaced if the operands change).
sk_status Solver::capture(const double* b, double* x, cudaStream_t cap) {
  if (gexec && gb == b && gx == x) return SK_OK;
  if (gexec) {
    cudaGraphExecDestroy(gexec);
    gexec = nullptr;
  }
  cudaGraph_t graph = nullptr;
  SK_CUDA(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
  const sk_status cs = S.pipe ? enqueue_cycle_pipelined(S, A, Av, b, x, cap, ev, true)
                              : enqueue_cycle(S, A, Av, b, x, cap, ev, true);
  const cudaError_t ce = cudaStreamEndCapture(cap, &graph);
  if (cs != SK_OK) {
    if (graph) cudaGraphDestroy(graph);
    return cs;
  }
  if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamEndCapture");
  const cudaError_t ie = cudaGraphInstantiate(&gexec, graph, 0);
  kernels_per_cycle = count_kernel_nodes(graph);
  cudaGraphDestroy(graph);
  if (ie != cudaSuccess) {
    gexec = nullptr;
    return cuda_fail(ie, "cudaGraphInstantiate");
  }
  gb = b;
  gx = x;
  return SK_OK;
}

sk_status Solver::run(const double* b, double* x, double tol, sk_info* info, cudaStream_t st) {
  const int d = S.d;
  if (info) std::memset(info, 0, sizeof(*info));
  cudaStream_t cap = st;
  if (own && (st == nullptr || st == cudaStreamLegacy)) {
    cap = own;
    SK_CUDA(cudaStreamSynchronize(st));
  }
  last = cap;
  // ||b||^2 and the initial residual
  norm2_kernel<<<vec_grid(S.n), kVecThreads, 0, cap>>>(b, S.n, S.vec_part, S.vec_cnt + 1, bn2d);
  SK_CUDA(cudaGetLastError());
  SK_CUDA(cudaMemcpyAsync(S.h_out + 5, bn2d, sizeof(double), cudaMemcpyDeviceToHost, cap));
  SK_TRY(enqueue_residual(S, Av, b, x, cap));
  SK_CUDA(cudaMemcpyAsync(S.h_out, S.bb.bp.rho2, sizeof(double), cudaMemcpyDeviceToHost, cap));
  SK_CUDA(cudaStreamSynchronize(cap));
  const long long pre_launches = setup_launches + 2;  // the setup's launches count once
  setup_launches = 0;
  const double bn2 = S.h_out[5];
  if (!std::isfinite(bn2) || !std::isfinite(S.h_out[0])) { set_error("NaN/Inf in b or x"); return SK_ENAN; }
  const double bnorm = std::sqrt(bn2);
  double relres = bnorm > 0 ? std::sqrt(S.h_out[0]) / bnorm : 0.0;
  if (info) info->relres = relres;
  if (bnorm == 0) {
    SK_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * S.n, cap));
    SK_CUDA(cudaStreamSynchronize(cap));
    if (info) { info->relres = 0; info->launches = pre_launches; }
    return SK_OK;
  }
  if (relres <= tol) {
    if (info) info->launches = pre_launches;
    return SK_OK;
  }
  if (!iter && S.o.use_graph) SK_TRY(capture(b, x, cap));
  long long iter_launches = 0;
  long long iter_matvecs = 0;
  SK_CUDA(cudaEventRecord(e0, cap));
  sk_status result = SK_ENOCONV;
  int cycles = 0;
  double kmax = 0, rhat = 0;
  int width = 0;
  float phase[5] = {0, 0, 0, 0, 0};
  int iter_used = 0;
  while (cycles < S.o.maxit) {
    if (iter) {
      int built = 0;
      SK_TRY(run_iterative_cycle(S, A, Av, b, x, tol / relres, chk, cap, ev, &iter_used, &built, &iter_launches));
      iter_matvecs += built + 1;
    } else if (gexec) SK_CUDA(cudaGraphLaunch(gexec, cap));
    else SK_TRY(enqueue_cycle(S, A, Av, b, x, cap, ev, false));
    SK_CUDA(cudaStreamSynchronize(cap));
    ++cycles;
    {
      float t;
      if (cudaEventElapsedTime(&t, ev[EV_UPDATE], ev[EV_RES]) == cudaSuccess) phase[0] += t;
      if (cudaEventElapsedTime(&t, ev[EV_G], ev[EV_BASIS]) == cudaSuccess) phase[1] += t;
      if (cudaEventElapsedTime(&t, ev[EV_START], ev[EV_G]) == cudaSuccess) phase[2] += t;
      if (cudaEventElapsedTime(&t, ev[EV_BASIS], ev[EV_SB]) == cudaSuccess) phase[2] += t;
      if (cudaEventElapsedTime(&t, ev[EV_SB], ev[EV_SMALL]) == cudaSuccess) phase[3] += t;
      if (cudaEventElapsedTime(&t, ev[EV_SMALL], ev[EV_UPDATE]) == cudaSuccess) phase[4] += t;
    }
    const double rho2 = S.h_out[0];
    rhat = S.h_out[1];
    const double kap = S.h_out[2];
    width = (int)S.h_out[3];
    if (kap > kmax) kmax = kap;
    if (*S.h_err) { set_error("persistent basis: a grid barrier timed out"); result = SK_ETIMEOUT; break; }
    if (!std::isfinite(rho2)) { set_error("NaN/Inf in the residual"); result = SK_ENAN; break; }
    relres = std::sqrt(rho2) / bnorm;
    if (relres <= tol) { result = SK_OK; break; }
    if (width == 0) { set_error("kappa(T) above stab_tol already for one column"); result = SK_EILLCOND; break; }
  }
  SK_CUDA(cudaEventRecord(e1, cap));
  SK_CUDA(cudaEventSynchronize(e1));
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  if (info) {
    int stop = 0;
    cudaMemcpy(&stop, S.bb.bp.stop, sizeof(int), cudaMemcpyDeviceToHost);
    info->cycles = cycles;
    info->matvecs = iter ? (int)iter_matvecs + 1 : cycles * (d + 1) + 1;
    info->d_used = iter ? iter_used : (stop < d ? stop : d);
    info->width = width;
    info->relres = relres;
    info->rhat_est = rhat;
    info->kappa_T_max = kmax;
    for (int q = 0; q < 5; ++q) info->ms[q] = phase[q];
    info->ms[5] = ms;
    info->launches = pre_launches + (iter ? iter_launches : kernels_per_cycle * cycles);
  }
  if (result == SK_ENOCONV) set_error("no convergence to tol=%g in %d cycles (relres %g)", tol, cycles, relres);
  return result;
}

}  // namespace sk

// A reusable solver: the library object behind sgmres_plan_*.
struct sk_solver {
  sk::Solver core;
};

// Restarted sGMRES after argument validation (also the per-job body of the
// batched driver's worker threads).
static sk_status sgmres_impl(const sk_op* A, const double* b, double* x, int d, int k, int s, double tol,
                             const sk_opts* opts, sk_info* info, cudaStream_t st, double* h_pinned = nullptr) {
  sk::Solver sv;
  SK_TRY(sv.setup(A, d, k, s, opts, st, h_pinned));
  return sv.run(b, x, tol, info, st);
}


// Device workspace of one sgmres_solve call: the buffers Solver::setup
// allocates, in the same order, each rounded up to 256 bytes.
extern "C" size_t sk_workspace_bytes(const sk_op* A, int d, int k, int s, const sk_opts* opts) {
  if (!A || d < 1 || k < 1 || k > d || k > kMaxK || s < d + 1 || d > 768) return 0;
  sk_opts o;
  resolve_opts(opts, &o, d);
  if (!(o.basis == SK_F64 || o.basis == SK_F32 || o.basis == SK_BF16)) return 0;
  auto r = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const int64_t n = A->n;
  const size_t esz = dtype_size(o.basis);
  const bool iter = o.iter_chunk != 0;
  const bool cheb = o.basis_kind == SK_BASIS_CHEBYSHEV;
  size_t t = 0;
  // basis buffers
  t += r((size_t)((n + 7) / 8) * 8 * (d + 1) * esz);
  if (o.basis == SK_F64) t += r((size_t)n * 8);
  int pg = 0, pe = 0;
  size_t psm = 0;
  if (o.persistent && !iter && !cheb && persist_shape(A, o.basis, k, &pg, &pe, &psm))
    t += r(2 * sizeof(unsigned)) + r(sizeof(int)) + r((size_t)3 * pg * (kMaxK + 1) * 8);
  const int nblk_cap = basis_grid(n, 1);
  t += r(((size_t)2 * d * k + 2 * (size_t)d + (size_t)(d + 1) * d + (size_t)nblk_cap * (kMaxK + 1) + 2 +
          (size_t)d * (kMaxK + 1)) * 8);
  t += r(8 * sizeof(unsigned)) + r(2 * sizeof(int));
  if (cheb) t += r((size_t)(d + 1) * 8) + r((size_t)(d + 1) * nblk_cap * 8);
  // the sketch plan and its workspaces
  sk_sketch sks{o.sketch, n, s, o.zeta, o.seed};
  SketchPlan sp;
  SrhtPlan hp;
  t += sketch_plan_shape(sks, &sp, &hp);
  auto ws = [&](int c, sk_dtype dt, bool blk) {
    return sks.kind == SK_SRHT ? srht_ws_doubles(hp, c, blk) : plan_ws_doubles(sp, c, dt, blk);
  };
  t += r((size_t)n * 8) + r((size_t)s * 8) + 2 * r((size_t)s * (d + 1) * 8) + 2 * r((size_t)d * 8) +
       r((size_t)((d + kQrNb - 1) / kQrNb) * kQrNb * kQrNb * 8) + r((size_t)d * 8) + r(ws(1, SK_F64, false) * 8);
  size_t wsb = ws(d + 1, o.basis, true);
  for (int c = 1; iter && c <= o.iter_chunk + 1 && c <= d + 1; ++c) wsb = std::max(wsb, ws(c, o.basis, true));
  t += r(wsb * 8);
  if (iter) t += r(2 * sizeof(int)) + r(8);  // the chunk check and the device tau
  t += r((size_t)vec_grid(n) * 8) + r(2 * sizeof(unsigned)) + r(4 * 8) + r(8);
  return t;
}

extern "C" sk_status sgmres_solve(const sk_op* A, const double* b, double* x, int d, int k, int s, double tol,
                                  const sk_opts* opts, sk_info* info, void* stream) {
  SK_CHECK_ARG(A != nullptr && b != nullptr && x != nullptr, "NULL argument");
  SK_CHECK_ARG(d >= 1 && k >= 1 && k <= d, "need d >= 1 and 1 <= k <= d");
  SK_CHECK_ARG(k <= kMaxK, "k <= 16 supported");
  SK_CHECK_ARG(s >= d + 1, "need s >= d + 1");
  SK_CHECK_ARG(tol > 0, "tol > 0");
  SK_CHECK_ARG(d <= 768, "d <= 768");
  return sgmres_impl(A, b, x, d, k, s, tol, opts, info, (cudaStream_t)stream);
}

extern "C" sk_status sgmres_plan_create(const sk_op* A, int d, int k, int s, const sk_opts* opts, sk_solver** out,
                                        void* stream) {
  SK_CHECK_ARG(A != nullptr && out != nullptr, "NULL argument");
  *out = nullptr;
  SK_CHECK_ARG(d >= 1 && k >= 1 && k <= d, "need d >= 1 and 1 <= k <= d");
  SK_CHECK_ARG(k <= kMaxK, "k <= 16 supported");
  SK_CHECK_ARG(s >= d + 1, "need s >= d + 1");
  SK_CHECK_ARG(d <= 768, "d <= 768");
  sk_solver* p = new (std::nothrow) sk_solver;
  if (!p) { set_error("out of host memory"); return SK_ENOMEM; }
  cudaStream_t st = (cudaStream_t)stream;
  sk_status r = p->core.setup(A, d, k, s, opts, st, nullptr);
  if (r == SK_OK) r = p->core.sc->alloc(&p->core.hb, (size_t)A->n);
  if (r == SK_OK) r = p->core.sc->alloc(&p->core.hx, (size_t)A->n);
  if (r == SK_OK) {
    const cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) r = cuda_fail(e, "cudaStreamSynchronize");
  }
  if (r != SK_OK) {
    delete p;
    return r;
  }
  *out = p;
  return SK_OK;
}

extern "C" sk_status sgmres_plan_solve(sk_solver* p, const double* b, double* x, double tol, sk_info* info,
                                       void* stream) {
  SK_CHECK_ARG(p != nullptr && b != nullptr && x != nullptr, "NULL argument");
  SK_CHECK_ARG(tol > 0, "tol > 0");
  cudaStream_t st = (cudaStream_t)stream;
  Solver& c = p->core;
  const size_t bytes = sizeof(double) * (size_t)c.S.n;
  SK_CUDA(cudaMemcpyAsync(c.hb, b, bytes, cudaMemcpyDeviceToDevice, st));
  SK_CUDA(cudaMemcpyAsync(c.hx, x, bytes, cudaMemcpyDeviceToDevice, st));
  const sk_status r = c.run(c.hb, c.hx, tol, info, st);
  std::string msg = r != SK_OK ? sk_last_error() : std::string();
  // x receives the last iterate whatever the status
  cudaStream_t done = c.last ? c.last : st;
  SK_CUDA(cudaMemcpyAsync(x, c.hx, bytes, cudaMemcpyDeviceToDevice, done));
  SK_CUDA(cudaStreamSynchronize(done));
  if (r != SK_OK) set_error("%s", msg.c_str());
  return r;
}

extern "C" void sgmres_plan_destroy(sk_solver* p) { delete p; }

// ----------------------------------------------------------------------------
// Batched sGMRES: many independent (system, right-hand side) jobs of uneven
// size.  A pool of worker threads, each with its own stream, takes jobs from
// a queue ordered by decreasing size (longest-processing-time first); every
// job runs the single-system path above (one captured graph per restart
// cycle), so small systems from several workers fill the GPU together.
// ----------------------------------------------------------------------------
extern "C" sk_status sgmres_solve_batched(int nsys, const sk_op* const* A, int nrhs, const double* const* b,
                                          double* const* x, int d, int k, int s, double tol, const sk_opts* opts,
                                          sk_status* per_job, sk_info* job_info, sk_info* info, void* stream) {
  SK_CHECK_ARG(nsys >= 1 && nrhs >= 1, "need nsys >= 1 and nrhs >= 1");
  SK_CHECK_ARG(A != nullptr && b != nullptr && x != nullptr, "NULL argument");
  SK_CHECK_ARG(d >= 1 && k >= 1 && k <= d && k <= kMaxK && s >= d + 1 && tol > 0 && d <= 768,
               "need 1 <= k <= min(d, 16), s >= d + 1, tol > 0, d <= 768");
  const int njobs = nsys * nrhs;
  for (int i = 0; i < nsys; ++i) SK_CHECK_ARG(A[i] != nullptr, "NULL operator");
  for (int j = 0; j < njobs; ++j) SK_CHECK_ARG(b[j] != nullptr && x[j] != nullptr, "NULL right-hand side or solution");
  sk_opts o;
  if (opts) o = *opts;
  else sk_opts_default(&o);
  bool grouped = false;
  {
    sk_opts ro;
    resolve_opts(&o, &ro, d);
    std::string why;
    const bool ok = grouped_supported(ro, d, s, &why);
    if (o.batch_mode == 1 && !ok) {
      set_error("invalid argument: grouped batches (batch_mode = 1) need %s", why.c_str());
      return SK_EINVAL;
    }
    grouped = o.batch_mode != 2 && ok;
  }
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0;
  SK_CUDA(cudaGetDevice(&dev));
  // FP32 parameter copies of every operator, before the workers share them
  if (o.basis != SK_F64) {
    for (int i = 0; i < nsys; ++i) {
      OpView<float> Af;
      SK_TRY(make_view(A[i], &Af, st));
    }
  }
  if (grouped) return sgmres_batched_grouped(nsys, A, nrhs, b, x, d, k, s, tol, o, per_job, job_info, info, st);
  // Worker threads: per-job graph instantiation serialises the host threads
  // (hundreds of kernel nodes per cycle for each small job), so these jobs
  // launch eagerly.
  o.use_graph = 0;
  int workers = o.batch_workers > 0 ? o.batch_workers : 16;
  if (workers > njobs) workers = njobs;
  if (workers > 128) workers = 128;
  std::vector<int> order(njobs);
  for (int j = 0; j < njobs; ++j) order[j] = j;
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return A[a / nrhs]->n > A[c / nrhs]->n; });
  cudaEvent_t start_ev;
  SK_CUDA(cudaEventCreateWithFlags(&start_ev, cudaEventDisableTiming));
  SK_CUDA(cudaEventRecord(start_ev, st));
  auto t0 = std::chrono::steady_clock::now();
  std::atomic<int> next(0);
  std::mutex mu;
  sk_status first_err = SK_OK;
  std::string first_msg;
  long long cycles = 0, matvecs = 0, launches = 0;
  double relmax = 0, kmax = 0;
  float msum[5] = {0, 0, 0, 0, 0};
  std::vector<cudaEvent_t> done(workers, nullptr);
  std::vector<std::thread> pool;
  for (int w = 0; w < workers; ++w) {
    pool.emplace_back([&, w]() {
      cudaSetDevice(dev);
      cudaStream_t ws = nullptr;
      if (cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking) != cudaSuccess) {
        std::lock_guard<std::mutex> lk(mu);
        if (first_err == SK_OK) { first_err = SK_ECUDA; first_msg = "batched: stream creation failed"; }
        return;
      }
      cudaStreamWaitEvent(ws, start_ev, 0);
      double* pinned = nullptr;
      if (cudaMallocHost((void**)&pinned, 8 * sizeof(double)) != cudaSuccess) pinned = nullptr;
      for (;;) {
        const int q = next.fetch_add(1);
        if (q >= njobs) break;
        const int job = order[q];
        sk_info ji;
        const sk_status r = sgmres_impl(A[job / nrhs], b[job], x[job], d, k, s, tol, &o, &ji, ws, pinned);
        std::lock_guard<std::mutex> lk(mu);
        if (per_job) per_job[job] = r;
        if (job_info) job_info[job] = ji;
        if (r != SK_OK && first_err == SK_OK) { first_err = r; first_msg = sk_last_error(); }
        cycles += ji.cycles;
        matvecs += ji.matvecs;
        launches += ji.launches;
        if (ji.relres > relmax) relmax = ji.relres;
        if (ji.kappa_T_max > kmax) kmax = ji.kappa_T_max;
        for (int p = 0; p < 5; ++p) msum[p] += ji.ms[p];
      }
      cudaEvent_t ev;
      if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess) {
        cudaEventRecord(ev, ws);
        done[w] = ev;
      }
      cudaStreamSynchronize(ws);
      cudaStreamDestroy(ws);
      if (pinned) cudaFreeHost(pinned);
    });
  }
  for (auto& t : pool) t.join();
  for (int w = 0; w < workers; ++w)
    if (done[w]) {
      cudaStreamWaitEvent(st, done[w], 0);
      cudaEventDestroy(done[w]);
    }
  cudaEventDestroy(start_ev);
  const double wall_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->cycles = (int)(cycles > 2147483647 ? 2147483647 : cycles);
    info->matvecs = (int)(matvecs > 2147483647 ? 2147483647 : matvecs);
    info->relres = relmax;
    info->kappa_T_max = kmax;
    for (int p = 0; p < 5; ++p) info->ms[p] = msum[p];
    info->ms[5] = (float)wall_ms;
    info->launches = launches;
  }
  if (first_err != SK_OK) set_error("%s", first_msg.c_str());
  return first_err;
}

extern "C" sk_status srr_eigs(const sk_op* A, const double* w1, int nev, int d, int k, int s, const sk_opts* opts,
                              double* lam_re, double* lam_im, double* X_re, double* X_im, double* rhat, int* nconv,
                              sk_info* info, void* stream) {
  SK_CHECK_ARG(A != nullptr && w1 != nullptr && lam_re != nullptr && X_re != nullptr, "NULL argument");
  SK_CHECK_ARG(d >= 3 && d <= kMaxSrrD, "sRR needs 3 <= d <= 232");
  SK_CHECK_ARG(nev >= 1 && nev <= d && nev <= kMaxNev, "need 1 <= nev <= min(d, 32)");
  SK_CHECK_ARG(k >= 1 && k <= d && k <= kMaxK, "need 1 <= k <= min(d, 16)");
  SK_CHECK_ARG(s >= d, "need s >= d");
  cudaStream_t st = (cudaStream_t)stream;
  sk_opts o;
  resolve_opts(opts, &o, d);
  SK_CHECK_ARG(o.basis == SK_F64 || o.basis == SK_F32 || o.basis == SK_BF16, "basis dtype");
  SK_TRY(check_passes(o));
  SK_CHECK_ARG(o.basis_kind == SK_BASIS_ARNOLDI, "srr_eigs uses the truncated-Arnoldi basis");
  if (info) std::memset(info, 0, sizeof(*info));
  const int64_t n = A->n;
  Scratch sc(st);
  cudaEvent_t e0, e1;
  SK_CUDA(cudaEventCreate(&e0));
  SK_CUDA(cudaEventCreate(&e1));
  struct EvFree { cudaEvent_t a, b; ~EvFree() { cudaEventDestroy(a); cudaEventDestroy(b); } } ef{e0, e1};
  SK_CUDA(cudaEventRecord(e0, st));
  BasisBuffers bb;
  SK_TRY(bb.alloc(n, d, k, o.basis, o.cgs_passes, o.breakdown, sc, nullptr, A, o.persistent != 0));
  bb.bp.r = w1;
  {
    double* part = nullptr;
    unsigned* cnt = nullptr;
    SK_TRY(sc.alloc(&part, vec_grid(n)));
    SK_TRY(sc.alloc(&cnt, 1));
    SK_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned), st));
    norm2_kernel<<<vec_grid(n), kVecThreads, 0, st>>>(w1, n, part, cnt, bb.rho2_mut());
    SK_CUDA(cudaGetLastError());
  }
  SK_TRY(enqueue_basis_build(bb, A, st));
  Sketcher skt;
  sk_sketch sks;
  sks.kind = o.sketch;
  sks.n = n;
  sks.s = s;
  sks.zeta = o.zeta;
  sks.seed = o.seed;
  SK_TRY(skt.create(sks, sc, st));
  double *SB, *ws, *Aug;
  SK_TRY(sc.alloc(&SB, (size_t)s * (d + 1)));
  SK_TRY(sc.alloc(&ws, skt.ws(d + 1, o.basis, true)));
  SK_TRY(sc.alloc(&Aug, (size_t)s * 2 * d));
  // C = S B (columns 0..d-1), D = S A B = (S B_{d+1}) Hbar
  SK_TRY(skt.apply(bb.bp.B, bb.bp.ldb, d + 1, o.basis, SB, ws, st, true));
  SK_TRY(enqueue_copy_sb(SB, s, d, bb.bp.stop, Aug, st));
  SK_TRY(enqueue_hbar_product(SB, bb.bp.Hbar, s, d, k, bb.bp.stop, Aug + (size_t)s * d, st));
  int hstat[2] = {0, 0};
  SK_CUDA(cudaMemcpyAsync(hstat, bb.bp.stop, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
  SK_CUDA(cudaStreamSynchronize(st));
  if (hstat[1]) { set_error("NaN/Inf in the basis recurrence"); return SK_ENAN; }
  if (hstat[0] < d) { set_error("basis breakdown at %d < d columns; sRR on a partial basis is not supported", hstat[0]); return SK_EILLCOND; }
  SrrOut out{lam_re, lam_im, X_re, X_im, rhat, nconv, nullptr};
  int eig_fail = 0;
  SK_TRY(srr_tail(Aug, s, d, bb.bp.B, bb.bp.ldb, n, o.basis, nullptr, nev, o.symmetric, o.tau, o.srr_trunc_tol, out,
                  sc, st, &eig_fail));
  SK_CUDA(cudaEventRecord(e1, st));
  SK_CUDA(cudaEventSynchronize(e1));
  if (info) {
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    info->ms[5] = ms;
    info->cycles = 1;
    info->d_used = d;
  }
  if (eig_fail) { set_error("eigensolver: QR iteration did not converge"); return SK_ENOCONV; }
  return SK_OK;
}
