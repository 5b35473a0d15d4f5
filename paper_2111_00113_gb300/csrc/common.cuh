// Shared device/host helpers of libsk: status handling, element types,
// block reductions, the counter hash and operator views.
#pragma once

#include <cuda_runtime.h>
#include <cuda/atomic>
#include <cuda_bf16.h>
#include <stdint.h>
#include <string>

#include "../../include/sk.h"

namespace sk {

// ----------------------------------------------------------------------------
// Errors: thread-local message, status propagation without exceptions.
// ----------------------------------------------------------------------------
void set_error(const char* fmt, ...);
sk_status cuda_fail(cudaError_t e, const char* what);

#define SK_CUDA(call)                                                   \
  do {                                                                  \
    cudaError_t _e = (call);                                            \
    if (_e != cudaSuccess) return ::sk::cuda_fail(_e, #call);           \
  } while (0)

#define SK_TRY(call)                                                    \
  do {                                                                  \
    sk_status _s = (call);                                              \
    if (_s != SK_OK) return _s;                                         \
  } while (0)

#define SK_CHECK_ARG(cond, msg)                                         \
  do {                                                                  \
    if (!(cond)) { ::sk::set_error("invalid argument: %s", msg); return SK_EINVAL; } \
  } while (0)

// Opt-in dynamic shared memory limit set on every kernel that uses more than
// 48 KB.  One fixed value (not the size of a particular launch): a captured
// graph keeps its launches' sizes while the attribute is per function, so
// the attribute must cover every launch of the function.
static constexpr int kDynSmemLimit = 200 * 1024;

inline int num_sms() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

// Stream-ordered scratch owned by one call; freed (stream-ordered) on scope exit.
struct Scratch {
  cudaStream_t st;
  void* ptr[32];
  int n = 0;
  explicit Scratch(cudaStream_t s) : st(s) {}
  ~Scratch() {
    for (int i = 0; i < n; ++i)
      if (ptr[i]) cudaFreeAsync(ptr[i], st);
  }
  template <typename T>
  sk_status alloc(T** p, size_t count) {
    *p = nullptr;
    if (n >= 32) { set_error("scratch: too many buffers"); return SK_ENOMEM; }
    if (count == 0) count = 1;
    cudaError_t e = cudaMallocAsync((void**)p, count * sizeof(T), st);
    if (e != cudaSuccess) { cudaGetLastError(); set_error("cudaMallocAsync(%zu bytes) failed: %s", count * sizeof(T), cudaGetErrorString(e)); return SK_ENOMEM; }
    ptr[n++] = *p;
    return SK_OK;
  }
};

// ----------------------------------------------------------------------------
// Element types: storage T, compute type C (double for FP64 storage, float
// for FP32 and BF16 storage).
// ----------------------------------------------------------------------------
template <typename T> struct Compute { using type = float; };
template <> struct Compute<double> { using type = double; };

__device__ __forceinline__ double to_c(double v) { return v; }
__device__ __forceinline__ float to_c(float v) { return v; }
__device__ __forceinline__ float to_c(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename T> __device__ __forceinline__ T from_c(typename Compute<T>::type v);
template <> __device__ __forceinline__ double from_c<double>(double v) { return v; }
template <> __device__ __forceinline__ float from_c<float>(float v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 from_c<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

inline size_t dtype_size(sk_dtype t) { return t == SK_F64 ? 8 : (t == SK_F32 ? 4 : 2); }

// ----------------------------------------------------------------------------
// Block reductions (deterministic order).
// ----------------------------------------------------------------------------
template <typename V>
__device__ __forceinline__ V warp_sum(V v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum K values over the block; result valid in thread 0.  `sh` needs
// K * (blockDim/32) entries.  Ends with a __syncthreads (sh reusable after).
template <int K, typename V>
__device__ __forceinline__ void block_sum_k(V (&v)[K], V* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int q = 0; q < K; ++q) v[q] = warp_sum(v[q]);
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < K; ++q) sh[q * nw + wid] = v[q];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < K; ++q) {
      V a = 0;
      for (int w = 0; w < nw; ++w) a += sh[q * nw + w];
      v[q] = a;
    }
  }
  __syncthreads();
}

// Last-block-done: every block calls this after writing its partials;
// the function returns true in exactly one block (the last to arrive).  One
// acq_rel atomic by thread 0 replaces fences by every thread: the barrier
// before it orders the block's partial writes before thread 0's release, and
// in the last block the barrier after it orders every thread's reads of the
// partials after thread 0's acquire.  The counter is reset by the last block
// so that the launch can be replayed (CUDA graphs).
// `nblocks` blocks share the counter (the whole grid, or one job's blocks of
// a grouped launch).
__device__ __forceinline__ bool last_block_arrived_n(unsigned int* counter, unsigned nblocks) {
  __shared__ bool s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    cuda::atomic_ref<unsigned int, cuda::thread_scope_device> c(*counter);
    const unsigned prev = c.fetch_add(1u, cuda::memory_order_acq_rel);
    s_last = (prev == nblocks - 1);
    if (s_last) c.store(0u, cuda::memory_order_relaxed);
  }
  __syncthreads();
  return s_last;
}
__device__ __forceinline__ bool last_block_arrived(unsigned int* counter) {
  return last_block_arrived_n(counter, gridDim.x * gridDim.y);
}

// Grouped launches of the batched solver over its small dense problems:
// blockIdx.y picks job slot ids[blockIdx.y] (ids NULL: slot blockIdx.y),
// whose buffers lie `stride` bytes apart (one slab per slot, the same
// layout in every slab).  stride = 0: a single problem (grid.y = 1).
struct JobSlab {
  const int* ids = nullptr;
  int64_t stride = 0;
};
template <typename P>
__device__ __forceinline__ P* at_job(P* p, const JobSlab& js) {
  if (js.stride == 0) return p;
  const int64_t j = js.ids ? js.ids[blockIdx.y] : blockIdx.y;
  return reinterpret_cast<P*>(reinterpret_cast<uintptr_t>(p) + j * js.stride);
}

// ----------------------------------------------------------------------------
// Counter hash H1 (bit-exact definition in include/sk.h).
// ----------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z ^= z >> 30;
  z *= 0xBF58476D1CE4E5B9ull;
  z ^= z >> 27;
  z *= 0x94D049BB133111EBull;
  z ^= z >> 31;
  return z;
}
__host__ __device__ __forceinline__ uint64_t h1(uint64_t seedkey, uint64_t i, uint32_t t, uint32_t a) {
  return mix64(seedkey ^ ((i << 8) | ((uint64_t)t << 4) | (uint64_t)a));
}
__host__ __device__ __forceinline__ uint64_t seed_key(uint64_t seed) { return seed * 0x9E3779B97F4A7C15ull; }
__host__ __device__ __forceinline__ uint32_t h1_row(uint64_t x, uint32_t s) {
  return (uint32_t)(((x & 0xFFFFFFFFull) * (uint64_t)s) >> 32);
}
__host__ __device__ __forceinline__ bool h1_neg(uint64_t x) { return (x >> 63) != 0; }

// ----------------------------------------------------------------------------
// Operators: device views templated on the compute type C.
// ----------------------------------------------------------------------------
enum OpKind { OP_STENCIL5 = 0, OP_DIFFUSION = 1, OP_CSR = 2 };

}  // namespace sk

// Library-side operator object (opaque in the C ABI).
struct sk_op {
  int kind;
  int nx, ny;
  int64_t n;
  double coef[5];
  const double* shift;    // borrowed, device, nullable
  const double* theta;    // borrowed, device
  const int32_t* rowptr;  // borrowed, device
  const int32_t* colind;
  const double* val;
  int64_t nnz;
  // FP32 copies owned by the op (made on first use by an FP32/BF16 solve)
  float* shift32;
  float* theta32;
  float* val32;
  bool owns_nothing_else;
  // CSR: the SELL-32 copy the kernels read (owned; built by sk_op_csr and
  // sk_op_transpose): slice q (rows 32q .. 32q+31) has width w_q and its
  // entries column-major at sell_ptr[q] + e*32 + (row % 32), e < w_q, padded
  // with zero values; so a warp of consecutive rows reads consecutive words.
  int64_t* sell_ptr;      // nslices + 1
  int32_t* sell_col;
  double* sell_val;
  float* sell_val32;
  // a transposed CSR op owns its CSR arrays (rowptr, colind, val above)
  int32_t* own_rowptr;
  int32_t* own_colind;
  double* own_val;
};

namespace sk {

template <typename C>
struct OpView {
  int kind;
  int nx, ny;
  int64_t n;
  C cP, cE, cW, cN, cS;
  const C* shift;
  const C* theta;
  const int32_t* rowptr;
  const int32_t* colind;
  const C* val;
  const int64_t* sell_ptr;  // SELL-32 (see sk_op); NULL: plain CSR rows
  const int32_t* sell_col;
  const C* sell_val;
  // i / nx for 0 <= i < 2^31 as (i * nx_m) >> nx_s (nx_s = 0: plain division);
  // set by make_view (set_div_magic)
  uint64_t nx_m;
  int nx_s;

  // grid position of unknown i: column ix, row iy
  __device__ __forceinline__ void grid_pos(int64_t i, int& ix, int64_t& iy) const {
    if (nx_s) {
      const int64_t q = (int64_t)(((uint64_t)i * nx_m) >> nx_s);
      iy = q;
      ix = (int)(i - q * nx);
    } else {
      iy = i / nx;
      ix = (int)(i - iy * nx);
    }
  }

  // (A x)_i, x of storage type T (converted to C on load).
  template <typename T>
  __device__ __forceinline__ C apply(const T* __restrict__ x, int64_t i) const {
    if (kind == OP_STENCIL5) {
      int ix;
      int64_t iy;
      grid_pos(i, ix, iy);
      C acc = cP * to_c(x[i]);
      if (ix + 1 < nx) acc += cE * to_c(x[i + 1]);
      if (ix > 0) acc += cW * to_c(x[i - 1]);
      if (iy + 1 < ny) acc += cN * to_c(x[i + nx]);
      if (iy > 0) acc += cS * to_c(x[i - nx]);
      if (shift) acc += shift[i] * to_c(x[i]);
      return acc;
    } else if (kind == OP_DIFFUSION) {
      int ix;
      int64_t iy;
      grid_pos(i, ix, iy);
      const C tP = theta[i];
      const C xP = to_c(x[i]);
      C acc = 0;
      // interior faces (theta_P+theta_Q)/2 (xP - xQ); boundary faces theta_P xP
      acc += (ix + 1 < nx) ? (C)0.5 * (tP + theta[i + 1]) * (xP - to_c(x[i + 1])) : tP * xP;
      acc += (ix > 0) ? (C)0.5 * (tP + theta[i - 1]) * (xP - to_c(x[i - 1])) : tP * xP;
      acc += (iy + 1 < ny) ? (C)0.5 * (tP + theta[i + nx]) * (xP - to_c(x[i + nx])) : tP * xP;
      acc += (iy > 0) ? (C)0.5 * (tP + theta[i - nx]) * (xP - to_c(x[i - nx])) : tP * xP;
      return acc;
    } else if (sell_ptr) {
      // row i = lane (i % 32) of slice i / 32: consecutive rows, consecutive words
      C acc = 0;
      const int64_t q = i >> 5, base = sell_ptr[q] + (i & 31);
      const int w = (int)((sell_ptr[q + 1] - sell_ptr[q]) >> 5);
      for (int e = 0; e < w; ++e) acc += sell_val[base + 32 * (int64_t)e] * to_c(x[sell_col[base + 32 * (int64_t)e]]);
      return acc;
    } else {
      C acc = 0;
      const int32_t e0 = rowptr[i], e1 = rowptr[i + 1];
      for (int32_t e = e0; e < e1; ++e) acc += val[e] * to_c(x[colind[e]]);
      return acc;
    }
  }
};

// Division by the invariant nx (Granlund and Montgomery, "Division by
// invariant integers using multiplication", 1994): with l = ceil(log2 nx) and
// m = floor(2^(31+l) / nx) + 1, (i * m) >> (31 + l) = floor(i / nx) for every
// 0 <= i < 2^31, because i * m / 2^(31+l) exceeds i / nx by less than
// 2^-l <= 1/nx, too little to cross the next integer; i * m < 2^64.  Views of
// operators with n > 2^31 keep plain division.
inline void set_div_magic(int nx, int64_t n, uint64_t* m, int* s) {
  *m = 0;
  *s = 0;
  if (nx < 1 || n > (1ll << 31)) return;
  int l = 0;
  while ((1ll << l) < nx) ++l;
  *s = 31 + l;
  *m = ((1ull << (31 + l)) / (uint64_t)nx) + 1;
}

// Build a view for compute type C (FP32 views use the op's FP32 copies).
sk_status make_view(const sk_op* op, OpView<double>* v);
sk_status make_view(const sk_op* op, OpView<float>* v, cudaStream_t st);

// Internal entry points shared between translation units.
sk_status sketch_apply_impl(const sk_sketch* S, const void* B, int64_t ldb, int ncols, sk_dtype dtype,
                            double* SB, cudaStream_t st);

struct SketchPlan {
  int64_t n = 0;
  int s = 0, zeta = 0;
  uint64_t seed = 0;
  int L = 0;           // chunk length (rows of the data per chunk)
  int nchunks = 0;
  uint32_t* rowptr = nullptr;   // nchunks x (s+1)
  uint16_t* entries = nullptr;  // nchunks x (L*zeta): bit15 = negative, bits0..14 = local index
  int* d_status = nullptr;      // device int: nonzero if the hash failed
};
sk_status plan_create(SketchPlan* p, const sk_sketch* S, Scratch& scratch, cudaStream_t st);
sk_status plan_apply(const SketchPlan& p, const void* B, int64_t ldb, int ncols, sk_dtype dtype,
                     double* SB, Scratch& scratch, cudaStream_t st);
// block = true: a sketch of basis columns inside a solver (fixed grouping,
// the same per-column summation order for any column count; see sketch.cu).
size_t plan_ws_doubles(const SketchPlan& p, int ncols, sk_dtype dtype, bool block = false);
sk_status plan_apply_ws(const SketchPlan& p, const void* B, int64_t ldb, int ncols, sk_dtype dtype, double* SB,
                        double* partial, cudaStream_t st, bool block = false);
sk_status check_plan_status(const SketchPlan& p, cudaStream_t st);
struct SrhtPlan;
// The device bytes of the plan for S and the shape fields that the
// workspace queries (plan_ws_doubles, srht_ws_doubles) read; allocates nothing.
size_t sketch_plan_shape(const sk_sketch& S, SketchPlan* sp, SrhtPlan* hp);
int default_zeta_for(int d);

struct SrhtPlan {
  int64_t n = 0, n_p = 0;
  int s = 0, logn = 0, b = 0;
  uint32_t* sign_bits = nullptr;  // n bits, 1 = negative
  int32_t* rows = nullptr;        // s sampled Hadamard rows
};
sk_status srht_plan_create(SrhtPlan* p, const sk_sketch* S, Scratch& scratch, cudaStream_t st);
size_t srht_ws_doubles(const SrhtPlan& p, int ncols, bool block = false);
sk_status srht_apply_ws(const SrhtPlan& p, const void* B, int64_t ldb, int ncols, sk_dtype dtype, double* SB,
                        double* partial, cudaStream_t st, bool block = false);

}  // namespace sk
