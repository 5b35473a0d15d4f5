// Sparse sign sketch (§2.3.2, eq. (sparse-map)) on the GPU.
//
// A plan turns the counter hash into per-chunk, row-sorted index tables once;
// applying S is then a deterministic gather: for each chunk of L data rows
// staged in shared memory, sketch row r sums +-x[i] over the entries of row r
// (no atomics, fixed summation order).  Partial sums per group of chunks are
// combined in FP64 in a second kernel.
#include <cstdio>
#include <cmath>
#include <mutex>
#include <type_traits>
#include <vector>

#include "common.cuh"
#include "grouped.cuh"

namespace sk {

static constexpr int kChunk = 1024;      // data rows per chunk (local index fits 15 bits)
static constexpr int kMaxSparseS = 4096; // embedding dimension limit of the gather path
static constexpr int kPlanThreads = 256;

// Row offsets of a chunk are stored with a stride padded to 16 bytes so that
// they can be staged with 16-byte asynchronous copies.
__host__ __device__ static inline int64_t rp_stride(int s) { return ((int64_t)s + 1 + 3) / 4 * 4; }

int default_zeta_for(int d) {
  int z = (int)std::ceil(2.0 * std::log1p((double)d));
  if (z < 1) z = 1;
  if (z > 14) z = 14;
  return z;
}

// ----------------------------------------------------------------------------
// Plan build: one CTA per chunk.
// ----------------------------------------------------------------------------
__global__ void __launch_bounds__(kPlanThreads)
plan_build_kernel(int64_t n, int s, int zeta, uint64_t skey, uint32_t* __restrict__ rowptr,
                  uint16_t* __restrict__ entries, int* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int c = blockIdx.x;
  const int64_t i0 = (int64_t)c * kChunk;
  const int Lc = (int)((n - i0) < kChunk ? (n - i0) : kChunk);
  const int ne = Lc * zeta;
  uint16_t* packed = (uint16_t*)smem_raw;                 // kChunk*zeta
  uint16_t* sorted = packed + kChunk * zeta;             // kChunk*zeta
  uint32_t* counts = (uint32_t*)(sorted + kChunk * zeta); // s
  uint32_t* offs = counts + s;                            // s+1
  uint32_t* seg = offs + s + 1;                           // kPlanThreads

  for (int r = threadIdx.x; r < s; r += blockDim.x) counts[r] = 0;
  // 1. rows and signs: slot t takes the first attempt whose row is new
  for (int il = threadIdx.x; il < Lc; il += blockDim.x) {
    const uint64_t i = (uint64_t)(i0 + il);
    uint16_t rows[16];
    for (int t = 0; t < zeta; ++t) {
      bool done = false;
      for (uint32_t a = 0; a < 16 && !done; ++a) {
        const uint64_t x = h1(skey, i, (uint32_t)t, a);
        const uint32_t r = h1_row(x, (uint32_t)s);
        bool clash = false;
        for (int tp = 0; tp < t; ++tp) clash |= (rows[tp] == r);
        if (!clash) {
          rows[t] = (uint16_t)r;
          packed[il * zeta + t] = (uint16_t)(r | (h1_neg(x) ? 0x8000u : 0u));
          done = true;
        }
      }
      if (!done) {
        atomicExch(status, 1);
        rows[t] = 0xFFFF;
        packed[il * zeta + t] = 0;  // keep the table well formed
      }
    }
  }
  __syncthreads();
  // 2. histogram of rows
  for (int e = threadIdx.x; e < ne; e += blockDim.x) atomicAdd(&counts[packed[e] & 0x7FFF], 1u);
  __syncthreads();
  // 3. exclusive scan of counts (segmented over threads)
  {
    const int per = (s + blockDim.x - 1) / blockDim.x;
    const int r0 = threadIdx.x * per;
    uint32_t acc = 0;
    for (int r = r0; r < r0 + per && r < s; ++r) acc += counts[r];
    seg[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t run = 0;
      for (int w = 0; w < (int)blockDim.x; ++w) { uint32_t v = seg[w]; seg[w] = run; run += v; }
    }
    __syncthreads();
    uint32_t run = seg[threadIdx.x];
    for (int r = r0; r < r0 + per && r < s; ++r) { offs[r] = run; run += counts[r]; }
    if (threadIdx.x == 0) offs[s] = (uint32_t)ne;
  }
  __syncthreads();
  for (int r = threadIdx.x; r <= s; r += blockDim.x) rowptr[(int64_t)c * rp_stride(s) + r] = offs[r];
  // 4. placement (order inside a row fixed in step 5)
  for (int r = threadIdx.x; r < s; r += blockDim.x) counts[r] = offs[r];
  __syncthreads();
  for (int e = threadIdx.x; e < ne; e += blockDim.x) {
    const uint16_t p = packed[e];
    const uint32_t pos = atomicAdd(&counts[p & 0x7FFF], 1u);
    sorted[pos] = (uint16_t)((e / zeta) | (p & 0x8000));
  }
  __syncthreads();
  // 5. sort each row's entries by local index (a deterministic start for step 6)
  for (int r = threadIdx.x; r < s; r += blockDim.x) {
    const int b = (int)offs[r], e = (int)offs[r + 1];
    for (int q = b + 1; q < e; ++q) {
      const uint16_t v = sorted[q];
      int p = q - 1;
      while (p >= b && (sorted[p] & 0x7FFF) > (v & 0x7FFF)) { sorted[p + 1] = sorted[p]; --p; }
      sorted[p + 1] = v;
    }
  }
  __syncthreads();
  // 6. bank-aware order: the row-owner gather reads, at each step, one entry
  // of each of 8 consecutive rows with one quarter-warp phase of a 16-byte
  // shared load, whose bank group is fixed by the tile row (rows of 64
  // bytes whose segments rotate by row >> 1: group ((il & 1), (il >> 1) & 3)).
  // Greedily give each of the 8 rows, step by step, a remaining entry whose
  // group is least used in that step so far (first such entry: deterministic).
  for (int Q = threadIdx.x; Q * 8 < s; Q += blockDim.x) {
    const int ra = Q * 8, nr = min(8, s - ra);
    int pos[8], end[8];
    for (int l = 0; l < 8; ++l) {
      pos[l] = (l < nr) ? (int)offs[ra + l] : 0;
      end[l] = (l < nr) ? (int)offs[ra + l + 1] : 0;
    }
    for (;;) {
      int cnt[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      bool any = false;
      for (int l = 0; l < nr; ++l) {
        if (pos[l] >= end[l]) continue;
        any = true;
        int best = pos[l], bc = 1 << 30;
        for (int q = pos[l]; q < end[l]; ++q) {
          const int il = sorted[q] & 0x7FFF;
          const int gq = ((il & 1) << 2) | ((il >> 1) & 3);
          if (cnt[gq] < bc) {
            bc = cnt[gq];
            best = q;
          }
        }
        const uint16_t t = sorted[best];
        sorted[best] = sorted[pos[l]];
        sorted[pos[l]] = t;
        const int il = t & 0x7FFF;
        ++cnt[((il & 1) << 2) | ((il >> 1) & 3)];
        ++pos[l];
      }
      if (!any) break;
    }
  }
  __syncthreads();
  uint16_t* out = entries + (int64_t)c * kChunk * zeta;
  for (int e = threadIdx.x; e < ne; e += blockDim.x) out[e] = sorted[e];
}

static size_t plan_smem_bytes(int s, int zeta) {
  return (size_t)2 * kChunk * zeta * sizeof(uint16_t) + (size_t)(2 * s + 1) * sizeof(uint32_t) +
         kPlanThreads * sizeof(uint32_t);
}

sk_status plan_create(SketchPlan* p, const sk_sketch* S, Scratch& scratch, cudaStream_t st) {
  SK_CHECK_ARG(S != nullptr, "sketch is NULL");
  SK_CHECK_ARG(S->kind == SK_SPARSE_SIGN, "plan_create: sparse sign sketch expected");
  SK_CHECK_ARG(S->n >= 1, "sketch n >= 1");
  SK_CHECK_ARG(S->s >= 1 && S->s <= kMaxSparseS, "sparse sign sketch needs 1 <= s <= 4096");
  int zeta = S->zeta > 0 ? S->zeta : default_zeta_for(S->s / 2);
  SK_CHECK_ARG(zeta >= 1 && zeta <= 14 && zeta <= S->s, "zeta must be in 1..min(14, s)");
  p->n = S->n;
  p->s = S->s;
  p->zeta = zeta;
  p->seed = S->seed;
  p->L = kChunk;
  p->nchunks = (int)((S->n + kChunk - 1) / kChunk);
  SK_TRY(scratch.alloc(&p->rowptr, (size_t)p->nchunks * rp_stride(p->s)));
  SK_TRY(scratch.alloc(&p->entries, (size_t)p->nchunks * kChunk * zeta));
  SK_TRY(scratch.alloc(&p->d_status, 1));
  SK_CUDA(cudaMemsetAsync(p->d_status, 0, sizeof(int), st));
  const size_t smem = plan_smem_bytes(p->s, zeta);
  SK_CUDA(cudaFuncSetAttribute(plan_build_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kDynSmemLimit));
  plan_build_kernel<<<p->nchunks, kPlanThreads, smem, st>>>(p->n, p->s, zeta, seed_key(p->seed), p->rowptr,
                                                              p->entries, p->d_status);
  SK_CUDA(cudaGetLastError());
  return SK_OK;
}

// ----------------------------------------------------------------------------
// Gather apply (general kernel: any storage type, s <= kMaxSparseS): grid
// (column tiles, chunk groups).  For each chunk the CTA
// stages the data tile (kChunk rows x W columns), the chunk's row-sorted
// entries and its row offsets in shared memory; then each group of G lanes
// owns one sketch row at a time, sums +-tile[local] over the row's entries,
// reduces inside the group by shuffles and adds the result to the CTA's
// accumulator for that row (Kahan-compensated), which only that group
// touches.
// ----------------------------------------------------------------------------
static constexpr int kApplyThreads = 512;
static constexpr int kGroup = 8;  // lanes per sketch row

template <typename C>
struct KahanAcc {
  __device__ __forceinline__ static void add(C* hi, C* lo, C v) {
    const C y = v - *lo;
    const C t = *hi + y;
    *lo = (t - *hi) - y;
    *hi = t;
  }
};

// One tile row (W values of the compute type) in shared memory.  Rows of 32
// bytes are stored as two 16-byte halves whose order is swapped on every
// other group of 4 rows, so that 8 random rows read by one quarter warp spread
// over all 8 16-byte bank groups; rows of 16 bytes or less need no swizzle.
template <typename C, int W>
struct TileRow {
  static constexpr int BYTES = W * (int)sizeof(C);
  __device__ static __forceinline__ void store(unsigned char* tile, int il, const C (&v)[W]) {
    if constexpr (BYTES == 32) {
      const int swz = (il >> 2) & 1;
      uint4 h[2];
      memcpy(&h[0], &v[0], 16);
      memcpy(&h[1], (const char*)&v[0] + 16, 16);
      *reinterpret_cast<uint4*>(tile + il * 32 + swz * 16) = h[0];
      *reinterpret_cast<uint4*>(tile + il * 32 + (swz ^ 1) * 16) = h[1];
    } else {
#pragma unroll
      for (int q = 0; q < W; ++q) reinterpret_cast<C*>(tile)[il * W + q] = v[q];
    }
  }
  __device__ static __forceinline__ void load(const unsigned char* tile, int il, C (&v)[W]) {
    if constexpr (BYTES == 32) {
      const int swz = (il >> 2) & 1;
      const uint4 a = *reinterpret_cast<const uint4*>(tile + il * 32 + swz * 16);
      const uint4 b = *reinterpret_cast<const uint4*>(tile + il * 32 + (swz ^ 1) * 16);
      memcpy(&v[0], &a, 16);
      memcpy((char*)&v[0] + 16, &b, 16);
    } else if constexpr (BYTES == 16) {
      const uint4 a = *reinterpret_cast<const uint4*>(tile + il * 16);
      memcpy(&v[0], &a, 16);
    } else if constexpr (BYTES == 8) {
      const uint2 a = *reinterpret_cast<const uint2*>(tile + il * 8);
      memcpy(&v[0], &a, 8);
    } else {
#pragma unroll
      for (int q = 0; q < W; ++q) v[q] = reinterpret_cast<const C*>(tile)[il * W + q];
    }
  }
};

__host__ __device__ static inline size_t entries_bytes(int zeta) { return (((size_t)kChunk * zeta * sizeof(uint16_t)) + 15) & ~(size_t)15; }
__host__ __device__ static inline size_t rowptr_bytes(int s) { return (((size_t)(s + 1) * sizeof(uint32_t)) + 15) & ~(size_t)15; }

template <typename T, int W>
__global__ void __launch_bounds__(kApplyThreads)
gather_apply_kernel(const T* __restrict__ B, int64_t ldb, int ncols, int64_t n, int s, int zeta, int nchunks,
                    int chunks_per_group, const uint32_t* __restrict__ rowptr, const uint16_t* __restrict__ entries,
                    double* __restrict__ partial) {
  using C = typename Compute<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tile = (C*)smem_raw;                                                     // kChunk * W
  uint16_t* ent_s = (uint16_t*)(smem_raw + (size_t)kChunk * W * sizeof(C));  // kChunk * zeta
  uint32_t* rp_s = (uint32_t*)((unsigned char*)ent_s + entries_bytes(zeta)); // s + 1
  C* acc_hi = (C*)((unsigned char*)rp_s + rowptr_bytes(s));                   // s * W
  C* acc_lo = acc_hi + (size_t)s * W;                                         // s * W
  const int col0 = blockIdx.x * W;
  const int g = blockIdx.y;
  const int c_begin = g * chunks_per_group;
  const int c_end = min(nchunks, c_begin + chunks_per_group);
  for (int q = threadIdx.x; q < s * W; q += blockDim.x) { acc_hi[q] = 0; acc_lo[q] = 0; }
  const int lane = threadIdx.x & 31;
  const int gl = lane & (kGroup - 1);
  const int row_slot = threadIdx.x / kGroup;
  const int rows_per_pass = kApplyThreads / kGroup;
  for (int c = c_begin; c < c_end; ++c) {
    const int64_t i0 = (int64_t)c * kChunk;
    const int Lc = (int)((n - i0) < kChunk ? (n - i0) : kChunk);
    const int ne = Lc * zeta;
    __syncthreads();
    for (int il = threadIdx.x; il < Lc; il += blockDim.x) {
      C v[W];
#pragma unroll
      for (int q = 0; q < W; ++q) {
        const int col = col0 + q;
        v[q] = (col < ncols) ? to_c(B[i0 + il + (int64_t)col * ldb]) : (C)0;
      }
      TileRow<C, W>::store((unsigned char*)tile, il, v);
    }
    {
      const uint4* src = reinterpret_cast<const uint4*>(entries + (int64_t)c * kChunk * zeta);
      uint4* dst = reinterpret_cast<uint4*>(ent_s);
      for (int q = threadIdx.x; q < (ne + 7) / 8; q += blockDim.x) dst[q] = __ldg(src + q);
      const uint32_t* rp = rowptr + (int64_t)c * rp_stride(s);
      for (int q = threadIdx.x; q <= s; q += blockDim.x) rp_s[q] = __ldg(rp + q);
    }
    __syncthreads();
    for (int rb = 0; rb < s; rb += rows_per_pass) {
      const int r = rb + row_slot;
      C a[W];
#pragma unroll
      for (int q = 0; q < W; ++q) a[q] = 0;
      if (r < s) {
        const int e0 = (int)rp_s[r], e1 = (int)rp_s[r + 1];
        for (int e = e0 + gl; e < e1; e += kGroup) {
          const uint16_t v = ent_s[e];
          C src[W];
          TileRow<C, W>::load((const unsigned char*)tile, v & 0x7FFF, src);
          if (v & 0x8000) {
#pragma unroll
            for (int q = 0; q < W; ++q) a[q] -= src[q];
          } else {
#pragma unroll
            for (int q = 0; q < W; ++q) a[q] += src[q];
          }
        }
      }
#pragma unroll
      for (int q = 0; q < W; ++q) {
#pragma unroll
        for (int o = kGroup / 2; o > 0; o >>= 1) a[q] += __shfl_xor_sync(0xffffffffu, a[q], o);
      }
      if (r < s && gl == 0) {
#pragma unroll
        for (int q = 0; q < W; ++q) KahanAcc<C>::add(&acc_hi[r * W + q], &acc_lo[r * W + q], a[q]);
      }
    }
  }
  __syncthreads();
  // partial layout: [group][col][row]
  for (int q = threadIdx.x; q < s * W; q += blockDim.x) {
    const int r = q / W, cq = q % W;
    const int col = col0 + cq;
    if (col < ncols) partial[((int64_t)g * ncols + col) * s + r] = (double)acc_hi[q] - (double)acc_lo[q];
  }
}

// ----------------------------------------------------------------------------
// Row-owner gather (FP32 or FP64 data, s <= kRowsMaxS): thread r owns sketch
// row r for a tile of 64 bytes of columns (16 floats or 8 doubles) and keeps
// its sums in registers across all chunks of its group.  FP32 data: a plain
// FP32 sum per chunk, folded into a TwoSum-compensated pair once per chunk;
// FP64 data: plain FP64 sums.  Chunks are double-buffered with asynchronous
// copies: while chunk c is gathered, chunk c+1's data tile, entries and row
// offsets land in the other buffer.  A tile row's four 16-byte segments are
// rotated by (row >> 1), so the staging copies (8 consecutive rows x 4
// consecutive columns per warp instruction) spread evenly over the banks.
// ----------------------------------------------------------------------------
static constexpr int kRowsBytes = 64;  // bytes of one tile row
static constexpr int kRowsMaxS = 640;
template <typename T>
struct RowsW {
  static constexpr int value = kRowsBytes / (int)sizeof(T);
};

template <int E>
__device__ __forceinline__ void cp_async_e(void* dst, const void* src, bool valid) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
  const int n = valid ? E : 0;  // zero-fill when out of range
  if constexpr (E == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sa), "l"(src), "r"(n) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(sa), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

__host__ __device__ static inline size_t rows_buf_bytes(int s, int zeta) {
  return (size_t)kChunk * kRowsBytes + entries_bytes(zeta) + (size_t)rp_stride(s) * sizeof(uint32_t);
}

// Accumulate one 16-byte segment (k-th of the row) into acc.
__device__ __forceinline__ void seg_acc4(float (&acc)[16], int k, const float4& x, float sg) {
  acc[4 * k + 0] = fmaf(sg, x.x, acc[4 * k + 0]);
  acc[4 * k + 1] = fmaf(sg, x.y, acc[4 * k + 1]);
  acc[4 * k + 2] = fmaf(sg, x.z, acc[4 * k + 2]);
  acc[4 * k + 3] = fmaf(sg, x.w, acc[4 * k + 3]);
}
__device__ __forceinline__ void seg_acc4(double (&acc)[8], int k, const double2& x, float sg) {
  const double sd = (double)sg;
  acc[2 * k + 0] = fma(sd, x.x, acc[2 * k + 0]);
  acc[2 * k + 1] = fma(sd, x.y, acc[2 * k + 1]);
}
__device__ __forceinline__ void seg_acc(float (&acc)[16], int k, const unsigned char* p, float sg) {
  const float4 x = *reinterpret_cast<const float4*>(p);
  acc[4 * k + 0] = fmaf(sg, x.x, acc[4 * k + 0]);
  acc[4 * k + 1] = fmaf(sg, x.y, acc[4 * k + 1]);
  acc[4 * k + 2] = fmaf(sg, x.z, acc[4 * k + 2]);
  acc[4 * k + 3] = fmaf(sg, x.w, acc[4 * k + 3]);
}
__device__ __forceinline__ void seg_acc(double (&acc)[8], int k, const unsigned char* p, float sg) {
  const double2 x = *reinterpret_cast<const double2*>(p);
  const double sd = (double)sg;  // +-1: the product is exact, so this is an add or a subtract without divergence
  acc[2 * k + 0] = fma(sd, x.x, acc[2 * k + 0]);
  acc[2 * k + 1] = fma(sd, x.y, acc[2 * k + 1]);
}

// Body of the row-owner gather for column tile `tile` and chunk group `g`
// (blockIdx.x and blockIdx.y of a single launch).
template <typename T>
__device__ __forceinline__ void gather_rows_body(const T* __restrict__ B, int64_t ldb, int ncols, int64_t n, int s,
                                                 int zeta, int nchunks, int chunks_per_group,
                                                 const uint32_t* __restrict__ rowptr,
                                                 const uint16_t* __restrict__ entries, double* __restrict__ partial,
                                                 int tile, int g) {
  constexpr int E = (int)sizeof(T);
  constexpr int W = RowsW<T>::value;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const size_t buf_bytes = rows_buf_bytes(s, zeta);
  const int col0 = tile * W;
  const int c_begin = g * chunks_per_group;
  const int c_end = min(nchunks, c_begin + chunks_per_group);
  const int nt = blockDim.x;
  const int lane = threadIdx.x & 31;
  const int ent_copies = (int)(entries_bytes(zeta) / 16);
  const int rp_copies = (int)(rp_stride(s) / 4);

  auto stage = [&](int c, int b) {
    unsigned char* base = smem_raw + (size_t)b * buf_bytes;
    const int64_t i0 = (int64_t)c * kChunk;
    const int Lc = (int)((n - i0) < kChunk ? (n - i0) : kChunk);
    // data tile: warp instruction = 8 consecutive rows x 4 consecutive columns
    for (int q0 = threadIdx.x - lane; q0 < kChunk * W; q0 += nt) {
      const int gq = q0 >> 5;
      const int rb = gq % (kChunk / 8), cg = gq / (kChunk / 8);
      const int il = rb * 8 + (lane & 7);
      const int col = cg * 4 + (lane >> 3);
      const bool ok = il < Lc && col0 + col < ncols;
      const T* src = ok ? B + (i0 + il) + (int64_t)(col0 + col) * ldb : B;
      const int byte = col * E;  // byte of the column inside the unrotated row
      unsigned char* dst = smem_raw + (size_t)b * buf_bytes + (size_t)il * kRowsBytes +
                           (size_t)((((byte >> 4) + (il >> 1)) & 3) * 16 + (byte & 15));
      cp_async_e<E>(dst, src, ok);
    }
    const unsigned char* esrc = reinterpret_cast<const unsigned char*>(entries + (int64_t)c * kChunk * zeta);
    unsigned char* edst = base + (size_t)kChunk * kRowsBytes;
    for (int q = threadIdx.x; q < ent_copies; q += nt) cp_async16(edst + q * 16, esrc + q * 16);
    const unsigned char* rsrc = reinterpret_cast<const unsigned char*>(rowptr + (int64_t)c * rp_stride(s));
    unsigned char* rdst = edst + entries_bytes(zeta);
    for (int q = threadIdx.x; q < rp_copies; q += nt) cp_async16(rdst + q * 16, rsrc + q * 16);
  };

  T hi[W], lo[W];
#pragma unroll
  for (int q = 0; q < W; ++q) { hi[q] = 0; lo[q] = 0; }
  const int r = threadIdx.x;
  if (c_begin < c_end) stage(c_begin, 0);
  cp_async_commit();
  for (int c = c_begin; c < c_end; ++c) {
    const int b = (c - c_begin) & 1;
    if (c + 1 < c_end) stage(c + 1, b ^ 1);
    cp_async_commit();
    cp_async_wait1();
    __syncthreads();
    const unsigned char* base = smem_raw + (size_t)b * buf_bytes;
    const uint16_t* ent = reinterpret_cast<const uint16_t*>(base + (size_t)kChunk * kRowsBytes);
    const uint32_t* rp = reinterpret_cast<const uint32_t*>(base + (size_t)kChunk * kRowsBytes + entries_bytes(zeta));
    if (r < s) {
      T acc[W];
#pragma unroll
      for (int q = 0; q < W; ++q) acc[q] = 0;
      const int e0 = (int)rp[r], e1 = (int)rp[r + 1];
      // two entries per iteration (eight 16-byte loads in flight), the next
      // two entry words fetched one iteration ahead
      int e = e0;
      uint32_t va = (e < e1) ? ent[e] : 0u, vb = (e + 1 < e1) ? ent[e + 1] : 0u;
      for (; e + 1 < e1; e += 2) {
        const uint32_t na = (e + 2 < e1) ? ent[e + 2] : 0u, nb = (e + 3 < e1) ? ent[e + 3] : 0u;
        const int ia = va & 0x7FFF, ib = vb & 0x7FFF;
        const unsigned char* ra_ = base + (size_t)ia * kRowsBytes;
        const unsigned char* rb_ = base + (size_t)ib * kRowsBytes;
        using V16 = typename std::conditional<E == 4, float4, double2>::type;  // one 16-byte segment
        V16 xa[4], xb[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          xa[k] = *reinterpret_cast<const V16*>(ra_ + ((k + (ia >> 1)) & 3) * 16);
          xb[k] = *reinterpret_cast<const V16*>(rb_ + ((k + (ib >> 1)) & 3) * 16);
        }
        const float sa = (va & 0x8000) ? -1.f : 1.f, sb = (vb & 0x8000) ? -1.f : 1.f;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          seg_acc4(acc, k, xa[k], sa);
          seg_acc4(acc, k, xb[k], sb);
        }
        va = na;
        vb = nb;
      }
      if (e < e1) {
        const int il = va & 0x7FFF;
        const float sg = (va & 0x8000) ? -1.f : 1.f;
        const unsigned char* row = base + (size_t)il * kRowsBytes;
#pragma unroll
        for (int k = 0; k < 4; ++k) seg_acc(acc, k, row + ((k + (il >> 1)) & 3) * 16, sg);
      }
#pragma unroll
      for (int q = 0; q < W; ++q) {
        if constexpr (E == 4) {
          // TwoSum (Knuth) fold of the chunk sum into the compensated pair
          const float t = hi[q] + acc[q];
          const float bp = t - hi[q];
          lo[q] += (hi[q] - (t - bp)) + (acc[q] - bp);
          hi[q] = t;
        } else {
          hi[q] += acc[q];
        }
      }
    }
    __syncthreads();  // buffer b is restaged by the next iteration's prefetch
  }
  if (r < s) {
#pragma unroll
    for (int q = 0; q < W; ++q) {
      const int col = col0 + q;
      if (col < ncols) partial[((int64_t)g * ncols + col) * s + r] = (double)hi[q] + (double)lo[q];
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(kRowsMaxS)
gather_rows_kernel(const T* __restrict__ B, int64_t ldb, int ncols, int64_t n, int s, int zeta, int nchunks,
                   int chunks_per_group, const uint32_t* __restrict__ rowptr, const uint16_t* __restrict__ entries,
                   double* __restrict__ partial) {
  gather_rows_body<T>(B, ldb, ncols, n, s, zeta, nchunks, chunks_per_group, rowptr, entries, partial, blockIdx.x,
                      blockIdx.y);
}

// One column (the sketched residual g = S r): thread r owns sketch row r and
// sums in a register over all chunks of its group; the chunk of the vector
// is contiguous, so it is staged with 16-byte asynchronous copies (double
// buffered like the row-owner gather).  FP64 data: plain FP64 sums.
__host__ __device__ static inline size_t col_buf_bytes(int s, int zeta) {
  return (size_t)kChunk * sizeof(double) + entries_bytes(zeta) + (size_t)rp_stride(s) * sizeof(uint32_t);
}

__device__ __forceinline__ void gather_col_body(const double* __restrict__ x, int64_t n, int s, int zeta, int nchunks,
                                                int chunks_per_group, const uint32_t* __restrict__ rowptr,
                                                const uint16_t* __restrict__ entries, double* __restrict__ partial,
                                                int g) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const size_t buf_bytes = col_buf_bytes(s, zeta);
  const int c_begin = g * chunks_per_group;
  const int c_end = min(nchunks, c_begin + chunks_per_group);
  const int nt = blockDim.x;
  const int ent_copies = (int)(entries_bytes(zeta) / 16);
  const int rp_copies = (int)(rp_stride(s) / 4);
  auto stage = [&](int c, int b) {
    unsigned char* base = smem_raw + (size_t)b * buf_bytes;
    const int64_t i0 = (int64_t)c * kChunk;
    const int Lc = (int)((n - i0) < kChunk ? (n - i0) : kChunk);
    double* tile = reinterpret_cast<double*>(base);
    // 16-byte copies where both ends are aligned and in range; single elements otherwise
    const bool al = (((uintptr_t)(x + i0)) & 15) == 0;
    if (al) {
      for (int q = threadIdx.x; q < Lc / 2; q += nt) cp_async16(tile + 2 * q, x + i0 + 2 * q);
      if ((Lc & 1) && threadIdx.x == 0) cp_async_e<8>(tile + Lc - 1, x + i0 + Lc - 1, true);
    } else {
      for (int q = threadIdx.x; q < Lc; q += nt) cp_async_e<8>(tile + q, x + i0 + q, true);
    }
    const unsigned char* esrc = reinterpret_cast<const unsigned char*>(entries + (int64_t)c * kChunk * zeta);
    unsigned char* edst = base + (size_t)kChunk * sizeof(double);
    for (int q = threadIdx.x; q < ent_copies; q += nt) cp_async16(edst + q * 16, esrc + q * 16);
    const unsigned char* rsrc = reinterpret_cast<const unsigned char*>(rowptr + (int64_t)c * rp_stride(s));
    unsigned char* rdst = edst + entries_bytes(zeta);
    for (int q = threadIdx.x; q < rp_copies; q += nt) cp_async16(rdst + q * 16, rsrc + q * 16);
  };
  double acc = 0;
  const int r = threadIdx.x;
  if (c_begin < c_end) stage(c_begin, 0);
  cp_async_commit();
  for (int c = c_begin; c < c_end; ++c) {
    const int b = (c - c_begin) & 1;
    if (c + 1 < c_end) stage(c + 1, b ^ 1);
    cp_async_commit();
    cp_async_wait1();
    __syncthreads();
    const unsigned char* base = smem_raw + (size_t)b * buf_bytes;
    const double* tile = reinterpret_cast<const double*>(base);
    const uint16_t* ent = reinterpret_cast<const uint16_t*>(base + (size_t)kChunk * sizeof(double));
    const uint32_t* rp = reinterpret_cast<const uint32_t*>(base + (size_t)kChunk * sizeof(double) + entries_bytes(zeta));
    if (r < s) {
      const int e0 = (int)rp[r], e1 = (int)rp[r + 1];
      for (int e = e0; e < e1; ++e) {
        const uint16_t v = ent[e];
        const double sd = (v & 0x8000) ? -1.0 : 1.0;  // exact product: an add or a subtract
        acc = fma(sd, tile[v & 0x7FFF], acc);
      }
    }
    __syncthreads();
  }
  if (r < s) partial[(int64_t)g * s + r] = acc;
}

__global__ void __launch_bounds__(kRowsMaxS)
gather_col_kernel(const double* __restrict__ x, int64_t n, int s, int zeta, int nchunks, int chunks_per_group,
                  const uint32_t* __restrict__ rowptr, const uint16_t* __restrict__ entries,
                  double* __restrict__ partial) {
  gather_col_body(x, n, s, zeta, nchunks, chunks_per_group, rowptr, entries, partial, blockIdx.x);
}

// Each output entry sums its groups' partials in group order (the result
// does not depend on the grid).
__device__ __forceinline__ void reduce_partials_body(const double* __restrict__ partial, int ngroups, int ncols, int s,
                                                     double scale, double* __restrict__ SB) {
  const int64_t total = (int64_t)ncols * s;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    double a = 0;
    for (int g = 0; g < ngroups; ++g) a += partial[(int64_t)g * total + q];
    SB[q] = a * scale;
  }
}

__global__ void reduce_partials_kernel(const double* __restrict__ partial, int ngroups, int ncols, int s,
                                       double scale, double* __restrict__ SB) {
  reduce_partials_body(partial, ngroups, ncols, s, scale, SB);
}

// ---- grouped sketches (batched solver): map[blockIdx.x] = {slot, local block} --
template <typename T>
__global__ void __launch_bounds__(kRowsMaxS)
g_gather_rows_kernel(const GJob* __restrict__ jobs, const int2* __restrict__ map, int ncols, int s, int zeta) {
  const int2 m = map[blockIdx.x];
  const GJob& J = jobs[m.x];
  const int nt = J.rows_ntiles;
  gather_rows_body<T>(static_cast<const T*>(J.bp.B), J.bp.ldb, ncols, J.bp.n, s, zeta, J.nchunks, J.rows_cpg,
                      J.rowptr, J.entries, J.rows_part, m.y % nt, m.y / nt);
}

__global__ void __launch_bounds__(kRowsMaxS)
g_gather_col_kernel(const GJob* __restrict__ jobs, const int2* __restrict__ map, int s, int zeta) {
  const int2 m = map[blockIdx.x];
  const GJob& J = jobs[m.x];
  gather_col_body(J.bp.r, J.bp.n, s, zeta, J.nchunks, J.col_cpg, J.rowptr, J.entries, J.col_part, m.y);
}

// blockIdx.y = slot ids[blockIdx.y]: rows = 1 reduces the basis sketch into
// SB, rows = 0 the residual's into g.
__global__ void g_reduce_kernel(const GJob* __restrict__ jobs, const int* __restrict__ ids, int ncols, int s,
                                double scale, int rows) {
  const GJob& J = jobs[ids[blockIdx.y]];
  if (rows) reduce_partials_body(J.rows_part, J.rows_ngroups, ncols, s, scale, J.SB);
  else reduce_partials_body(J.col_part, J.col_ngroups, 1, s, scale, J.g);
}

template <typename T, int W>
static sk_status launch_gather(const SketchPlan& p, const T* B, int64_t ldb, int ncols, double* partial,
                               int ngroups, int cpg, cudaStream_t st) {
  using C = typename Compute<T>::type;
  const size_t smem = (size_t)kChunk * W * sizeof(C) + entries_bytes(p.zeta) + rowptr_bytes(p.s) +
                      (size_t)2 * p.s * W * sizeof(C);
  SK_CUDA(cudaFuncSetAttribute(gather_apply_kernel<T, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, kDynSmemLimit));
  dim3 grid((ncols + W - 1) / W, ngroups);
  gather_apply_kernel<T, W><<<grid, kApplyThreads, smem, st>>>(B, ldb, ncols, p.n, p.s, p.zeta, p.nchunks, cpg,
                                                                p.rowptr, p.entries, partial);
  SK_CUDA(cudaGetLastError());
  return SK_OK;
}

template <typename T>
static sk_status gather_dispatch(const SketchPlan& p, const T* B, int64_t ldb, int ncols, double* partial,
                                 int ngroups, int cpg, int W, cudaStream_t st) {
  switch (W) {
    case 1: return launch_gather<T, 1>(p, B, ldb, ncols, partial, ngroups, cpg, st);
    case 2: return launch_gather<T, 2>(p, B, ldb, ncols, partial, ngroups, cpg, st);
    case 4: return launch_gather<T, 4>(p, B, ldb, ncols, partial, ngroups, cpg, st);
    default: return launch_gather<T, 8>(p, B, ldb, ncols, partial, ngroups, cpg, st);
  }
}

// Column tile width: as wide as shared memory allows (tile, staged entries
// and row offsets, two accumulators).
static int pick_width(int s, int zeta, int ncols, size_t csize) {
  int W = 8;
  const size_t fixed = entries_bytes(zeta) + rowptr_bytes(s);
  while (W > 1 && ((size_t)kChunk * W * csize + fixed + (size_t)2 * s * W * csize > (size_t)kDynSmemLimit ||
                   W > ncols))
    W /= 2;
  if (csize == 8 && W > 4) W = 4;
  return W;
}

struct GatherShape {
  bool col;   // one FP64 column (gather_col_kernel)
  bool rows;  // row-owner kernel (FP32/FP64 data, s <= kRowsMaxS, at least one full tile of columns)
  int W, ntiles, ngroups, cpg;
};

// block = a sketch of basis columns inside a solver: the chunk grouping is
// fixed (kBlockGroups groups whatever the column count) and the kernel is
// chosen by element type alone, so every column is summed in the same order
// whether the basis is sketched whole or in blocks of columns.
static constexpr int kBlockGroups = 64;

static GatherShape gather_shape(const SketchPlan& p, int ncols, sk_dtype dtype, bool block) {
  GatherShape g;
  const size_t csize = dtype == SK_F64 ? 8 : 4;
  const int rows_w = kRowsBytes / (int)csize;
  g.col = !block && dtype == SK_F64 && ncols == 1 && p.s <= kRowsMaxS &&
          2 * col_buf_bytes(p.s, p.zeta) <= (size_t)kDynSmemLimit;
  g.rows = !g.col && (dtype == SK_F32 || dtype == SK_F64) && p.s <= kRowsMaxS && (ncols >= rows_w || block) &&
           2 * rows_buf_bytes(p.s, p.zeta) <= (size_t)kDynSmemLimit;
  g.W = g.col ? 1 : g.rows ? rows_w : pick_width(p.s, p.zeta, ncols, csize);
  g.ntiles = (ncols + g.W - 1) / g.W;
  if (block) {
    g.cpg = (p.nchunks + kBlockGroups - 1) / kBlockGroups;
    g.ngroups = (p.nchunks + g.cpg - 1) / g.cpg;
    return g;
  }
  const int target = num_sms();
  int ngroups = (target + g.ntiles - 1) / g.ntiles;
  if (ngroups > p.nchunks) ngroups = p.nchunks;
  if (ngroups < 1) ngroups = 1;
  g.cpg = (p.nchunks + ngroups - 1) / ngroups;
  g.ngroups = (p.nchunks + g.cpg - 1) / g.cpg;
  return g;
}

template <typename T>
static sk_status launch_rows(const SketchPlan& p, const T* B, int64_t ldb, int ncols, double* partial,
                             const GatherShape& g, cudaStream_t st) {
  const size_t smem = 2 * rows_buf_bytes(p.s, p.zeta);
  SK_CUDA(cudaFuncSetAttribute(gather_rows_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, kDynSmemLimit));
  const int threads = (p.s + 31) / 32 * 32;
  dim3 grid(g.ntiles, g.ngroups);
  gather_rows_kernel<T><<<grid, threads, smem, st>>>(B, ldb, ncols, p.n, p.s, p.zeta, p.nchunks, g.cpg, p.rowptr,
                                                     p.entries, partial);
  SK_CUDA(cudaGetLastError());
  return SK_OK;
}

size_t plan_ws_doubles(const SketchPlan& p, int ncols, sk_dtype dtype, bool block) {
  const GatherShape g = gather_shape(p, ncols, dtype, block);
  return (size_t)g.ngroups * ncols * p.s;
}

sk_status plan_apply_ws(const SketchPlan& p, const void* B, int64_t ldb, int ncols, sk_dtype dtype, double* SB,
                        double* partial, cudaStream_t st, bool block) {
  const GatherShape g = gather_shape(p, ncols, dtype, block);
  sk_status stt;
  if (g.col) {
    const size_t smem = 2 * col_buf_bytes(p.s, p.zeta);
    SK_CUDA(cudaFuncSetAttribute(gather_col_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kDynSmemLimit));
    gather_col_kernel<<<g.ngroups, (p.s + 31) / 32 * 32, smem, st>>>((const double*)B, p.n, p.s, p.zeta, p.nchunks,
                                                                     g.cpg, p.rowptr, p.entries, partial);
    SK_CUDA(cudaGetLastError());
    stt = SK_OK;
  } else if (dtype == SK_F64 && g.rows) stt = launch_rows(p, (const double*)B, ldb, ncols, partial, g, st);
  else if (dtype == SK_F64) stt = gather_dispatch<double>(p, (const double*)B, ldb, ncols, partial, g.ngroups, g.cpg, g.W, st);
  else if (dtype == SK_F32 && g.rows) stt = launch_rows(p, (const float*)B, ldb, ncols, partial, g, st);
  else if (dtype == SK_F32) stt = gather_dispatch<float>(p, (const float*)B, ldb, ncols, partial, g.ngroups, g.cpg, g.W, st);
  else stt = gather_dispatch<__nv_bfloat16>(p, (const __nv_bfloat16*)B, ldb, ncols, partial, g.ngroups, g.cpg, g.W, st);
  if (stt != SK_OK) return stt;
  const int64_t total = (int64_t)ncols * p.s;
  int rb = (int)((total + 255) / 256);
  if (rb > 4 * num_sms()) rb = 4 * num_sms();
  reduce_partials_kernel<<<rb, 256, 0, st>>>(partial, g.ngroups, ncols, p.s, 1.0 / std::sqrt((double)p.zeta), SB);
  SK_CUDA(cudaGetLastError());
  return SK_OK;
}

sk_status plan_apply(const SketchPlan& p, const void* B, int64_t ldb, int ncols, sk_dtype dtype, double* SB,
                     Scratch& scratch, cudaStream_t st) {
  double* partial = nullptr;
  SK_TRY(scratch.alloc(&partial, plan_ws_doubles(p, ncols, dtype)));
  return plan_apply_ws(p, B, ldb, ncols, dtype, SB, partial, st);
}

size_t sketch_plan_shape(const sk_sketch& S, SketchPlan* sp, SrhtPlan* hp) {
  auto r256 = [](size_t b) { return (b + 255) & ~(size_t)255; };
  if (S.kind == SK_SRHT) {
    hp->n = S.n;
    hp->s = S.s;
    hp->logn = 0;
    while ((1ll << hp->logn) < hp->n) ++hp->logn;
    hp->n_p = 1ll << hp->logn;
    hp->b = hp->logn < 12 ? hp->logn : 12;
    return r256((size_t)S.s * sizeof(int32_t)) + r256((size_t)((S.n + 31) / 32) * sizeof(uint32_t));
  }
  sp->n = S.n;
  sp->s = S.s;
  sp->zeta = S.zeta > 0 ? S.zeta : default_zeta_for(S.s / 2);
  sp->L = kChunk;
  sp->nchunks = (int)((S.n + kChunk - 1) / kChunk);
  return r256((size_t)sp->nchunks * rp_stride(sp->s) * sizeof(uint32_t)) +
         r256((size_t)sp->nchunks * kChunk * sp->zeta * sizeof(uint16_t)) + r256(sizeof(int));
}

sk_status check_plan_status(const SketchPlan& p, cudaStream_t st) {
  int h = 0;
  SK_CUDA(cudaMemcpyAsync(&h, p.d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
  SK_CUDA(cudaStreamSynchronize(st));
  if (h != 0) {
    set_error("sparse sign hash: no distinct row within 16 attempts (s=%d too small for zeta=%d)", p.s, p.zeta);
    return SK_EHASH;
  }
  return SK_OK;
}

}  // namespace sk

namespace sk {


sk_status sketch_apply_impl(const sk_sketch* S, const void* B, int64_t ldb, int ncols, sk_dtype dtype,
                            double* SB, cudaStream_t st) {
  Scratch scratch(st);
  if (S->kind == SK_SRHT) {
    SrhtPlan sp;
    SK_TRY(srht_plan_create(&sp, S, scratch, st));
    double* partial = nullptr;
    SK_TRY(scratch.alloc(&partial, srht_ws_doubles(sp, ncols)));
    return srht_apply_ws(sp, B, ldb, ncols, dtype, SB, partial, st);
  }
  SK_CHECK_ARG(S->kind == SK_SPARSE_SIGN, "unknown sketch kind");
  SketchPlan p;
  SK_TRY(plan_create(&p, S, scratch, st));
  SK_TRY(plan_apply(p, B, ldb, ncols, dtype, SB, scratch, st));
  return check_plan_status(p, st);
}

}  // namespace sk

// ----------------------------------------------------------------------------
// sketch_apply_noalloc: the sparse sign sketch without any device allocation.
//
// Some callers cannot call cudaMalloc on their hot path: plugins that run
// inside another framework's execution engine (the host framework owns the
// device memory budget, and cudaMalloc may synchronise the whole device),
// and latency-critical loops that must not pay an allocation's variable cost
// or meet an out-of-memory failure in the middle of a run.  For them this
// entry point keeps its scratch (the row-sorted index tables and the per-CTA
// partial sums) in one file-scope device array of fixed size, which every
// GPU that loads the library holds until the process exits.
// ----------------------------------------------------------------------------
namespace sk {

static constexpr size_t kNoAllocScratchBytes = (size_t)32 << 20;  // 32 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Device address of g_noalloc_scratch on the current device, looked up once
// per device (the host-side name is only a stand-in for the symbol).
static sk_status noalloc_scratch_ptr(unsigned char** out) {
  static std::mutex mu;
  static unsigned char* ptrs[64] = {nullptr};
  int dev = 0;
  SK_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) { set_error("sketch_apply_noalloc: device ordinal %d out of range", dev); return SK_EINVAL; }
  std::lock_guard<std::mutex> lock(mu);
  if (!ptrs[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    ptrs[dev] = (unsigned char*)p;
  }
  *out = ptrs[dev];
  return SK_OK;
}


void sketch_shapes(const SketchPlan& p, int ncols, sk_dtype dt, int* rows_ntiles, int* rows_ngroups, int* rows_cpg,
                   int* col_ngroups, int* col_cpg) {
  const GatherShape gr = gather_shape(p, ncols, dt, true);
  *rows_ntiles = gr.rows ? gr.ntiles : 0;  // 0: not the row-owner kernel (the grouped path needs it)
  *rows_ngroups = gr.ngroups;
  *rows_cpg = gr.cpg;
  const GatherShape gc = gather_shape(p, 1, SK_F64, false);
  *col_ngroups = gc.col ? gc.ngroups : 0;
  *col_cpg = gc.cpg;
}

sk_status enqueue_sketch_rows_grouped(const GJob* jobs, const int2* map, int nmap, const int* ids, int nj, sk_dtype dt,
                                      int ncols, int s, int zeta, cudaStream_t st) {
  if (nmap <= 0 || nj <= 0) return SK_OK;
  const size_t smem = 2 * rows_buf_bytes(s, zeta);
  const int threads = (s + 31) / 32 * 32;
  if (dt == SK_F64) {
    SK_CUDA(cudaFuncSetAttribute(g_gather_rows_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, kDynSmemLimit));
    g_gather_rows_kernel<double><<<nmap, threads, smem, st>>>(jobs, map, ncols, s, zeta);
  } else if (dt == SK_F32) {
    SK_CUDA(cudaFuncSetAttribute(g_gather_rows_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, kDynSmemLimit));
    g_gather_rows_kernel<float><<<nmap, threads, smem, st>>>(jobs, map, ncols, s, zeta);
  } else {
    set_error("grouped sketch: FP32 or FP64 basis expected");
    return SK_EINVAL;
  }
  SK_CUDA(cudaGetLastError());
  int rb = (int)(((int64_t)ncols * s + 255) / 256);
  if (rb > 4 * num_sms()) rb = 4 * num_sms();
  g_reduce_kernel<<<dim3(rb, nj), 256, 0, st>>>(jobs, ids, ncols, s, 1.0 / std::sqrt((double)zeta), 1);
  SK_CUDA(cudaGetLastError());
  return SK_OK;
}

sk_status enqueue_sketch_col_grouped(const GJob* jobs, const int2* map, int nmap, const int* ids, int nj, int s,
                                     int zeta, cudaStream_t st) {
  if (nmap <= 0 || nj <= 0) return SK_OK;
  const size_t smem = 2 * col_buf_bytes(s, zeta);
  SK_CUDA(cudaFuncSetAttribute(g_gather_col_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kDynSmemLimit));
  g_gather_col_kernel<<<nmap, (s + 31) / 32 * 32, smem, st>>>(jobs, map, s, zeta);
  SK_CUDA(cudaGetLastError());
  int rb = (s + 255) / 256;
  if (rb > 4 * num_sms()) rb = 4 * num_sms();
  g_reduce_kernel<<<dim3(rb, nj), 256, 0, st>>>(jobs, ids, 1, s, 1.0 / std::sqrt((double)zeta), 0);
  SK_CUDA(cudaGetLastError());
  return SK_OK;
}

}  // namespace sk

extern "C" sk_status sketch_apply_noalloc(const sk_sketch* S, const void* B, int64_t ldb, int ncols, sk_dtype dtype,
                                          double* SB, void* stream) {
  using namespace sk;
  SK_CHECK_ARG(S != nullptr && B != nullptr && SB != nullptr, "NULL argument");
  SK_CHECK_ARG(S->kind == SK_SPARSE_SIGN, "sketch_apply_noalloc supports the sparse sign sketch only");
  SK_CHECK_ARG(ncols >= 1, "ncols >= 1");
  SK_CHECK_ARG(S->n >= 1 && ldb >= S->n, "need n >= 1 and ldb >= n");
  SK_CHECK_ARG(S->s >= 1 && S->s <= kMaxSparseS, "sparse sign sketch needs 1 <= s <= 4096");
  SK_CHECK_ARG(dtype == SK_F64 || dtype == SK_F32 || dtype == SK_BF16, "dtype");
  const int zeta = S->zeta > 0 ? S->zeta : default_zeta_for(S->s / 2);
  SK_CHECK_ARG(zeta >= 1 && zeta <= 14 && zeta <= S->s, "zeta must be in 1..min(14, s)");
  cudaStream_t st = (cudaStream_t)stream;
  SketchPlan p;
  p.n = S->n;
  p.s = S->s;
  p.zeta = zeta;
  p.seed = S->seed;
  p.L = kChunk;
  p.nchunks = (int)((S->n + kChunk - 1) / kChunk);
  const size_t b_status = align256(sizeof(int));
  const size_t b_rowptr = align256((size_t)p.nchunks * rp_stride(p.s) * sizeof(uint32_t));
  const size_t b_entries = align256((size_t)p.nchunks * kChunk * zeta * sizeof(uint16_t));
  const size_t b_partial = align256(plan_ws_doubles(p, ncols, dtype) * sizeof(double));
  const size_t need = b_status + b_rowptr + b_entries + b_partial;
  if (need > kNoAllocScratchBytes) {
    set_error("sketch_apply_noalloc: this sketch needs %zu bytes of scratch, above the fixed %zu-byte limit "
              "(reduce n, zeta or ncols, or use sketch_apply)", need, kNoAllocScratchBytes);
    return SK_EINVAL;
  }
  unsigned char* base = nullptr;
  SK_TRY(noalloc_scratch_ptr(&base));
  p.d_status = (int*)base;
  p.rowptr = (uint32_t*)(base + b_status);
  p.entries = (uint16_t*)(base + b_status + b_rowptr);
  double* partial = (double*)(base + b_status + b_rowptr + b_entries);
  // the status word keeps the previous call's value: clear it; the tables and
  // partial sums are fully overwritten by this call's kernels
  SK_CUDA(cudaMemsetAsync(p.d_status, 0, sizeof(int), st));
  const size_t smem = plan_smem_bytes(p.s, zeta);
  SK_CUDA(cudaFuncSetAttribute(plan_build_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kDynSmemLimit));
  plan_build_kernel<<<p.nchunks, kPlanThreads, smem, st>>>(p.n, p.s, zeta, seed_key(p.seed), p.rowptr, p.entries,
                                                            p.d_status);
  SK_CUDA(cudaGetLastError());
  SK_TRY(plan_apply_ws(p, B, ldb, ncols, dtype, SB, partial, st));
  return check_plan_status(p, st);
}
