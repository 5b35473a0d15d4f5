// Subsampled randomized Hadamard transform (§2.3.1, eq. (SRFT), with the
// Walsh-Hadamard transform standing in for the DFT and Rademacher E, §8.1.1).
//
// S v = (1/sqrt(s)) (H_raw E v)[rows],  H_raw[r,i] = (-1)^popcount(r & i).
// Only s outputs are needed, so the transform is split as in a subsampled
// FFT: with i = (i_hi, i_lo), H_raw = H_hi (x) H_lo and
//   y_r = sum_{i_hi} (-1)^popc(r_hi & i_hi) * FWHT_lo(E v restricted to block i_hi)[r_lo].
// One pass over the data: each CTA transforms whole blocks of 2^b entries in
// shared memory and keeps, per sketch row, the signed sum over its blocks;
// the per-CTA partials are combined in FP64 afterwards.
#include <cmath>
#include <unordered_map>
#include <vector>

#include "common.cuh"

namespace sk {

static constexpr int kSrhtThreads = 256;


__global__ void srht_signs_kernel(int64_t n, uint64_t skey, uint32_t* __restrict__ bits) {
  const int64_t nw = (n + 31) / 32;
  for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < nw; w += (int64_t)gridDim.x * blockDim.x) {
    uint32_t m = 0;
    for (int q = 0; q < 32; ++q) {
      const int64_t i = w * 32 + q;
      if (i < n && h1_neg(h1(skey, (uint64_t)i, 15u, 0u))) m |= (1u << q);
    }
    bits[w] = m;
  }
}

// Partial Fisher-Yates over 0..n_p-1: s distinct rows (definition in sk.h).
static void srht_rows_host(uint64_t seed, int64_t n_p, int s, std::vector<int32_t>& out) {
  std::unordered_map<int64_t, int64_t> perm;
  out.resize(s);
  const uint64_t key = seed_key(seed);
  for (int q = 0; q < s; ++q) {
    const uint64_t x = h1(key, (uint64_t)q, 14u, 0u);
    const int64_t j = q + (int64_t)(((x & 0xFFFFFFFFull) * (uint64_t)(n_p - q)) >> 32);
    auto iq = perm.find(q);
    auto ij = perm.find(j);
    const int64_t vq = iq == perm.end() ? q : iq->second;
    const int64_t vj = ij == perm.end() ? j : ij->second;
    perm[q] = vj;
    perm[j] = vq;
    out[q] = (int32_t)vj;
  }
}

// grid: (ncols, groups).  Each CTA handles one column and a contiguous range
// of blocks; smem: block of 2^b values + s accumulators.
template <typename T>
__global__ void __launch_bounds__(kSrhtThreads)
srht_kernel(const T* __restrict__ B, int64_t ldb, int64_t n, int b, int nblocks, int blocks_per_group, int s,
            const uint32_t* __restrict__ sign_bits, const int32_t* __restrict__ rows, double* __restrict__ partial) {
  using C = typename Compute<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int L = 1 << b;
  C* blk = (C*)smem_raw;  // L
  C* acc = blk + L;       // s
  const int col = blockIdx.x;
  const int g = blockIdx.y;
  const int ncols = gridDim.x;
  const T* x = B + (int64_t)col * ldb;
  for (int q = threadIdx.x; q < s; q += blockDim.x) acc[q] = 0;
  const int hb0 = g * blocks_per_group;
  const int hb1 = min(nblocks, hb0 + blocks_per_group);
  for (int hb = hb0; hb < hb1; ++hb) {
    const int64_t base = (int64_t)hb * L;
    __syncthreads();
    for (int il = threadIdx.x; il < L; il += blockDim.x) {
      const int64_t i = base + il;
      C v = 0;
      if (i < n) {
        v = to_c(x[i]);
        if ((sign_bits[i >> 5] >> (i & 31)) & 1u) v = -v;
      }
      blk[il] = v;
    }
    __syncthreads();
    // in-place radix-2 Walsh-Hadamard butterflies over the block
    for (int h = 1; h < L; h <<= 1) {
      for (int p = threadIdx.x; p < L / 2; p += blockDim.x) {
        const int lo = p & (h - 1);
        const int i0 = ((p - lo) << 1) + lo;
        const C a = blk[i0], c = blk[i0 + h];
        blk[i0] = a + c;
        blk[i0 + h] = a - c;
      }
      __syncthreads();
    }
    for (int q = threadIdx.x; q < s; q += blockDim.x) {
      const int r = rows[q];
      const int rlo = r & (L - 1);
      const int rhi = r >> b;
      const C v = blk[rlo];
      acc[q] += (__popc(rhi & hb) & 1) ? -v : v;
    }
  }
  __syncthreads();
  for (int q = threadIdx.x; q < s; q += blockDim.x) partial[((int64_t)g * ncols + col) * s + q] = (double)acc[q];
}

__global__ void srht_reduce_kernel(const double* __restrict__ partial, int ngroups, int ncols, int s, double scale,
                                   double* __restrict__ SB) {
  const int64_t total = (int64_t)ncols * s;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    double a = 0;
    for (int g = 0; g < ngroups; ++g) a += partial[(int64_t)g * total + q];
    SB[q] = a * scale;
  }
}

template <typename T>
static sk_status srht_launch(const SrhtPlan& p, const T* B, int64_t ldb, int ncols, double* partial, int ngroups,
                             int bpg, int nblocks, cudaStream_t st) {
  using C = typename Compute<T>::type;
  const size_t smem = ((size_t)(1 << p.b) + p.s) * sizeof(C);
  SK_CUDA(cudaFuncSetAttribute(srht_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, kDynSmemLimit));
  dim3 grid(ncols, ngroups);
  srht_kernel<T><<<grid, kSrhtThreads, smem, st>>>(B, ldb, p.n, p.b, nblocks, bpg, p.s, p.sign_bits, p.rows,
                                                   partial);
  SK_CUDA(cudaGetLastError());
  return SK_OK;
}

// block = a sketch of basis columns inside a solver: a fixed number of
// groups per column, so each column's sum has the same order whatever the
// column count.
static constexpr int kSrhtBlockGroups = 16;

static void srht_shape(const SrhtPlan& p, int ncols, bool block, int* ngroups_out, int* bpg_out,
                       int* data_blocks_out) {
  const int data_blocks = (int)((p.n + (1ll << p.b) - 1) >> p.b);
  const int target = 2 * num_sms();
  int ngroups = block ? kSrhtBlockGroups : (target + ncols - 1) / ncols;
  if (ngroups > data_blocks) ngroups = data_blocks;
  if (ngroups < 1) ngroups = 1;
  const int bpg = (data_blocks + ngroups - 1) / ngroups;
  *ngroups_out = (data_blocks + bpg - 1) / bpg;
  *bpg_out = bpg;
  *data_blocks_out = data_blocks;
}

sk_status srht_plan_create(SrhtPlan* p, const sk_sketch* S, Scratch& scratch, cudaStream_t st) {
  SK_CHECK_ARG(S != nullptr && S->n >= 1, "sketch n >= 1");
  p->n = S->n;
  p->s = S->s;
  p->logn = 0;
  while ((1ll << p->logn) < p->n) ++p->logn;
  p->n_p = 1ll << p->logn;
  SK_CHECK_ARG(p->logn <= 30, "SRHT needs n <= 2^30");
  SK_CHECK_ARG(p->s >= 1 && p->s <= p->n_p, "SRHT needs 1 <= s <= n_p");
  SK_CHECK_ARG(p->s <= 16384, "SRHT needs s <= 16384");
  p->b = p->logn < 12 ? p->logn : 12;
  std::vector<int32_t> rows;
  srht_rows_host(S->seed, p->n_p, p->s, rows);
  SK_TRY(scratch.alloc(&p->rows, (size_t)p->s));
  SK_CUDA(cudaMemcpyAsync(p->rows, rows.data(), sizeof(int32_t) * p->s, cudaMemcpyHostToDevice, st));
  SK_CUDA(cudaStreamSynchronize(st));  // rows lives on the host stack
  const int64_t nwords = (p->n + 31) / 32;
  SK_TRY(scratch.alloc(&p->sign_bits, (size_t)nwords));
  int sb = (int)((nwords + 255) / 256);
  if (sb > 8 * num_sms()) sb = 8 * num_sms();
  srht_signs_kernel<<<sb, 256, 0, st>>>(p->n, seed_key(S->seed), p->sign_bits);
  SK_CUDA(cudaGetLastError());
  return SK_OK;
}

size_t srht_ws_doubles(const SrhtPlan& p, int ncols, bool block) {
  int ngroups, bpg, db;
  srht_shape(p, ncols, block, &ngroups, &bpg, &db);
  return (size_t)ngroups * ncols * p.s;
}

sk_status srht_apply_ws(const SrhtPlan& p, const void* B, int64_t ldb, int ncols, sk_dtype dtype, double* SB,
                        double* partial, cudaStream_t st, bool block) {
  int ngroups, bpg, data_blocks;
  srht_shape(p, ncols, block, &ngroups, &bpg, &data_blocks);
  sk_status stt;
  if (dtype == SK_F64) stt = srht_launch<double>(p, (const double*)B, ldb, ncols, partial, ngroups, bpg, data_blocks, st);
  else if (dtype == SK_F32) stt = srht_launch<float>(p, (const float*)B, ldb, ncols, partial, ngroups, bpg, data_blocks, st);
  else stt = srht_launch<__nv_bfloat16>(p, (const __nv_bfloat16*)B, ldb, ncols, partial, ngroups, bpg, data_blocks, st);
  if (stt != SK_OK) return stt;
  const int64_t total = (int64_t)ncols * p.s;
  int rb = (int)((total + 255) / 256);
  if (rb > 4 * num_sms()) rb = 4 * num_sms();
  srht_reduce_kernel<<<rb, 256, 0, st>>>(partial, ngroups, ncols, p.s, 1.0 / std::sqrt((double)p.s), SB);
  SK_CUDA(cudaGetLastError());
  return SK_OK;
}

}  // namespace sk
