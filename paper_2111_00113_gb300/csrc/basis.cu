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
// m = A b_j is recomputed from the stored b_j in each pass instead of being
// stored: a 5-point product costs less than writing and re-reading a vector.
// The Arnoldi coefficients are kept: A b_j = sum_q (h1+h2)_q b_{j-q} +
// nu_j b_{j+1}, i.e. AB_d = B_{d+1} Hbar with Hbar (d+1) x d, k+1 diagonals.
#include <cmath>

#include "common.cuh"
#include "basis.cuh"

namespace sk {

template <typename T>
__device__ __forceinline__ T* bcol(void* B, int64_t ldb, int c) {
  return (T*)B + (int64_t)c * ldb;
}

template <typename T, int KM>
__global__ void __launch_bounds__(kBasisThreads)
form_kernel(BasisParams p, OpView<typename Compute<T>::type> A, int c) {
  using C = typename Compute<T>::type;
  if (c >= *p.stop) return;
  T* out = bcol<T>(p.B, p.ldb, c);
  const int64_t n = p.n;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t i_begin = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c == 0) {
    const double inv = 1.0 / sqrt(*p.rho2);
    for (int64_t i = i_begin; i < n; i += stride) out[i] = from_c<T>((C)(p.r[i] * inv));
    return;
  }
  const int j = c - 1;
  const int kw = min(p.k, j + 1);
  C h[KM];
#pragma unroll
  for (int q = 0; q < KM; ++q) h[q] = (q < kw) ? (C)(p.h1[j * p.k + q] + p.h2[j * p.k + q]) : (C)0;
  const C inv = (C)(1.0 / p.nu[j]);
  const T* bj = bcol<T>(p.B, p.ldb, j);
  for (int64_t i = i_begin; i < n; i += stride) {
    C m = A.apply(bj, i);
#pragma unroll
    for (int q = 0; q < KM; ++q)
      if (q < kw) m -= h[q] * to_c(bcol<T>(p.B, p.ldb, j - q)[i]);
    out[i] = from_c<T>(m * inv);
  }
}

// pass = 1: dots with m;  pass = 2: dots with w = m - W h1.
template <typename T, int KM, int PASS>
__global__ void __launch_bounds__(kBasisThreads)
dots_kernel(BasisParams p, OpView<typename Compute<T>::type> A, int j) {
  using C = typename Compute<T>::type;
  __shared__ C red[(KM + 1) * (kBasisThreads / 32)];
  if (j >= *p.stop) return;
  const int kw = min(p.k, j + 1);
  const int64_t n = p.n;
  const T* bj = bcol<T>(p.B, p.ldb, j);
  C h[KM];
  if (PASS == 2) {
#pragma unroll
    for (int q = 0; q < KM; ++q) h[q] = (q < kw) ? (C)p.h1[j * p.k + q] : (C)0;
  }
  C acc[KM + 1];
#pragma unroll
  for (int q = 0; q <= KM; ++q) acc[q] = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) {
    C m = A.apply(bj, i);
    C bw[KM];
#pragma unroll
    for (int q = 0; q < KM; ++q) bw[q] = (q < kw) ? to_c(bcol<T>(p.B, p.ldb, j - q)[i]) : (C)0;
    if (PASS == 2) {
#pragma unroll
      for (int q = 0; q < KM; ++q) m -= h[q] * bw[q];
    }
#pragma unroll
    for (int q = 0; q < KM; ++q) acc[q] += bw[q] * m;
    acc[KM] += m * m;
  }
  block_sum_k<KM + 1>(acc, red);
  double* part = p.partial;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q <= KM; ++q) part[blockIdx.x * (KM + 1) + q] = (double)acc[q];
  }
  if (!last_block_arrived(p.counters + (PASS - 1))) return;
  if (threadIdx.x != 0) return;
  double tot[KM + 1];
  for (int q = 0; q <= KM; ++q) tot[q] = 0;
  for (int b = 0; b < (int)gridDim.x; ++b)
    for (int q = 0; q <= KM; ++q) tot[q] += __ldcg(part + b * (KM + 1) + q);
  if (PASS == 1) {
    for (int q = 0; q < kw; ++q) p.h1[j * p.k + q] = tot[q];
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
  // finalise step j: nu_j and the Hessenberg column
  double h2sq = 0;
  for (int q = 0; q < kw; ++q) h2sq += tot[q] * tot[q];
  const double nu2 = tot[KM] - h2sq;
  const double mn2 = p.mn2[j];
  bool brk = !(nu2 > p.bd * p.bd * mn2) || !(mn2 > 0);
  if (!isfinite(nu2)) { *p.nanflag = 1; brk = true; }
  const double nu = brk ? 0.0 : sqrt(nu2);
  p.nu[j] = nu;
  if (p.Hbar) {
    double* col = p.Hbar + (int64_t)j * (p.d + 1);
    for (int q = 0; q < kw; ++q) col[j - q] = p.h1[j * p.k + q] + p.h2[j * p.k + q];
    col[j + 1] = nu;
  }
  if (brk) *p.stop = j + 1;
}

template <typename T, int KM>
static sk_status enqueue_basis_t(const BasisParams& p, const OpView<typename Compute<T>::type>& A,
                                 cudaStream_t st) {
  const int g = p.nblk;
  form_kernel<T, KM><<<g, kBasisThreads, 0, st>>>(p, A, 0);
  for (int j = 0; j < p.d; ++j) {
    dots_kernel<T, KM, 1><<<g, kBasisThreads, 0, st>>>(p, A, j);
    if (p.passes == 2) dots_kernel<T, KM, 2><<<g, kBasisThreads, 0, st>>>(p, A, j);
    form_kernel<T, KM><<<g, kBasisThreads, 0, st>>>(p, A, j + 1);
  }
  SK_CUDA(cudaGetLastError());
  return SK_OK;
}

template <typename T, typename C>
static sk_status enqueue_basis_k(const BasisParams& p, const OpView<C>& A, cudaStream_t st) {
  if (p.k <= 2) return enqueue_basis_t<T, 2>(p, A, st);
  if (p.k <= 4) return enqueue_basis_t<T, 4>(p, A, st);
  if (p.k <= 8) return enqueue_basis_t<T, 8>(p, A, st);
  return enqueue_basis_t<T, 16>(p, A, st);
}

int basis_grid(int64_t n) {
  int64_t g = (n + kBasisThreads * 4 - 1) / (kBasisThreads * 4);
  const int64_t gmax = 2 * num_sms();
  if (g > gmax) g = gmax;
  if (g < 1) g = 1;
  return (int)g;
}

sk_status enqueue_basis(const BasisParams& p, const sk_op* op, cudaStream_t st) {
  if (p.k > kMaxK) { set_error("k <= %d supported", kMaxK); return SK_EINVAL; }
  if (p.dtype == SK_F64) {
    OpView<double> A;
    make_view(op, &A);
    return enqueue_basis_k<double>(p, A, st);
  }
  OpView<float> A;
  SK_TRY(make_view(op, &A, st));
  if (p.dtype == SK_F32) return enqueue_basis_k<float>(p, A, st);
  return enqueue_basis_k<__nv_bfloat16>(p, A, st);
}

}  // namespace sk
