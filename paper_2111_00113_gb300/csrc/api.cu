// C ABI plumbing: errors, options, operator objects, operator apply and the
// sketch_apply entry point.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "common.cuh"

namespace sk {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

sk_status cuda_fail(cudaError_t e, const char* what) {
  set_error("CUDA error in %s: %s", what, cudaGetErrorString(e));
  return SK_ECUDA;
}

// ----------------------------------------------------------------------------
// Operator views.
// ----------------------------------------------------------------------------
sk_status make_view(const sk_op* op, OpView<double>* v) {
  v->kind = op->kind;
  v->nx = op->nx;
  v->ny = op->ny;
  v->n = op->n;
  v->cP = op->coef[0]; v->cE = op->coef[1]; v->cW = op->coef[2]; v->cN = op->coef[3]; v->cS = op->coef[4];
  v->shift = op->shift;
  v->theta = op->theta;
  v->rowptr = op->rowptr;
  v->colind = op->colind;
  v->val = op->val;
  v->sell_ptr = op->sell_ptr;
  v->sell_col = op->sell_col;
  v->sell_val = op->sell_val;
  set_div_magic(op->nx, op->n, &v->nx_m, &v->nx_s);
  return SK_OK;
}

__global__ void f64_to_f32_kernel(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

static sk_status f32_copy(const double* src, int64_t n, float** dst, cudaStream_t st) {
  if (*dst) return SK_OK;
  SK_CUDA(cudaMalloc((void**)dst, (size_t)n * sizeof(float)));
  int blocks = (int)((n + 255) / 256);
  if (blocks > 8 * num_sms()) blocks = 8 * num_sms();
  f64_to_f32_kernel<<<blocks, 256, 0, st>>>(src, *dst, n);
  SK_CUDA(cudaGetLastError());
  return SK_OK;
}

sk_status make_view(const sk_op* cop, OpView<float>* v, cudaStream_t st) {
  sk_op* op = const_cast<sk_op*>(cop);  // FP32 copies are a cache owned by the op
  v->kind = op->kind;
  v->nx = op->nx;
  v->ny = op->ny;
  v->n = op->n;
  v->cP = (float)op->coef[0]; v->cE = (float)op->coef[1]; v->cW = (float)op->coef[2];
  v->cN = (float)op->coef[3]; v->cS = (float)op->coef[4];
  v->shift = nullptr; v->theta = nullptr; v->val = nullptr;
  v->rowptr = op->rowptr;
  v->colind = op->colind;
  if (op->shift) { SK_TRY(f32_copy(op->shift, op->n, &op->shift32, st)); v->shift = op->shift32; }
  if (op->theta) { SK_TRY(f32_copy(op->theta, op->n, &op->theta32, st)); v->theta = op->theta32; }
  if (op->val) { SK_TRY(f32_copy(op->val, op->nnz, &op->val32, st)); v->val = op->val32; }
  v->sell_ptr = op->sell_ptr;
  v->sell_col = op->sell_col;
  v->sell_val = nullptr;
  if (op->sell_ptr && !op->sell_val32) {  // first FP32 use (solvers make it before any capture)
    int64_t total = 0;
    SK_CUDA(cudaMemcpyAsync(&total, op->sell_ptr + (op->n + 31) / 32, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    SK_CUDA(cudaStreamSynchronize(st));
    SK_TRY(f32_copy(op->sell_val, total, &op->sell_val32, st));
  }
  v->sell_val = op->sell_val32;
  set_div_magic(op->nx, op->n, &v->nx_m, &v->nx_s);
  return SK_OK;
}

__global__ void op_apply_kernel(OpView<double> A, const double* __restrict__ x, double* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < A.n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = A.apply(x, i);
}

// d(lam^T A x)/dtheta for the variable-coefficient diffusion operator.
__global__ void diffusion_grad_kernel(int nx, int ny, const double* __restrict__ lam, const double* __restrict__ x,
                                      double alpha, double* __restrict__ g) {
  const int64_t n = (int64_t)nx * ny;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int ix = (int)(i % nx);
    const int64_t iy = i / nx;
    const double lP = lam[i], xP = x[i];
    double a = 0;
    a += (ix + 1 < nx) ? 0.5 * (lP - lam[i + 1]) * (xP - x[i + 1]) : lP * xP;
    a += (ix > 0) ? 0.5 * (lP - lam[i - 1]) * (xP - x[i - 1]) : lP * xP;
    a += (iy + 1 < ny) ? 0.5 * (lP - lam[i + nx]) * (xP - x[i + nx]) : lP * xP;
    a += (iy > 0) ? 0.5 * (lP - lam[i - nx]) * (xP - x[i - nx]) : lP * xP;
    g[i] = alpha * a;
  }
}

// d(lam^T A x)/dc for the five stencil coefficients (per-CTA partials, then
// one fixed-order sum) and d/dshift_P = lam_P x_P.
__global__ void stencil_grad_kernel(int nx, int ny, const double* __restrict__ lam, const double* __restrict__ x,
                                    double alpha, double* __restrict__ part, double* __restrict__ gshift) {
  __shared__ double red[5 * 8];
  const int64_t n = (int64_t)nx * ny;
  double a[5] = {0, 0, 0, 0, 0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int ix = (int)(i % nx);
    const int64_t iy = i / nx;
    const double l = lam[i];
    a[0] += l * x[i];
    if (ix + 1 < nx) a[1] += l * x[i + 1];
    if (ix > 0) a[2] += l * x[i - 1];
    if (iy + 1 < ny) a[3] += l * x[i + nx];
    if (iy > 0) a[4] += l * x[i - nx];
    if (gshift) gshift[i] = alpha * (l * x[i]);
  }
  block_sum_k<5>(a, red);
  if (threadIdx.x == 0)
    for (int q = 0; q < 5; ++q) part[blockIdx.x * 5 + q] = a[q];
}

__global__ void sum_parts_kernel(const double* __restrict__ part, int nblk, int K, double alpha,
                                 double* __restrict__ out) {
  for (int q = threadIdx.x; q < K; q += blockDim.x) {
    double a = 0;
    for (int b = 0; b < nblk; ++b) a += part[b * K + q];
    out[q] = alpha * a;
  }
}

__global__ void csr_grad_kernel(int64_t n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                const double* __restrict__ lam, const double* __restrict__ x, double alpha,
                                double* __restrict__ g) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double l = alpha * lam[i];
    for (int32_t e = rowptr[i]; e < rowptr[i + 1]; ++e) g[e] = l * x[col[e]];
  }
}

// ---- CSR: SELL-32 copy and transpose ---------------------------------------------------
__global__ void sell_width_kernel(const int32_t* __restrict__ rowptr, int64_t n, int64_t* __restrict__ w) {
  const int64_t ns = (n + 31) / 32;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < ns; q += (int64_t)gridDim.x * blockDim.x) {
    int32_t m = 0;
    for (int64_t i = 32 * q; i < 32 * q + 32 && i < n; ++i) m = max(m, rowptr[i + 1] - rowptr[i]);
    w[q] = (int64_t)m * 32;
  }
}

__global__ void sell_fill_kernel(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                 const double* __restrict__ val, int64_t n, const int64_t* __restrict__ sptr,
                                 int32_t* __restrict__ scol, double* __restrict__ sval) {
  const int64_t ns = (n + 31) / 32;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < ns * 32; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = t >> 5, i = t;
    const int w = (int)((sptr[q + 1] - sptr[q]) >> 5);
    const int32_t e0 = i < n ? rowptr[i] : 0, len = i < n ? rowptr[i + 1] - e0 : 0;
    for (int e = 0; e < w; ++e) {
      const int64_t idx = sptr[q] + 32 * (int64_t)e + (i & 31);
      scol[idx] = e < len ? col[e0 + e] : (int32_t)(i < n ? i : 0);
      sval[idx] = e < len ? val[e0 + e] : 0.0;
    }
  }
}

// the SELL-32 copy of op's CSR arrays (synchronous, legacy default stream)
static sk_status build_sell(sk_op* op) {
  const int64_t n = op->n, ns = (n + 31) / 32;
  int64_t* w = nullptr;
  SK_CUDA(cudaMalloc((void**)&op->sell_ptr, sizeof(int64_t) * (ns + 1)));
  SK_CUDA(cudaMalloc((void**)&w, sizeof(int64_t) * ns));
  const int g = (int)std::min<int64_t>((ns + 255) / 256, 8 * num_sms());
  sell_width_kernel<<<g > 0 ? g : 1, 256>>>(op->rowptr, n, w);
  SK_CUDA(cudaGetLastError());
  int64_t* hw = new (std::nothrow) int64_t[ns + 1];
  if (!hw) { cudaFree(w); set_error("out of host memory"); return SK_ENOMEM; }
  cudaError_t e = cudaMemcpy(hw, w, sizeof(int64_t) * ns, cudaMemcpyDeviceToHost);
  cudaFree(w);
  if (e != cudaSuccess) { delete[] hw; return cuda_fail(e, "cudaMemcpy(SELL widths)"); }
  int64_t run = 0;
  for (int64_t q = 0; q < ns; ++q) { const int64_t v = hw[q]; hw[q] = run; run += v; }
  hw[ns] = run;
  e = cudaMemcpy(op->sell_ptr, hw, sizeof(int64_t) * (ns + 1), cudaMemcpyHostToDevice);
  delete[] hw;
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(SELL offsets)");
  SK_CUDA(cudaMalloc((void**)&op->sell_col, sizeof(int32_t) * (run > 0 ? run : 1)));
  SK_CUDA(cudaMalloc((void**)&op->sell_val, sizeof(double) * (run > 0 ? run : 1)));
  const int g2 = (int)std::min<int64_t>((ns * 32 + 255) / 256, 16 * num_sms());
  sell_fill_kernel<<<g2 > 0 ? g2 : 1, 256>>>(op->rowptr, op->colind, op->val, n, op->sell_ptr, op->sell_col,
                                            op->sell_val);
  SK_CUDA(cudaGetLastError());
  SK_CUDA(cudaDeviceSynchronize());
  return SK_OK;
}

__global__ void csr_count_kernel(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col, int64_t n,
                                 int32_t* __restrict__ cnt) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    for (int32_t e = rowptr[i]; e < rowptr[i + 1]; ++e) atomicAdd(&cnt[col[e]], 1);
}

// entry (i, j, v) of A lands in row j of A^T at a slot claimed atomically;
// the rows are sorted afterwards, so the result does not depend on the order
__global__ void csr_scatter_kernel(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                   const double* __restrict__ val, int64_t n, const int32_t* __restrict__ tptr,
                                   int32_t* __restrict__ fill, int32_t* __restrict__ tcol, double* __restrict__ tval) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    for (int32_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
      const int32_t j = col[e];
      const int32_t pos = tptr[j] + atomicAdd(&fill[j], 1);
      tcol[pos] = (int32_t)i;
      tval[pos] = val[e];
    }
}

// each row of A^T sorted by column (insertion sort; rows are short)
__global__ void csr_sort_rows_kernel(const int32_t* __restrict__ tptr, int64_t n, int32_t* __restrict__ tcol,
                                     double* __restrict__ tval) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    const int32_t b = tptr[j], e = tptr[j + 1];
    for (int32_t q = b + 1; q < e; ++q) {
      const int32_t c = tcol[q];
      const double v = tval[q];
      int32_t p = q - 1;
      while (p >= b && tcol[p] > c) { tcol[p + 1] = tcol[p]; tval[p + 1] = tval[p]; --p; }
      tcol[p + 1] = c;
      tval[p + 1] = v;
    }
  }
}

// A^T of a CSR op into t's own arrays (synchronous)
static sk_status build_csr_transpose(const sk_op* op, sk_op* t) {
  const int64_t n = op->n, nnz = op->nnz;
  int32_t *cnt = nullptr, *fill = nullptr;
  SK_CUDA(cudaMalloc((void**)&t->own_rowptr, sizeof(int32_t) * (n + 1)));
  SK_CUDA(cudaMalloc((void**)&t->own_colind, sizeof(int32_t) * (nnz > 0 ? nnz : 1)));
  SK_CUDA(cudaMalloc((void**)&t->own_val, sizeof(double) * (nnz > 0 ? nnz : 1)));
  SK_CUDA(cudaMalloc((void**)&cnt, sizeof(int32_t) * n));
  SK_CUDA(cudaMalloc((void**)&fill, sizeof(int32_t) * n));
  SK_CUDA(cudaMemset(cnt, 0, sizeof(int32_t) * n));
  SK_CUDA(cudaMemset(fill, 0, sizeof(int32_t) * n));
  const int g = (int)std::min<int64_t>((n + 255) / 256, 16 * num_sms());
  csr_count_kernel<<<g > 0 ? g : 1, 256>>>(op->rowptr, op->colind, n, cnt);
  SK_CUDA(cudaGetLastError());
  int32_t* h = new (std::nothrow) int32_t[n + 1];
  if (!h) { cudaFree(cnt); cudaFree(fill); set_error("out of host memory"); return SK_ENOMEM; }
  cudaError_t e = cudaMemcpy(h + 1, cnt, sizeof(int32_t) * n, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) {
    h[0] = 0;
    for (int64_t j = 0; j < n; ++j) h[j + 1] += h[j];
    e = cudaMemcpy(t->own_rowptr, h, sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice);
  }
  delete[] h;
  cudaFree(cnt);
  if (e != cudaSuccess) { cudaFree(fill); return cuda_fail(e, "cudaMemcpy(transpose counts)"); }
  csr_scatter_kernel<<<g > 0 ? g : 1, 256>>>(op->rowptr, op->colind, op->val, n, t->own_rowptr, fill, t->own_colind,
                                             t->own_val);
  csr_sort_rows_kernel<<<g > 0 ? g : 1, 256>>>(t->own_rowptr, n, t->own_colind, t->own_val);
  SK_CUDA(cudaGetLastError());
  SK_CUDA(cudaDeviceSynchronize());
  cudaFree(fill);
  t->rowptr = t->own_rowptr;
  t->colind = t->own_colind;
  t->val = t->own_val;
  return SK_OK;
}

}  // namespace sk

using namespace sk;

extern "C" {

const char* sk_last_error(void) { return g_err; }

const char* sk_status_string(sk_status st) {
  switch (st) {
    case SK_OK: return "SK_OK";
    case SK_EINVAL: return "SK_EINVAL";
    case SK_ENOMEM: return "SK_ENOMEM";
    case SK_ECUDA: return "SK_ECUDA";
    case SK_ENAN: return "SK_ENAN";
    case SK_ENOCONV: return "SK_ENOCONV";
    case SK_EILLCOND: return "SK_EILLCOND";
    case SK_ETIMEOUT: return "SK_ETIMEOUT";
    case SK_EHASH: return "SK_EHASH";
  }
  return "unknown status";
}

void sk_opts_default(sk_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->sketch = SK_SPARSE_SIGN;
  o->zeta = 0;
  o->seed = 7;
  o->stab_tol = 0;
  o->maxit = 10000;
  o->basis = SK_F64;
  o->cgs_passes = 2;
  o->tau = 1e-8;
  o->symmetric = 0;
  o->breakdown = 0;
  o->use_graph = 1;
  o->persistent = 0;
  o->batch_workers = 0;
  o->basis_kind = SK_BASIS_ARNOLDI;
  o->cheb_c = o->cheb_dx = o->cheb_dy = 0;
  o->barrier_spins = 0;
  o->iter_chunk = 0;
  o->pipeline = 1;
  o->batch_mode = 0;
  o->batch_elems = 0;
}

static sk_op* new_op() {
  sk_op* op = new (std::nothrow) sk_op;
  if (op) std::memset(op, 0, sizeof(*op));
  return op;
}

sk_status sk_op_stencil5(sk_op** out, int nx, int ny, const double* coef, const double* shift) {
  SK_CHECK_ARG(out != nullptr && coef != nullptr, "op and coef must not be NULL");
  SK_CHECK_ARG(nx >= 1 && ny >= 1, "nx, ny >= 1");
  for (int q = 0; q < 5; ++q) SK_CHECK_ARG(std::isfinite(coef[q]), "coefficients must be finite");
  sk_op* op = new_op();
  if (!op) { set_error("out of host memory"); return SK_ENOMEM; }
  op->kind = OP_STENCIL5;
  op->nx = nx;
  op->ny = ny;
  op->n = (int64_t)nx * ny;
  for (int q = 0; q < 5; ++q) op->coef[q] = coef[q];
  op->shift = shift;
  *out = op;
  return SK_OK;
}

sk_status sk_op_diffusion_var(sk_op** out, int nx, int ny, const double* theta) {
  SK_CHECK_ARG(out != nullptr && theta != nullptr, "op and theta must not be NULL");
  SK_CHECK_ARG(nx >= 1 && ny >= 1, "nx, ny >= 1");
  sk_op* op = new_op();
  if (!op) { set_error("out of host memory"); return SK_ENOMEM; }
  op->kind = OP_DIFFUSION;
  op->nx = nx;
  op->ny = ny;
  op->n = (int64_t)nx * ny;
  op->theta = theta;
  *out = op;
  return SK_OK;
}

sk_status sk_op_csr(sk_op** out, int64_t n, int64_t nnz, const int32_t* rowptr, const int32_t* colind,
                    const double* val) {
  SK_CHECK_ARG(out != nullptr && rowptr != nullptr && colind != nullptr && val != nullptr, "NULL CSR array");
  SK_CHECK_ARG(n >= 1 && nnz >= 0 && n < (1ll << 31) && nnz < (1ll << 31), "CSR sizes must fit int32");
  sk_op* op = new_op();
  if (!op) { set_error("out of host memory"); return SK_ENOMEM; }
  op->kind = OP_CSR;
  op->n = n;
  op->nx = (int)n;
  op->ny = 1;
  op->nnz = nnz;
  op->rowptr = rowptr;
  op->colind = colind;
  op->val = val;
  const sk_status r = build_sell(op);
  if (r != SK_OK) { sk_op_destroy(op); return r; }
  *out = op;
  return SK_OK;
}

sk_status sk_op_transpose(const sk_op* op, sk_op** opT) {
  SK_CHECK_ARG(op != nullptr && opT != nullptr, "NULL op");
  sk_op* t = new_op();
  if (!t) { set_error("out of host memory"); return SK_ENOMEM; }
  if (op->kind == OP_CSR) {
    t->kind = OP_CSR;
    t->n = op->n;
    t->nx = op->nx;
    t->ny = 1;
    t->nnz = op->nnz;
    sk_status r = build_csr_transpose(op, t);
    if (r == SK_OK) r = build_sell(t);
    if (r != SK_OK) { sk_op_destroy(t); return r; }
    *opT = t;
    return SK_OK;
  }
  t->kind = op->kind;
  t->nx = op->nx;
  t->ny = op->ny;
  t->n = op->n;
  t->shift = op->shift;
  t->theta = op->theta;
  t->coef[0] = op->coef[0];
  // (A^T)_{P,Q} = A_{Q,P}: the E coefficient of A^T is A's W coefficient, etc.
  t->coef[1] = op->coef[2];
  t->coef[2] = op->coef[1];
  t->coef[3] = op->coef[4];
  t->coef[4] = op->coef[3];
  *opT = t;
  return SK_OK;
}

int64_t sk_op_n(const sk_op* op) { return op ? op->n : 0; }

sk_status sk_op_param_grad(const sk_op* op, const double* lam, const double* x, double alpha, double* grad,
                           void* stream) {
  SK_CHECK_ARG(op != nullptr && lam != nullptr && x != nullptr && grad != nullptr, "NULL argument");
  SK_CHECK_ARG(std::isfinite(alpha), "alpha must be finite");
  cudaStream_t st = (cudaStream_t)stream;
  int blocks = (int)((op->n + 255) / 256);
  if (blocks > 4 * num_sms()) blocks = 4 * num_sms();
  if (op->kind == OP_DIFFUSION) {
    diffusion_grad_kernel<<<blocks, 256, 0, st>>>(op->nx, op->ny, lam, x, alpha, grad);
  } else if (op->kind == OP_STENCIL5) {
    Scratch sc(st);
    double* part = nullptr;
    SK_TRY(sc.alloc(&part, (size_t)blocks * 5));
    stencil_grad_kernel<<<blocks, 256, 0, st>>>(op->nx, op->ny, lam, x, alpha, part, op->shift ? grad + 5 : nullptr);
    sum_parts_kernel<<<1, 32, 0, st>>>(part, blocks, 5, alpha, grad);
  } else {
    csr_grad_kernel<<<blocks, 256, 0, st>>>(op->n, op->rowptr, op->colind, lam, x, alpha, grad);
  }
  SK_CUDA(cudaGetLastError());
  return SK_OK;
}

void sk_op_destroy(sk_op* op) {
  if (!op) return;
  if (op->shift32) cudaFree(op->shift32);
  if (op->theta32) cudaFree(op->theta32);
  if (op->val32) cudaFree(op->val32);
  if (op->sell_ptr) cudaFree(op->sell_ptr);
  if (op->sell_col) cudaFree(op->sell_col);
  if (op->sell_val) cudaFree(op->sell_val);
  if (op->sell_val32) cudaFree(op->sell_val32);
  if (op->own_rowptr) cudaFree(op->own_rowptr);
  if (op->own_colind) cudaFree(op->own_colind);
  if (op->own_val) cudaFree(op->own_val);
  delete op;
}

sk_status sk_op_apply(const sk_op* op, const double* x, double* y, void* stream) {
  SK_CHECK_ARG(op != nullptr && x != nullptr && y != nullptr, "NULL argument");
  SK_CHECK_ARG(x != y, "x and y must not alias");
  cudaStream_t st = (cudaStream_t)stream;
  OpView<double> v;
  make_view(op, &v);
  int blocks = (int)((op->n + 255) / 256);
  if (blocks > 8 * num_sms()) blocks = 8 * num_sms();
  op_apply_kernel<<<blocks, 256, 0, st>>>(v, x, y);
  SK_CUDA(cudaGetLastError());
  return SK_OK;
}

sk_status sketch_apply(const sk_sketch* S, const void* B, int64_t ldb, int ncols, sk_dtype dtype, double* SB,
                       void* stream) {
  SK_CHECK_ARG(S != nullptr && B != nullptr && SB != nullptr, "NULL argument");
  SK_CHECK_ARG(ncols >= 1, "ncols >= 1");
  SK_CHECK_ARG(ldb >= S->n, "ldb >= n");
  SK_CHECK_ARG(dtype == SK_F64 || dtype == SK_F32 || dtype == SK_BF16, "dtype");
  return sketch_apply_impl(S, B, ldb, ncols, dtype, SB, (cudaStream_t)stream);
}

}  // extern "C"
