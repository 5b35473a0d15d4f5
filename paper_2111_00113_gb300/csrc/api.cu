// C ABI plumbing: errors, options, operator objects, operator apply and the
// sketch_apply entry point.
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
  *out = op;
  return SK_OK;
}

sk_status sk_op_transpose(const sk_op* op, sk_op** opT) {
  SK_CHECK_ARG(op != nullptr && opT != nullptr, "NULL op");
  SK_CHECK_ARG(op->kind != OP_CSR, "transpose of a CSR op is not supported");
  sk_op* t = new_op();
  if (!t) { set_error("out of host memory"); return SK_ENOMEM; }
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
