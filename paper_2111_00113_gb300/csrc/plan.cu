// Reusable sketch plans: the sparse sign map's row-sorted index tables (or
// the SRHT's signs and sampled rows) built once and applied to many blocks
// of columns, so that repeated sketches of the same shape pay only the
// gather (or the transform) and the reduction.
#include "common.cuh"
#include "srr.cuh"

struct sk_sketch_plan {
  sk::Sketcher sk;
  sk::Scratch* tables;  // the plan's device tables
  double* ws;           // per-group partial sums, grown on demand
  size_t ws_cap;        // doubles
  int64_t n;
};

using namespace sk;

static void plan_free(sk_sketch_plan* p) {
  if (!p) return;
  if (p->tables) {
    for (int i = 0; i < p->tables->n; ++i)
      if (p->tables->ptr[i]) cudaFree(p->tables->ptr[i]);
    p->tables->n = 0;
    delete p->tables;
  }
  if (p->ws) cudaFree(p->ws);
  delete p;
}

extern "C" sk_status sk_sketch_plan_create(const sk_sketch* S, sk_sketch_plan** plan, void* stream) {
  SK_CHECK_ARG(S != nullptr && plan != nullptr, "NULL argument");
  SK_CHECK_ARG(S->n >= 1 && S->s >= 1, "need n >= 1 and s >= 1");
  SK_CHECK_ARG(S->kind == SK_SPARSE_SIGN || S->kind == SK_SRHT, "unknown sketch kind");
  *plan = nullptr;
  cudaStream_t st = (cudaStream_t)stream;
  sk_sketch_plan* p = new (std::nothrow) sk_sketch_plan();
  if (!p) { set_error("out of host memory"); return SK_ENOMEM; }
  p->tables = new (std::nothrow) Scratch(st);
  p->ws = nullptr;
  p->ws_cap = 0;
  p->n = S->n;
  if (!p->tables) { plan_free(p); set_error("out of host memory"); return SK_ENOMEM; }
  const sk_status r = p->sk.create(*S, *p->tables, st);
  if (r != SK_OK) { plan_free(p); return r; }
  *plan = p;
  return SK_OK;
}

extern "C" sk_status sk_sketch_plan_apply(sk_sketch_plan* p, const void* B, int64_t ldb, int ncols, sk_dtype dtype,
                                          double* SB, void* stream) {
  SK_CHECK_ARG(p != nullptr && B != nullptr && SB != nullptr, "NULL argument");
  SK_CHECK_ARG(ncols >= 1, "ncols >= 1");
  SK_CHECK_ARG(ldb >= p->n, "ldb >= n");
  SK_CHECK_ARG(dtype == SK_F64 || dtype == SK_F32 || dtype == SK_BF16, "dtype");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t need = p->sk.ws(ncols, dtype, false);
  if (need > p->ws_cap) {
    if (p->ws) {
      SK_CUDA(cudaStreamSynchronize(st));
      SK_CUDA(cudaFree(p->ws));
      p->ws = nullptr;
      p->ws_cap = 0;
    }
    cudaError_t e = cudaMalloc((void**)&p->ws, need * sizeof(double));
    if (e != cudaSuccess) {
      cudaGetLastError();
      p->ws = nullptr;
      set_error("cudaMalloc(%zu bytes) failed: %s", need * sizeof(double), cudaGetErrorString(e));
      return SK_ENOMEM;
    }
    p->ws_cap = need;
  }
  return p->sk.apply(B, ldb, ncols, dtype, SB, p->ws, st, false);
}

extern "C" void sk_sketch_plan_destroy(sk_sketch_plan* p) { plan_free(p); }
