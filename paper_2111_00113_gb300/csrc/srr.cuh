// Internal interfaces shared by the solvers (solve.cu) and the sketched
// Rayleigh-Ritz code (srr.cu).
#pragma once
#include "common.cuh"

namespace sk {

static constexpr int kMaxSrrD = 232;  // the eigensolver's shared-memory limit (eig.cu)
static constexpr int kMaxNev = 32;

struct Sketcher {
  sk_sketch_kind kind = SK_SPARSE_SIGN;
  SketchPlan sp;
  SrhtPlan hp;
  int s = 0, zeta = 0;
  sk_status create(const sk_sketch& S, Scratch& sc, cudaStream_t st) {
    kind = S.kind;
    s = S.s;
    if (kind == SK_SRHT) return srht_plan_create(&hp, &S, sc, st);
    SK_TRY(plan_create(&sp, &S, sc, st));
    zeta = sp.zeta;
    return check_plan_status(sp, st);
  }
  // block = basis columns (a fixed summation order per column, whether the
  // basis is sketched whole or in blocks); false for the residual
  size_t ws(int ncols, sk_dtype dt, bool block) const {
    return kind == SK_SRHT ? srht_ws_doubles(hp, ncols, block) : plan_ws_doubles(sp, ncols, dt, block);
  }
  sk_status apply(const void* B, int64_t ldb, int ncols, sk_dtype dt, double* out, double* ws, cudaStream_t st,
                  bool block) const {
    if (kind == SK_SRHT) return srht_apply_ws(hp, B, ldb, ncols, dt, out, ws, st, block);
    return plan_apply_ws(sp, B, ldb, ncols, dt, out, ws, st, block);
  }
};

void resolve_opts(const sk_opts* in, sk_opts* o, int d);
sk_status check_passes(const sk_opts& o);

// Outputs of a sketched Rayleigh-Ritz call (host arrays of nev, device X).
struct SrrOut {
  double* lam_re;
  double* lam_im;
  double* X_re;   // device n x nev
  double* X_im;   // device n x nev or NULL
  double* rhat;
  int* nconv;
  int* rank;      // stabilized form: singular values kept (host, or NULL)
};

// The reduction after the sketches (§6.3-§6.5).  Aug (device, s x 2d, ld s):
// columns [0, d) = C = S B, [d, 2d) = D = S A B; overwritten.  B: the basis
// (device, n x d of dt, leading dimension ldb); colscale (device, d, or
// NULL): B's column j is used as B[:, j] * colscale[j] (C and D already hold
// the scaled columns).  trunc_tol <= 0: Algorithm 2 (Householder QR of C,
// M-hat = T^{-1} U^T D); > 0: the stabilized form of §6.5 (truncated SVD of
// C keeping sigma_1 / sigma_i <= trunc_tol, eig of Sigma_r^{-1} U_r^T D V_r).
// Synchronises the stream; fills `out`.  *eig_fail is set when the QR
// iteration did not converge.
sk_status srr_tail(double* Aug, int s, int d, const void* B, int64_t ldb, int64_t n, sk_dtype dt,
                   const double* colscale, int nev, int symmetric, double tau, double trunc_tol, SrrOut out,
                   Scratch& sc, cudaStream_t st, int* eig_fail);

}  // namespace sk
