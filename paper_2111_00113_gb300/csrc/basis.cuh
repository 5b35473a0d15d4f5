// Parameters of the truncated-Arnoldi basis kernels (basis.cu).
#pragma once
#include "common.cuh"

namespace sk {

static constexpr int kBasisThreads = 256;
static constexpr int kMaxK = 16;

struct BasisParams {
  int64_t n;
  int d, k, passes;
  sk_dtype dtype;
  void* B;            // n x (d+1) basis, storage dtype, leading dimension ldb
  int64_t ldb;
  double* h1;         // d x k first-pass coefficients
  double* h2;         // d x k second-pass coefficients
  double* nu;         // d: ||w_{j+1}||
  double* mn2;        // d: ||A b_j||^2
  double* Hbar;       // (d+1) x d or NULL (zeroed by the caller)
  double* M;          // n: A b_j in FP64 (FP64 basis only; NULL otherwise)
  double* partial;    // nblk x (kMaxK+1) per-CTA partial sums (held in the compute type)
  void* coef;         // d x (kMaxK+1) in the compute type: step j's combined
                      // coefficients h1+h2 (first k) and 1/nu_j (entry kMaxK),
                      // written once by the step's finalising thread
  unsigned* counters; // 2 last-block counters (zero)
  int* stop;          // valid basis columns (init d+1; lowered on breakdown)
  int* nanflag;       // set on NaN/Inf
  const double* r;    // starting vector (FP64)
  const double* rho2; // ||r||^2 (device)
  double bd;          // breakdown threshold
  int nblk;           // CTAs per pass (set by enqueue_basis)
  int nblk_cap;       // partial-sum rows allocated
  int j_begin, j_end; // truncated Arnoldi: steps [j_begin, j_end) of this launch
                      // sequence (j_end = 0: all d); step j forms b_{j+1}.
                      // j_begin > 0 resumes a build whose steps < j_begin ran
  int pdl_resume;     // j_begin > 0: the previous node in the stream is the form
                      // kernel of step j_begin - 1 (programmatic edge allowed)
  int prio;           // launch priority of the basis kernels (0: the stream's)
  // Chebyshev basis (kind == SK_BASIS_CHEBYSHEV): B holds the recurrence's
  // vectors v_j (scaled by powers of two, not normalised); sigma[j] =
  // ||v_j||, and Hbar = H_v diag(1/sigma) so that S B Hbar = S A B diag(1/sigma)
  int kind;
  double cheb_c, cheb_rho, cheb_gamma;
  double* sigma;      // d+1
  double* cheb_part;  // (d+1) x nblk_cap per-CTA partial sums of ||v_j||^2 (compute type)
};

// Workspace of the persistent (cooperative) basis kernel.
struct PersistWork {
  unsigned* bar;         // 2: barrier count and generation (reset before each launch)
  int* err;              // SK_ETIMEOUT if a grid barrier gave up
  double* part;          // 3 x grid x (kMaxK+1) partial sums
  long long spin_limit;  // barrier spin iterations before giving up
};

bool persist_shape(const sk_op* op, sk_dtype dt, int k, int* grid, int* ept, size_t* smem);
sk_status enqueue_basis_persistent(const BasisParams& bp, const sk_op* op, PersistWork& w, cudaStream_t st);

int basis_grid(int64_t n, int G);
bool basis_vector_path(const sk_op* op, int64_t ldb, const void* B);
sk_status enqueue_basis(const BasisParams& p, const sk_op* op, cudaStream_t st);
// Chebyshev, a build in step ranges (j_end > 0): sigma_j and column j of
// Hbar for j in [j0, j1), once the steps forming v_j (and v_1, for j = 0)
// have run.
sk_status enqueue_cheb_finalize(const BasisParams& p, const sk_op* op, int j0, int j1, cudaStream_t st);
// Chebyshev: rescale B's columns to unit norm and Hbar to the unit basis
// (diag(sigma) Hbar), for callers that want the normalised basis itself.
sk_status enqueue_cheb_normalize(const BasisParams& p, cudaStream_t st);

}  // namespace sk
