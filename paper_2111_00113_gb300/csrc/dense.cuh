// Small dense FP64 kernels of the sketched problems (dense.cu).
#pragma once
#include "common.cuh"

namespace sk {

static constexpr int kQrNb = 16;            // panel width of the blocked Householder QR
static constexpr int kQrPanelThreads = 512;

// js, nj: the same problem shape for nj job slots at once (grid.y = nj; see
// JobSlab); the defaults are one problem at the given pointers.
sk_status enqueue_hbar_product(const double* SB, const double* Hbar, int s, int d, int k, const int* stop,
                               double* Aug, cudaStream_t st, const JobSlab& js = JobSlab(), int nj = 1);
sk_status enqueue_copy_sb(const double* SB, int s, int d, const int* stop, double* Aug, cudaStream_t st);
sk_status enqueue_qr(double* Aug, int s, int nq, int ncols, double* rdiag, double* tau, double* Tws,
                     cudaStream_t st, const JobSlab& js = JobSlab(), int nj = 1);
sk_status enqueue_ls_solve(const double* Aug, const double* rdiag, int s, int d, double stab_tol, double* y,
                           double* diag, cudaStream_t st, const JobSlab& js = JobSlab(), int nj = 1);
// Iterative sGMRES (§5.2): the product on columns [c0, c1) only; the solve
// with Q^T g read from z (d = the prefix solved); the QR grown by columns
// [c0, c1) with column zc holding Q^T g; the early-stop test of a chunk.
sk_status enqueue_hbar_product_cols(const double* SB, const double* Hbar, int s, int d, int k, const int* stop,
                                    int c0, int c1, double* Aug, cudaStream_t st, const JobSlab& js = JobSlab(),
                                    int nj = 1);
sk_status enqueue_ls_solve_z(const double* Aug, const double* rdiag, const double* z, int s, int d, double stab_tol,
                             double* y, double* diag, cudaStream_t st, const JobSlab& js = JobSlab(), int nj = 1);
sk_status enqueue_qr_append(double* Aug, int s, int c0, int c1, int zc, double* rdiag, double* tau, double* Tws,
                            long long* launches, cudaStream_t st);
// tau: device scalar (read when the check runs, so a captured chunk serves
// every cycle)
sk_status enqueue_prefix_check(const double* z, const double* rdiag, const int* stop, int s, int c0, int c1,
                               const double* tau, double stab_tol, int* out, cudaStream_t st);

// Eigenpairs of a d x d FP64 matrix (eig.cu).  M is overwritten by its
// Hessenberg form and reflectors; tau needs 2d entries.  Yre/Yim (d x nev)
// receive the eigenvectors of the nev selected eigenvalues (largest real
// part first) in the order of sel.
sk_status enqueue_eig(double* M, int n, int nev, double* tau, double* wr, double* wi, int* sel, double* Wre,
                      double* Wim, double* Yre, double* Yim, int* status, cudaStream_t st);

}  // namespace sk
