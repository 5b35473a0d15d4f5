// Grouped batched sGMRES: one launch advances one phase of every active job
// (grouped.cu drives it).  Kernels whose grid depends on a job's n take a
// flat block map (map[blockIdx.x] = {job slot, the job's own block index})
// and read the job's parameters from a GJob array in device memory; the
// small dense problems (same shape in every job) take blockIdx.y = slot and
// a JobSlab.  Each job's arithmetic is the single-system path's, block for
// block, so a job's iterates do not depend on which jobs share its launches.
#pragma once
#include <string>

#include "basis.cuh"
#include "common.cuh"

namespace sk {

struct GJob {
  BasisParams bp;        // the job's basis build (pointers into its buffers and slab)
  OpView<float> Af;      // operator views (FP32 one only for FP32/BF16 bases)
  OpView<double> Ad;
  int vec;               // basis path: 1 = 4 cells of one row, 2 = 4 cells across rows, 0 = scalar
  int vgrid;             // blocks of the residual and norm kernels
  int ugrid, uvec;       // blocks of the update kernel; 4 rows per thread if uvec
  const double* b;
  double* x;
  double* vpart;         // vgrid partial sums
  unsigned* vcnt;        // 2 last-block counters (residual, norm of b)
  double* bn2;           // ||b||^2
  // sparse sign sketch (shared by the jobs of one n)
  const uint32_t* rowptr;
  const uint16_t* entries;
  int nchunks;
  int rows_ntiles, rows_ngroups, rows_cpg;  // S B_{d+1}: row-owner gather shape
  int col_ngroups, col_cpg;                 // g = S r: one-column gather shape
  double* rows_part;     // rows_ngroups x (d+1) x s
  double* col_part;      // col_ngroups x s
  double* g;             // s (in the slab)
  double* SB;            // s x (d+1) (in the slab)
  double* y;             // d: the LS solution (in the slab)
  double* out;           // [rho2, rhat, kappa, width] (in the slab; the LS solve writes out + 1)
};

template <typename C> __device__ __forceinline__ const OpView<C>& job_view(const GJob& J);
template <> __device__ __forceinline__ const OpView<float>& job_view<float>(const GJob& J) { return J.Af; }
template <> __device__ __forceinline__ const OpView<double>& job_view<double>(const GJob& J) { return J.Ad; }

// Grouped launches of the basis (basis.cu), the sketches (sketch.cu) and the
// vector kernels (solve.cu).  `map` and `ids` are device arrays; `nmap`
// blocks in the flat launches, `nj` slots in the per-slot ones.
sk_status enqueue_basis_grouped(const GJob* jobs, const int2* map, int nmap, sk_dtype dt, int k, int passes, int d,
                                cudaStream_t st);
sk_status enqueue_sketch_rows_grouped(const GJob* jobs, const int2* map, int nmap, const int* ids, int nj, sk_dtype dt,
                                      int ncols, int s, int zeta, cudaStream_t st);
sk_status enqueue_sketch_col_grouped(const GJob* jobs, const int2* map, int nmap, const int* ids, int nj, int s,
                                     int zeta, cudaStream_t st);
enum GroupedVec { GV_RESIDUAL = 0, GV_NORM_B = 1, GV_UPDATE = 2 };
// r = b - A x with ||r||^2 into bp.rho2; ||b||^2 into bn2; x += B y (width
// out[3]).  Blocks per job: vgrid (residual, norm) and ugrid (update).
sk_status enqueue_vec_grouped(GroupedVec which, const GJob* jobs, const int2* map, int nmap, sk_dtype dt, int d,
                              cudaStream_t st);
int vec_grid(int64_t n);
int update_grid(int64_t n, int G);
// Gather shapes of one job: rows gather of ncols basis columns (block
// grouping) and the one-column FP64 gather of r, as the single path picks them.
void sketch_shapes(const SketchPlan& p, int ncols, sk_dtype dt, int* rows_ntiles, int* rows_ngroups, int* rows_cpg,
                   int* col_ngroups, int* col_cpg);

// The grouped driver (grouped.cu): whether the options allow it (else *why
// names what it needs), and the batched solve itself (the arguments of
// sgmres_solve_batched; opts unresolved).
bool grouped_supported(const sk_opts& o, int d, int s, std::string* why);
sk_status sgmres_batched_grouped(int nsys, const sk_op* const* A, int nrhs, const double* const* b, double* const* x,
                                 int d, int k, int s, double tol, const sk_opts& o, sk_status* per_job,
                                 sk_info* job_info, sk_info* info, cudaStream_t st);

}  // namespace sk
