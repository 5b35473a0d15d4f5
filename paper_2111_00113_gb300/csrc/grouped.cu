// Grouped batched sGMRES (sgmres_solve_batched, batch_mode 0 or 1): many
// independent (system, right-hand side) jobs advanced together, one launch
// per phase of a restart cycle (Algorithm 1 with restarts, §3.5) for every
// resident job.
//
// Jobs are admitted largest first while the resident systems' sizes sum to
// at most opts.batch_elems; each job owns a slot (a slab of its small dense
// problem, the same layout in every slot) and its n-sized buffers.  Per
// cycle the host builds flat block maps of the resident jobs, launches the
// cycle's kernels once each (about 3d + 20 launches for all jobs), reads
// back one row of scalars per job, retires the jobs that converged or
// failed and admits new ones.  A job's arithmetic is the single-system
// path's kernel bodies with the same block shapes, so its iterates are
// those of sgmres_solve on the same inputs (captured-graph cycle).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "basis.cuh"
#include "common.cuh"
#include "dense.cuh"
#include "grouped.cuh"
#include "srr.cuh"

namespace sk {

namespace {

constexpr int kResStride = 8;  // doubles read back per job and cycle

// Slab of one slot (in doubles, 256-byte aligned pieces).
struct SlabLayout {
  int64_t SB, Aug, g, rdiag, tau, Tws, y, out, Hbar, h1, h2, nu, mn2, coef, rho2, ints, total;
  void init(int s, int d, int k) {
    int64_t o = 0;
    auto take = [&](int64_t n) {
      const int64_t at = o;
      o += (n + 31) / 32 * 32;
      return at;
    };
    SB = take((int64_t)s * (d + 1));
    Aug = take((int64_t)s * (d + 1));
    g = take(s);
    rdiag = take(d);
    tau = take(d);
    Tws = take((int64_t)((d + kQrNb - 1) / kQrNb) * kQrNb * kQrNb);
    y = take(d);
    out = take(4);
    Hbar = take((int64_t)(d + 1) * d);
    h1 = take((int64_t)d * k);
    h2 = take((int64_t)d * k);
    nu = take(d);
    mn2 = take(d);
    coef = take((int64_t)d * (kMaxK + 1));
    rho2 = take(2);   // ||r||^2, ||b||^2
    ints = take(8);   // stop, nanflag, 8 basis counters, 2 vector counters (12 ints)
    total = o;
  }
};

// stop = d + 1, nanflag = 0 and Hbar = 0 in every listed slot (the start of
// a basis build).
__global__ void g_init_kernel(double* Hbar, int* stop, int d, JobSlab js) {
  Hbar = at_job(Hbar, js);
  stop = at_job(stop, js);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    stop[0] = d + 1;
    stop[1] = 0;
  }
  const int64_t total = (int64_t)(d + 1) * d;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x)
    Hbar[q] = 0.0;
}

// Aug[:, d] = g in every listed slot.
__global__ void g_copy_kernel(const double* src, double* dst, int count, JobSlab js) {
  src = at_job(src, js);
  dst = at_job(dst, js);
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < count; q += gridDim.x * blockDim.x) dst[q] = src[q];
}

// One row of scalars per listed job: rho2, rhat, kappa, width, stop,
// nanflag, ||b||^2.
__global__ void g_collect_kernel(const GJob* __restrict__ jobs, const int* __restrict__ ids, int nj,
                                 double* __restrict__ res) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nj) return;
  const GJob& J = jobs[ids[t]];
  double* o = res + (int64_t)kResStride * t;
  o[0] = *J.bp.rho2;
  o[1] = J.out[1];
  o[2] = J.out[2];
  o[3] = J.out[3];
  o[4] = (double)*J.bp.stop;
  o[5] = (double)*J.bp.nanflag;
  o[6] = *J.bn2;
  o[7] = 0.0;
}

size_t r256(size_t b) { return (b + 255) & ~(size_t)255; }

// n-sized buffers of one job (byte offsets into one allocation).
struct VecLayout {
  size_t B, r, M, bpart, vpart, rows_part, col_part, total;
};

struct PlanEntry {
  Scratch* sc = nullptr;
  SketchPlan plan;
  int rows_ntiles = 0, rows_ngroups = 0, rows_cpg = 0, col_ngroups = 0, col_cpg = 0;
};

struct SlotState {
  int job = -1;
  unsigned char* mem = nullptr;
  double bnorm = 0, relres = 0, rhat = 0, kmax = 0;
  int cycles = 0, width = 0, stop = 0;
  long long launches = 0;
  float ms[5] = {0, 0, 0, 0, 0};
  std::chrono::steady_clock::time_point t0;
};

}  // namespace

bool grouped_supported(const sk_opts& o, int d, int s, std::string* why) {
  if (o.sketch != SK_SPARSE_SIGN) { *why = "the sparse sign sketch"; return false; }
  if (o.basis_kind != SK_BASIS_ARNOLDI) { *why = "the truncated-Arnoldi basis"; return false; }
  if (o.iter_chunk != 0) { *why = "iter_chunk = 0"; return false; }
  if (o.basis != SK_F32 && o.basis != SK_F64) { *why = "an FP32 or FP64 basis"; return false; }
  if ((size_t)d * 33 * sizeof(double) > (size_t)kDynSmemLimit) { *why = "d small enough for the LS solve"; return false; }
  // the gathers' kernels depend on s, zeta and the type only
  sk_sketch S;
  S.kind = SK_SPARSE_SIGN;
  S.n = 1 << 20;
  S.s = s;
  S.zeta = o.zeta;
  S.seed = o.seed;
  SketchPlan sp;
  SrhtPlan hp;
  sketch_plan_shape(S, &sp, &hp);
  int a = 0, b = 0, c = 0, e = 0, f = 0;
  sketch_shapes(sp, d + 1, o.basis, &a, &b, &c, &e, &f);
  if (a == 0 || e == 0) { *why = "s <= 640 (the row-owner sketch kernels)"; return false; }
  return true;
}

sk_status sgmres_batched_grouped(int nsys, const sk_op* const* A, int nrhs, const double* const* b, double* const* x,
                                 int d, int k, int s, double tol, const sk_opts& oin, sk_status* per_job,
                                 sk_info* job_info, sk_info* info, cudaStream_t st) {
  sk_opts o;
  resolve_opts(&oin, &o, d);
  SK_TRY(check_passes(o));
  const sk_dtype dt = o.basis;
  const int njobs = nsys * nrhs;
  const long long cap = o.batch_elems > 0 ? o.batch_elems : (1ll << 22);
  auto job_n = [&](int q) { return A[q / nrhs]->n; };
  std::vector<int> order(njobs);
  for (int q = 0; q < njobs; ++q) order[q] = q;
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return job_n(a) > job_n(c); });
  int64_t nmin = job_n(order[njobs - 1]);
  if (nmin < 1) nmin = 1;
  int64_t ns64 = cap / nmin + 1;
  if (ns64 > njobs) ns64 = njobs;
  if (ns64 > 65535) ns64 = 65535;
  const int nslots = (int)ns64;
  SlabLayout L;
  L.init(s, d, k);
  JobSlab js;
  js.stride = L.total * (int64_t)sizeof(double);

  auto t_start = std::chrono::steady_clock::now();
  Scratch sc(st);
  double* slab = nullptr;
  GJob* d_jobs = nullptr;
  int* d_ids = nullptr;
  double* d_res = nullptr;
  SK_TRY(sc.alloc(&slab, (size_t)L.total * nslots));
  SK_TRY(sc.alloc(&d_jobs, (size_t)nslots));
  SK_TRY(sc.alloc(&d_ids, (size_t)nslots));
  SK_TRY(sc.alloc(&d_res, (size_t)kResStride * nslots));
  SK_CUDA(cudaMemsetAsync(slab, 0, sizeof(double) * (size_t)L.total * nslots, st));
  js.ids = d_ids;

  // host state; pinned staging for the job descriptors, ids, maps and results
  std::vector<SlotState> slots(nslots);
  struct Host {
    GJob* jobs = nullptr;
    int* ids = nullptr;
    double* res = nullptr;
    int* pstat = nullptr;
    int2* map = nullptr;
    size_t map_cap = 0;
    int2* d_map = nullptr;
    size_t d_map_cap = 0;
    cudaStream_t st = nullptr;
    cudaEvent_t ev[8] = {};
    std::map<int64_t, PlanEntry> plans;
    std::vector<SlotState>* slots = nullptr;
    ~Host() {
      if (st) cudaStreamSynchronize(st);
      if (slots)
        for (auto& S : *slots)
          if (S.mem) cudaFreeAsync(S.mem, st);
      for (auto& kv : plans) delete kv.second.sc;
      if (d_map) cudaFreeAsync(d_map, st);
      if (jobs) cudaFreeHost(jobs);
      if (ids) cudaFreeHost(ids);
      if (res) cudaFreeHost(res);
      if (pstat) cudaFreeHost(pstat);
      if (map) cudaFreeHost(map);
      for (cudaEvent_t e : ev)
        if (e) cudaEventDestroy(e);
    }
  } H;
  H.st = st;
  H.slots = &slots;
  SK_CUDA(cudaMallocHost((void**)&H.jobs, sizeof(GJob) * (size_t)nslots));
  SK_CUDA(cudaMallocHost((void**)&H.ids, sizeof(int) * (size_t)nslots));
  SK_CUDA(cudaMallocHost((void**)&H.res, sizeof(double) * (size_t)kResStride * nslots));
  SK_CUDA(cudaMallocHost((void**)&H.pstat, sizeof(int) * (size_t)nslots));
  for (int e = 0; e < 8; ++e) SK_CUDA(cudaEventCreate(&H.ev[e]));

  // maps and ids of a slot list: uploaded into H.d_map / d_ids (call after a sync)
  struct Maps { size_t basis, vec, upd, rows, col, end; };
  auto upload = [&](const std::vector<int>& list, Maps* m) -> sk_status {
    std::vector<int2> hm;
    auto add = [&](auto count) {
      for (int slot : list) {
        const int c = count(H.jobs[slot]);
        for (int i = 0; i < c; ++i) hm.push_back(make_int2(slot, i));
      }
    };
    m->basis = hm.size();
    add([](const GJob& J) { return J.bp.nblk; });
    m->vec = hm.size();
    add([](const GJob& J) { return J.vgrid; });
    m->upd = hm.size();
    add([](const GJob& J) { return J.ugrid; });
    m->rows = hm.size();
    add([](const GJob& J) { return J.rows_ntiles * J.rows_ngroups; });
    m->col = hm.size();
    add([](const GJob& J) { return J.col_ngroups; });
    m->end = hm.size();
    if (hm.size() > H.map_cap) {
      if (H.map) cudaFreeHost(H.map);
      H.map = nullptr;
      H.map_cap = hm.size() + hm.size() / 2 + 1024;
      SK_CUDA(cudaMallocHost((void**)&H.map, sizeof(int2) * H.map_cap));
    }
    if (hm.size() > H.d_map_cap) {
      if (H.d_map) SK_CUDA(cudaFreeAsync(H.d_map, st));
      H.d_map = nullptr;
      H.d_map_cap = hm.size() + hm.size() / 2 + 1024;
      SK_CUDA(cudaMallocAsync((void**)&H.d_map, sizeof(int2) * H.d_map_cap, st));
    }
    std::memcpy(H.map, hm.data(), sizeof(int2) * hm.size());
    for (size_t i = 0; i < list.size(); ++i) H.ids[i] = list[i];
    SK_CUDA(cudaMemcpyAsync(H.d_map, H.map, sizeof(int2) * hm.size(), cudaMemcpyHostToDevice, st));
    SK_CUDA(cudaMemcpyAsync(d_ids, H.ids, sizeof(int) * list.size(), cudaMemcpyHostToDevice, st));
    return SK_OK;
  };
  auto collect = [&](int nj) -> sk_status {
    g_collect_kernel<<<(nj + 127) / 128, 128, 0, st>>>(d_jobs, d_ids, nj, d_res);
    SK_CUDA(cudaGetLastError());
    SK_CUDA(cudaMemcpyAsync(H.res, d_res, sizeof(double) * (size_t)kResStride * nj, cudaMemcpyDeviceToHost, st));
    return SK_OK;
  };

  // the sketch plan of size n (one per distinct n; the jobs of one n share it)
  std::vector<int64_t> new_plans;
  auto plan_for = [&](int64_t n, PlanEntry** out) -> sk_status {
    auto it = H.plans.find(n);
    if (it != H.plans.end()) { *out = &it->second; return SK_OK; }
    PlanEntry& e = H.plans[n];
    e.sc = new Scratch(st);
    sk_sketch S;
    S.kind = SK_SPARSE_SIGN;
    S.n = n;
    S.s = s;
    S.zeta = o.zeta;
    S.seed = o.seed;
    SK_TRY(plan_create(&e.plan, &S, *e.sc, st));
    sketch_shapes(e.plan, d + 1, dt, &e.rows_ntiles, &e.rows_ngroups, &e.rows_cpg, &e.col_ngroups, &e.col_cpg);
    if (e.rows_ntiles == 0 || e.col_ngroups == 0) { set_error("grouped batch: unsupported sketch shape"); return SK_EINVAL; }
    new_plans.push_back(n);
    *out = &e;
    return SK_OK;
  };

  // admission of job q into slot `slot`: buffers, descriptor, upload
  auto admit = [&](int q, int slot) -> sk_status {
    const sk_op* op = A[q / nrhs];
    const int64_t n = op->n;
    PlanEntry* pe = nullptr;
    SK_TRY(plan_for(n, &pe));
    const int64_t ldb = ((n + 7) / 8) * 8;
    const int vec_guess = (op->kind == OP_STENCIL5 && n < (1ll << 31)) ? 1 : 0;
    const int nblk = basis_grid(n, vec_guess ? 4 : 1);
    VecLayout v;
    size_t off = 0;
    v.B = off; off += r256((size_t)ldb * (d + 1) * dtype_size(dt));
    v.r = off; off += r256((size_t)n * sizeof(double));
    v.M = off; if (dt == SK_F64) off += r256((size_t)n * sizeof(double));
    v.bpart = off; off += r256((size_t)nblk * (kMaxK + 1) * sizeof(double));
    v.vpart = off; off += r256((size_t)vec_grid(n) * sizeof(double));
    v.rows_part = off; off += r256((size_t)pe->rows_ngroups * (d + 1) * s * sizeof(double));
    v.col_part = off; off += r256((size_t)pe->col_ngroups * s * sizeof(double));
    v.total = off;
    unsigned char* mem = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&mem, v.total, st);
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_error("grouped batch: cudaMallocAsync(%zu bytes) failed: %s", v.total, cudaGetErrorString(e));
      return SK_ENOMEM;
    }
    double* sl = slab + (int64_t)slot * L.total;
    int* ints = reinterpret_cast<int*>(sl + L.ints);
    GJob& J = H.jobs[slot];
    std::memset(&J, 0, sizeof(J));
    BasisParams& bp = J.bp;
    bp.n = n;
    bp.d = d;
    bp.k = k;
    bp.passes = o.cgs_passes;
    bp.dtype = dt;
    bp.B = mem + v.B;
    bp.ldb = ldb;
    bp.h1 = sl + L.h1;
    bp.h2 = sl + L.h2;
    bp.nu = sl + L.nu;
    bp.mn2 = sl + L.mn2;
    bp.Hbar = sl + L.Hbar;
    bp.M = dt == SK_F64 ? reinterpret_cast<double*>(mem + v.M) : nullptr;
    bp.partial = reinterpret_cast<double*>(mem + v.bpart);
    bp.coef = sl + L.coef;
    bp.counters = reinterpret_cast<unsigned*>(ints + 2);
    bp.stop = ints;
    bp.nanflag = ints + 1;
    bp.r = reinterpret_cast<double*>(mem + v.r);
    bp.rho2 = sl + L.rho2;
    bp.bd = o.breakdown;
    bp.kind = SK_BASIS_ARNOLDI;
    J.vec = basis_vector_path(op, ldb, bp.B) ? (op->nx % 4 == 0 ? 1 : 2) : 0;
    bp.nblk = basis_grid(n, J.vec ? 4 : 1);
    bp.nblk_cap = bp.nblk;
    make_view(op, &J.Ad);
    if (dt != SK_F64) SK_TRY(make_view(op, &J.Af, st));
    J.vgrid = vec_grid(n);
    const double* xq = x[q];
    J.uvec = (n % 4 == 0 && ldb % 8 == 0 && ((uintptr_t)bp.B % 16) == 0 && ((uintptr_t)xq % 32) == 0) ? 1 : 0;
    J.ugrid = update_grid(n, J.uvec ? 4 : 1);
    J.b = b[q];
    J.x = x[q];
    J.vpart = reinterpret_cast<double*>(mem + v.vpart);
    J.vcnt = reinterpret_cast<unsigned*>(ints + 10);
    J.bn2 = sl + L.rho2 + 1;
    J.rowptr = pe->plan.rowptr;
    J.entries = pe->plan.entries;
    J.nchunks = pe->plan.nchunks;
    J.rows_ntiles = pe->rows_ntiles;
    J.rows_ngroups = pe->rows_ngroups;
    J.rows_cpg = pe->rows_cpg;
    J.col_ngroups = pe->col_ngroups;
    J.col_cpg = pe->col_cpg;
    J.rows_part = reinterpret_cast<double*>(mem + v.rows_part);
    J.col_part = reinterpret_cast<double*>(mem + v.col_part);
    J.g = sl + L.g;
    J.SB = sl + L.SB;
    J.y = sl + L.y;
    J.out = sl + L.out;
    if (J.bp.nblk != nblk) {  // the map and the partial buffer follow the vector path actually taken
      cudaFreeAsync(mem, st);
      set_error("grouped batch: inconsistent basis shape");
      return SK_EINVAL;
    }
    SK_CUDA(cudaMemcpyAsync(d_jobs + slot, &J, sizeof(GJob), cudaMemcpyHostToDevice, st));
    SlotState& S = slots[slot];
    S = SlotState();
    S.job = q;
    S.mem = mem;
    S.t0 = std::chrono::steady_clock::now();
    return SK_OK;
  };

  // ---- the loop: admit, initial residuals, cycles -----------------------------
  std::vector<int> free_slots;
  for (int i = nslots - 1; i >= 0; --i) free_slots.push_back(i);
  std::vector<int> active;
  size_t next = 0;
  long long resident = 0;
  sk_status first_err = SK_OK;
  std::string first_msg;
  long long total_launches = 0, sum_cycles = 0, sum_matvecs = 0;
  double relmax = 0, kmax_all = 0;
  float phase_sum[5] = {0, 0, 0, 0, 0};
  const int npanels = (d + kQrNb - 1) / kQrNb;
  const long long cycle_launches = 2 + 1 + (1 + (long long)d * (o.cgs_passes + 1)) + 2 + 1 + 1 + 2 * npanels + 1 + 1 + 1 + 1;

  auto finish = [&](int slot, sk_status r) {
    SlotState& S = slots[slot];
    const int q = S.job;
    if (per_job) per_job[q] = r;
    if (job_info) {
      sk_info& ji = job_info[q];
      std::memset(&ji, 0, sizeof(ji));
      ji.cycles = S.cycles;
      ji.matvecs = S.cycles * (d + 1) + 1;
      ji.d_used = S.cycles > 0 ? (S.stop < d ? S.stop : d) : 0;
      ji.width = S.width;
      ji.relres = S.relres;
      ji.rhat_est = S.rhat;
      ji.kappa_T_max = S.kmax;
      for (int p = 0; p < 5; ++p) ji.ms[p] = S.ms[p];
      ji.ms[5] = (float)std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - S.t0).count();
      ji.launches = S.launches;
    }
    if (r != SK_OK && first_err == SK_OK) {
      first_err = r;
      first_msg = sk_last_error();
    }
    sum_cycles += S.cycles;
    sum_matvecs += S.cycles * (d + 1) + 1;
    if (S.relres > relmax) relmax = S.relres;
    if (S.kmax > kmax_all) kmax_all = S.kmax;
    cudaFreeAsync(S.mem, st);
    S.mem = nullptr;
    S.job = -1;
    resident -= job_n(q);
    free_slots.push_back(slot);
  };
  auto fail_all = [&](sk_status r) {
    // a CUDA or allocation failure: every unfinished job reports it
    const std::string msg = sk_last_error();
    for (int slot : active) {
      set_error("%s", msg.c_str());
      finish(slot, r);
    }
    active.clear();
    for (; next < (size_t)njobs; ++next) {
      if (per_job) per_job[order[next]] = r;
      if (job_info) std::memset(&job_info[order[next]], 0, sizeof(sk_info));
    }
    set_error("%s", msg.c_str());
    if (first_err == SK_OK) { first_err = r; first_msg = msg; }
    return r;
  };

  Maps mp{};
  std::vector<int> uploaded;
  while (next < (size_t)njobs || !active.empty()) {
    // admit, largest first, within the element budget
    std::vector<int> fresh;
    new_plans.clear();
    while (next < (size_t)njobs && !free_slots.empty()) {
      const int q = order[next];
      const int64_t n = job_n(q);
      if ((!active.empty() || !fresh.empty()) && resident + n > cap) break;
      const int slot = free_slots.back();
      const sk_status as = admit(q, slot);
      if (as == SK_ENOMEM && (!active.empty() || !fresh.empty())) break;  // wait for resident jobs to leave
      if (as != SK_OK) {
        for (int f : fresh) active.push_back(f);
        return fail_all(as);
      }
      free_slots.pop_back();
      resident += n;
      fresh.push_back(slot);
      ++next;
    }
    if (!fresh.empty()) {
      // ||b||^2 and r = b - A x0 of the new jobs (as sgmres_solve before its first cycle)
      sk_status rs = upload(fresh, &mp);
      if (rs == SK_OK) rs = enqueue_vec_grouped(GV_NORM_B, d_jobs, H.d_map + mp.vec, (int)(mp.upd - mp.vec), dt, d, st);
      if (rs == SK_OK) rs = enqueue_vec_grouped(GV_RESIDUAL, d_jobs, H.d_map + mp.vec, (int)(mp.upd - mp.vec), dt, d, st);
      if (rs == SK_OK) rs = collect((int)fresh.size());
      for (size_t i = 0; rs == SK_OK && i < new_plans.size(); ++i) {
        const cudaError_t ce = cudaMemcpyAsync(H.pstat + i, H.plans[new_plans[i]].plan.d_status, sizeof(int),
                                               cudaMemcpyDeviceToHost, st);
        if (ce != cudaSuccess) rs = cuda_fail(ce, "cudaMemcpyAsync");
      }
      if (rs == SK_OK) {
        const cudaError_t ce = cudaStreamSynchronize(st);
        if (ce != cudaSuccess) rs = cuda_fail(ce, "cudaStreamSynchronize");
      }
      uploaded = fresh;
      if (rs != SK_OK) {
        for (int f : fresh) active.push_back(f);
        return fail_all(rs);
      }
      total_launches += 3;
      std::vector<int64_t> bad_n;
      for (size_t i = 0; i < new_plans.size(); ++i)
        if (H.pstat[i] != 0) bad_n.push_back(new_plans[i]);
      for (size_t t = 0; t < fresh.size(); ++t) {
        const int slot = fresh[t];
        SlotState& S = slots[slot];
        const int q = S.job;
        S.launches = 3;
        const double* rr = H.res + kResStride * t;
        const double bn2 = rr[6], rho2 = rr[0];
        if (std::find(bad_n.begin(), bad_n.end(), job_n(q)) != bad_n.end()) {
          set_error("sparse sign hash: no distinct row within 16 attempts (s=%d too small for zeta=%d)", s, o.zeta);
          finish(slot, SK_EHASH);
          continue;
        }
        if (!std::isfinite(bn2) || !std::isfinite(rho2)) {
          set_error("NaN/Inf in b or x");
          finish(slot, SK_ENAN);
          continue;
        }
        S.bnorm = std::sqrt(bn2);
        S.relres = S.bnorm > 0 ? std::sqrt(rho2) / S.bnorm : 0.0;
        if (S.bnorm == 0) {
          cudaMemsetAsync(x[q], 0, sizeof(double) * job_n(q), st);
          S.relres = 0;
          finish(slot, SK_OK);
          continue;
        }
        if (S.relres <= tol) {
          finish(slot, SK_OK);
          continue;
        }
        active.push_back(slot);
      }
    }
    if (active.empty()) continue;

    // one restart cycle of every active job
    sk_status rs = SK_OK;
    if (uploaded != active) {
      rs = upload(active, &mp);
      uploaded = active;
    }
    const int nj = (int)active.size();
    auto ev = [&](int i) { if (rs == SK_OK) { const cudaError_t ce = cudaEventRecord(H.ev[i], st); if (ce != cudaSuccess) rs = cuda_fail(ce, "cudaEventRecord"); } };
    ev(0);
    if (rs == SK_OK) rs = enqueue_sketch_col_grouped(d_jobs, H.d_map + mp.col, (int)(mp.end - mp.col), d_ids, nj, s, o.zeta, st);
    ev(1);
    if (rs == SK_OK) {
      int blocks = (int)(((int64_t)(d + 1) * d + 255) / 256);
      if (blocks > 64) blocks = 64;
      g_init_kernel<<<dim3(blocks, nj), 256, 0, st>>>(slab + L.Hbar, reinterpret_cast<int*>(slab + L.ints), d, js);
      const cudaError_t ce = cudaGetLastError();
      if (ce != cudaSuccess) rs = cuda_fail(ce, "g_init_kernel");
    }
    if (rs == SK_OK) rs = enqueue_basis_grouped(d_jobs, H.d_map + mp.basis, (int)(mp.vec - mp.basis), dt, k, o.cgs_passes, d, st);
    ev(2);
    if (rs == SK_OK)
      rs = enqueue_sketch_rows_grouped(d_jobs, H.d_map + mp.rows, (int)(mp.col - mp.rows), d_ids, nj, dt, d + 1, s,
                                       o.zeta, st);
    ev(3);
    if (rs == SK_OK)
      rs = enqueue_hbar_product(slab + L.SB, slab + L.Hbar, s, d, k, reinterpret_cast<const int*>(slab + L.ints),
                                slab + L.Aug, st, js, nj);
    if (rs == SK_OK) {
      g_copy_kernel<<<dim3(1, nj), 256, 0, st>>>(slab + L.g, slab + L.Aug + (int64_t)d * s, s, js);
      const cudaError_t ce = cudaGetLastError();
      if (ce != cudaSuccess) rs = cuda_fail(ce, "g_copy_kernel");
    }
    if (rs == SK_OK) rs = enqueue_qr(slab + L.Aug, s, d, d + 1, slab + L.rdiag, slab + L.tau, slab + L.Tws, st, js, nj);
    if (rs == SK_OK)
      rs = enqueue_ls_solve(slab + L.Aug, slab + L.rdiag, s, d, o.stab_tol, slab + L.y, slab + L.out + 1, st, js, nj);
    ev(4);
    if (rs == SK_OK) rs = enqueue_vec_grouped(GV_UPDATE, d_jobs, H.d_map + mp.upd, (int)(mp.rows - mp.upd), dt, d, st);
    ev(5);
    if (rs == SK_OK) rs = enqueue_vec_grouped(GV_RESIDUAL, d_jobs, H.d_map + mp.vec, (int)(mp.upd - mp.vec), dt, d, st);
    ev(6);
    if (rs == SK_OK) rs = collect(nj);
    if (rs == SK_OK) {
      const cudaError_t ce = cudaStreamSynchronize(st);
      if (ce != cudaSuccess) rs = cuda_fail(ce, "cudaStreamSynchronize");
    }
    if (rs != SK_OK) return fail_all(rs);
    total_launches += cycle_launches;
    float ph[5] = {0, 0, 0, 0, 0};
    {
      float t;
      if (cudaEventElapsedTime(&t, H.ev[5], H.ev[6]) == cudaSuccess) ph[0] = t;
      if (cudaEventElapsedTime(&t, H.ev[1], H.ev[2]) == cudaSuccess) ph[1] = t;
      if (cudaEventElapsedTime(&t, H.ev[0], H.ev[1]) == cudaSuccess) ph[2] = t;
      if (cudaEventElapsedTime(&t, H.ev[2], H.ev[3]) == cudaSuccess) ph[2] += t;
      if (cudaEventElapsedTime(&t, H.ev[3], H.ev[4]) == cudaSuccess) ph[3] = t;
      if (cudaEventElapsedTime(&t, H.ev[4], H.ev[5]) == cudaSuccess) ph[4] = t;
    }
    for (int p = 0; p < 5; ++p) phase_sum[p] += ph[p];
    std::vector<int> keep;
    for (int t = 0; t < nj; ++t) {
      const int slot = active[t];
      SlotState& S = slots[slot];
      const double* rr = H.res + kResStride * t;
      ++S.cycles;
      S.launches += cycle_launches;
      for (int p = 0; p < 5; ++p) S.ms[p] += ph[p];
      const double rho2 = rr[0];
      S.rhat = rr[1];
      const double kap = rr[2];
      S.width = (int)rr[3];
      S.stop = (int)rr[4];
      if (kap > S.kmax) S.kmax = kap;
      if (!std::isfinite(rho2)) {
        set_error("NaN/Inf in the residual");
        finish(slot, SK_ENAN);
        continue;
      }
      S.relres = std::sqrt(rho2) / S.bnorm;
      if (S.relres <= tol) {
        finish(slot, SK_OK);
        continue;
      }
      if (S.width == 0) {
        set_error("kappa(T) above stab_tol already for one column");
        finish(slot, SK_EILLCOND);
        continue;
      }
      if (S.cycles >= o.maxit) {
        set_error("no convergence to tol=%g in %d cycles (relres %g)", tol, S.cycles, S.relres);
        finish(slot, SK_ENOCONV);
        continue;
      }
      keep.push_back(slot);
    }
    active.swap(keep);
  }
  SK_CUDA(cudaStreamSynchronize(st));
  const double wall_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->cycles = (int)(sum_cycles > 2147483647 ? 2147483647 : sum_cycles);
    info->matvecs = (int)(sum_matvecs > 2147483647 ? 2147483647 : sum_matvecs);
    info->relres = relmax;
    info->kappa_T_max = kmax_all;
    for (int p = 0; p < 5; ++p) info->ms[p] = phase_sum[p];
    info->ms[5] = (float)wall_ms;
    info->launches = total_launches;
  }
  if (first_err != SK_OK) set_error("%s", first_msg.c_str());
  return first_err;
}

}  // namespace sk
