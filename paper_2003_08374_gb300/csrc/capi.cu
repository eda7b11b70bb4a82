// capi.cu -- C-ABI of libmdbs (include/mdbs.h): device arena, field transfer and
// the host-side orchestration of the time step of section 3.2.  Every numerical
// step runs in the kernels of step_kernels.cu and pressure.cu.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <string>
#include <utility>
#include <algorithm>
#include <vector>

#include <nvtx3/nvToolsExt.h>  // header-only: the ranges cost nothing unless a profiler attaches

#include "../../include/mdbs.h"
#include "mdbs_internal.cuh"

using namespace mdbs;

namespace mdbs {

const char* const kKernelNames[K_COUNT] = {
    "alpha_flux", "alpha_lo", "alpha_limit", "alpha_update", "finalize", "properties", "normals",
    "curvature", "momentum_assemble", "jacobi", "hbya", "correct", "boundary", "field_stats", "cfl",
    "static_geometry", "pressure_assemble", "diag", "convert", "coarsen", "smooth_fine", "smooth_coarse",
    "zero", "restrict_fine", "restrict_coarse", "prolong_fine", "prolong_coarse", "cg_resid0",
    "cg_spmv_dot", "cg_update_xr", "cg_dots", "cg_update_d", "tail_vcycle", "coarse_coop", "edge_viscosity"};

// Per-simulation launch counter and optional event timer.
struct Profiler {
  bool on = false;
  int only = -1;  // time only this kernel id (-1: all)
  long long launches = 0;
  std::vector<cudaEvent_t> pool;
  size_t next = 0;
  struct Rec {
    int id;
    size_t e0, e1;
  };
  std::vector<Rec> recs;
  int open_id = -1;
  size_t open_ev = 0;
  double ms[K_COUNT] = {};
  long long count[K_COUNT] = {};

  size_t event(cudaStream_t s) {
    if (next == pool.size()) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return (size_t)-1;
      pool.push_back(e);
    }
    cudaEventRecord(pool[next], s);
    return next++;
  }
  void resolve() {
    if (recs.empty()) return;
    cudaEventSynchronize(pool[recs.back().e1]);
    for (const Rec& r : recs) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, pool[r.e0], pool[r.e1]) == cudaSuccess) {
        ms[r.id] += t;
        count[r.id] += 1;
      }
    }
    recs.clear();
    next = 0;
  }
  void reset() {
    for (int i = 0; i < K_COUNT; i++) {
      ms[i] = 0.0;
      count[i] = 0;
    }
  }
  ~Profiler() {
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
  }
};

static thread_local Profiler* g_active = nullptr;

void prof_begin(int id, cudaStream_t s) {
  Profiler* p = g_active;
  if (!p) return;
  p->launches++;
  if (!p->on || (p->only >= 0 && p->only != id)) return;
  p->open_id = id;
  p->open_ev = p->event(s);
}

long long launch_count() { return g_active ? g_active->launches : 0; }

static thread_local cudaError_t g_launch_error = cudaSuccess;
void set_launch_error(cudaError_t e) {
  if (g_launch_error == cudaSuccess) g_launch_error = e;
}
cudaError_t take_launch_error() {
  const cudaError_t e = g_launch_error;
  g_launch_error = cudaSuccess;
  return e;
}

void prof_end(int id, cudaStream_t s) {
  Profiler* p = g_active;
  if (!p || !p->on || p->open_id != id || p->open_ev == (size_t)-1) return;
  size_t e1 = p->event(s);
  if (e1 != (size_t)-1) p->recs.push_back({id, p->open_ev, e1});
  p->open_id = -1;
}

}  // namespace mdbs

// A batch plan plus the step captured from it as one CUDA graph (CG loops as
// conditional WHILE nodes).
struct Exec {
  BatchPlan plan{};
  bool planned = false;
  cudaStream_t cap_stream = nullptr, body_stream = nullptr;
  cudaStream_t side_stream = nullptr;               // the pressure operator's branch of the step graph
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;  // its fork from and join to the main branch
  cudaGraphExec_t graph = nullptr;
  long long static_launches = 0;  // kernels outside the CG loops per step
  long long body_launches = 0;    // kernels per CG iteration
  double* host_flag = nullptr;    // pinned
};

struct mdbs_sim {
  Profiler prof;
  Prm P;
  Fld F;
  mdbs_options opt;
  int precision;
  cudaStream_t stream;
  void* arena;
  DevBlock arena_mem;  // owner record of the arena (allocator hook)
  size_t arena_bytes;
  PressureSolver* ps;
  double* partials;   // 4 channels of pcap
  long long pcap;
  double* scal;       // device step scalars (kSlot* in mdbs_internal.cuh)
  double* host_scal;  // pinned copy of scal
  mdbs_stats st;
  double alpha_lo_seen = 0.0, alpha_hi_seen = 1.0;  // extremes of alpha this simulation's steps produced
  bool fields_set;
  bool in_batch;
  std::string err;
  mdbs_tuning tun;    // schedule of the multigrid kernels
  Exec ex;            // batch of one: this simulation alone
};

struct mdbs_batch {
  Profiler prof;
  std::vector<mdbs_sim*> sims;
  mdbs_options opt;
  cudaStream_t stream;
  mdbs_tuning tun;
  Exec ex;
  double* gather;       // device: ndom x kNumSlots step scalars
  double* host_gather;  // pinned
  std::string err;
};

static thread_local std::string g_create_error;

// ---------------------------------------------------------------- device memory hook
static mdbs_alloc_fn g_alloc = nullptr;
static mdbs_free_fn g_free = nullptr;
static void* g_alloc_ctx = nullptr;

namespace mdbs {
cudaError_t dev_block_alloc(DevBlock* b, size_t bytes) {
  *b = DevBlock{};
  if (g_alloc) {
    void* p = g_alloc(bytes, g_alloc_ctx);
    if (!p) return cudaErrorMemoryAllocation;
    if ((uintptr_t)p & 255) {  // the arena layout and the TMA descriptors need 256-byte alignment
      g_free(p, g_alloc_ctx);
      return cudaErrorInvalidValue;
    }
    b->ptr = p;
    b->free_fn = g_free;
    b->ctx = g_alloc_ctx;
    return cudaSuccess;
  }
  return cudaMalloc(&b->ptr, bytes);
}

void dev_block_free(DevBlock* b) {
  if (!b->ptr) return;
  if (b->free_fn)
    b->free_fn(b->ptr, b->ctx);
  else
    cudaFree(b->ptr);
  *b = DevBlock{};
}
}  // namespace mdbs

extern "C" int mdbs_set_allocator(mdbs_alloc_fn alloc, mdbs_free_fn free_fn, void* ctx) {
  if ((alloc == nullptr) != (free_fn == nullptr)) return MDBS_ERR_ARG;
  g_alloc = alloc;
  g_free = free_fn;
  g_alloc_ctx = alloc ? ctx : nullptr;
  return MDBS_OK;
}

namespace {

struct Activate {
  Profiler* prev;
  explicit Activate(mdbs_sim* s) : prev(g_active) { g_active = &s->prof; }
  explicit Activate(mdbs_batch* b) : prev(g_active) { g_active = &b->prof; }
  ~Activate() {
    if (g_active && g_active->on) g_active->resolve();
    g_active = prev;
  }
};

size_t a256(size_t b) { return (b + 255) & ~(size_t)255; }

struct Layout {
  long long cells, nf[3];
  long long n[3];
  int dim;
};

Layout layout_of(const mdbs_grid* g) {
  Layout L;
  L.dim = g->nz == 1 ? 2 : 3;
  L.cells = (long long)g->nx * g->ny * g->nz;
  L.n[0] = g->nx;
  L.n[1] = g->ny;
  L.n[2] = g->nz;
  L.nf[0] = (long long)(g->nx + 1) * g->ny * g->nz;
  L.nf[1] = (long long)g->nx * (g->ny + 1) * g->nz;
  L.nf[2] = (long long)g->nx * g->ny * (g->nz + 1);
  return L;
}


// carve the arena; base == nullptr only measures
size_t carve(mdbs_sim* s, const Layout& L, char* base) {
  size_t off = 0;
  auto take = [&](size_t bytes) -> char* {
    char* p = base ? base + off : nullptr;
    off += a256(bytes);
    return p;
  };
  auto cd = [&]() { return (double*)take(L.cells * 8); };
  Fld F{};
  F.phi = cd();
  F.k0 = cd();
  F.is_free = (uint8_t*)take(L.cells);
  for (int e = 0; e < 3; e++) F.nw[e] = cd();
  F.iphi2 = cd();
  F.iphiV = cd();
  F.alpha = cd();
  F.p = cd();
  F.Ml = cd();
  F.Mg = cd();
  F.fw = cd();
  F.pc = cd();
  F.cf = cd();
  F.rho = cd();
  F.mu = cd();
  F.drag = cd();
  for (int e = 0; e < 3; e++) F.m[e] = cd();
  F.kappa = cd();
  for (int q = 0; q < 3; q++) {  // edge viscosities of the axis pairs (0,1), (0,2), (1,2)
    const int a = q == 2 ? 1 : 0, b = q == 0 ? 1 : 2;
    const bool has = b < L.dim;
    long long ext[3] = {L.n[0], L.n[1], L.n[2]};
    ext[a] += 1;
    ext[b] += 1;
    F.muE[q] = (double*)take((has ? ext[0] * ext[1] * ext[2] : 1) * 8);
  }
  F.aL = cd();
  F.Rp = cd();
  F.Rm = cd();
  for (int e = 0; e < 3; e++) F.T[e] = cd();
  F.Dd = cd();
  F.diag = cd();
  F.dinv = cd();
  F.b = cd();
  for (int d = 0; d < 3; d++) {
    const long long nf = (d < L.dim) ? L.nf[d] : 1;
    auto fd = [&]() { return (double*)take(nf * 8); };
    F.u[d] = fd();
    F.FLO[d] = fd();
    F.AF[d] = fd();
    F.aP[d] = fd();
    F.anb[d] = (double*)take(6 * nf * 8);
    F.rhs0[d] = fd();
    F.B[d] = fd();
    F.hbya[d] = fd();
    F.utmp[d] = fd();
    F.iphif[d] = fd();
    F.gphi[d] = (double*)take(3 * nf * 8);
  }
  const long long faces = L.nf[0] + L.nf[1] + (L.dim == 3 ? L.nf[2] : 0);
  const long long pcap = (std::max(L.cells, faces) + kBlock * kRepBig - 1) / (kBlock * kRepBig);
  double* partials = (double*)take(4 * pcap * 8);
  double* scal = (double*)take(kNumSlots * 8);
  if (s) {
    s->F = F;
    s->partials = partials;
    s->pcap = pcap;
    s->scal = scal;
  }
  return off;
}

int fail(mdbs_sim* s, int code, const std::string& msg) {
  if (s)
    s->err = msg;
  else
    g_create_error = msg;
  return code;
}

int cuda_fail(mdbs_sim* s, cudaError_t e, const char* where) {
  return fail(s, MDBS_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                   \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return cuda_fail(s, e_, #call); \
  } while (0)

// statistics of one simulation from a host copy of its scalars
int stats_from(mdbs_sim* s, const double* h) {
  s->st.mass = h[kSlotMass];
  s->st.alpha_min = h[kSlotAmin];
  s->st.alpha_max = h[kSlotAmax];
  s->st.boundary_in = h[kSlotInflow];
  s->st.dt = h[kSlotDt];
  s->st.time = h[kSlotTime];
  for (int c = 0; c < s->opt.n_corr && c < 8; c++) {
    s->st.cg_iters[c] = (int32_t)h[kSlotIters + c];
    s->st.cg_resid[c] = h[kSlotResid + c];
  }
  s->st.cg_iters_total = (int64_t)h[kSlotItersTotal];
  s->st.not_converged = (int32_t)h[kSlotNotConverged];
  if (h[kSlotBad] != 0.0) return fail(s, MDBS_ERR_DIVERGED, "non-finite alpha or pressure");
  s->alpha_lo_seen = std::min(s->alpha_lo_seen, s->st.alpha_min);
  s->alpha_hi_seen = std::max(s->alpha_hi_seen, s->st.alpha_max);
  return MDBS_OK;
}

// MDBS_ERR_NOT_CONVERGED when pressure solves of the steps just taken stopped at max_cg
int convergence_check(mdbs_sim* s, double not_converged_before) {
  const double nc = s->host_scal[kSlotNotConverged] - not_converged_before;
  if (nc <= 0.0) return MDBS_OK;
  return fail(s, MDBS_ERR_NOT_CONVERGED,
              std::to_string((long long)nc) + " pressure solve(s) stopped at max_cg before the tolerance; the steps "
              "were taken (last relative residual " + std::to_string(s->st.cg_resid[0]) + " ... " +
              std::to_string(s->st.cg_resid[std::max(0, std::min(7, s->opt.n_corr - 1))]) + ")");
}

// copies the device scalars and the statistics they hold; checks health
int refresh_stats(mdbs_sim* s) {
  CK(cudaMemcpyAsync(s->host_scal, s->scal, kNumSlots * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  s->st.kernel_launches = s->prof.launches;
  return stats_from(s, s->host_scal);
}

StepDom step_view(const mdbs_sim* s) {
  StepDom d{};
  d.P = s->P;
  d.F = s->F;
  d.scal = s->scal;
  d.partials = s->partials;
  d.pcap = s->pcap;
  return d;
}

// Enqueues one time step (section 3.2) of every domain of the plan on st.
// capture: st is capturing a graph.  Returns a CUDA error.
// NVTX range of one step phase (host-side marks around the phase's launches: in eager
// steps they bracket the kernels; under graph capture they mark the capture)
struct Phase {
  explicit Phase(const char* name) { nvtxRangePushA(name); }
  ~Phase() { nvtxRangePop(); }
};

cudaError_t record_step(Exec& ex, const mdbs_options& opt, cudaStream_t st, bool capture) {
  const BatchPlan& B = ex.plan;
  Phase step("mdbs step");
  {
    // 1. saturation (Eq. 15) by flux-corrected transport
    Phase ph("saturation (Eq. 15, FCT)");
    launch_alpha_step(B, st);
  }
  {
    // 3. properties at alpha^{k+1}
    Phase ph("properties (Eqs. 41-45)");
    launch_properties(B, st);
  }
  {
    // 4. momentum predictor (Eq. 50) from u^k and p^k.  The pressure operator of
    // Eq. 53 depends on a_P alone: in the step graph it is assembled, with its
    // multigrid hierarchy, on a side branch while the Jacobi sweeps run, and joins
    // before the first pressure solve (eager steps run it in line).
    Phase ph("momentum predictor (Eq. 50)");
    launch_momentum_assemble(B, st);
    cudaStream_t ms = st;
    if (capture) {
      cudaError_t e = cudaEventRecord(ex.ev_fork, st);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(ex.side_stream, ex.ev_fork, 0);
      if (e != cudaSuccess) return e;
      ms = ex.side_stream;
    }
    launch_pressure_matrix(B, opt.mg_coarse_sweeps, ms);
    if (capture) {
      const cudaError_t e = cudaEventRecord(ex.ev_join, ms);
      if (e != cudaSuccess) return e;
    }
    launch_jacobi_sweeps(B, opt.mom_sweeps, st);
  }
  // 5. PISO correctors (Eqs. 51-53)
  for (int c = 0; c < opt.n_corr; c++) {
    Phase ph("PISO corrector (Eqs. 51-53)");
    launch_hbya(B, st);
    launch_pressure_rhs(B, st);
    if (capture && c == 0) {
      const cudaError_t e = cudaStreamWaitEvent(st, ex.ev_join, 0);
      if (e != cudaSuccess) return e;
    }
    cudaError_t e = pressure_solve(B, opt.p_tol, opt.max_cg, opt.mg_nu1, opt.mg_nu2, opt.mg_coarse_sweeps, c,
                                   capture, st, ex.body_stream, ex.host_flag, &ex.body_launches);
    if (e != cudaSuccess) return e;
    launch_correct(B, st);
  }
  {
    // 6. time and next time step; statistics and health sentinel
    Phase ph("time step and health");
    launch_time_advance(B, st);
    launch_field_stats(B, st);
  }
  const cudaError_t le = take_launch_error();
  return le != cudaSuccess ? le : cudaGetLastError();
}

cudaError_t exec_setup(Exec& ex, const StepDom* sd, const CgDom* cg, int ndom, int flexible, const mdbs_tuning& t) {
  cudaError_t e =
      plan_create(sd, cg, ndom, flexible, t.smooth_rows, t.snake, t.sweep_kz, t.tail_ctas, t.coarse_coop,
                  t.vec_sweeps, &ex.plan);
  if (e != cudaSuccess) return e;
  ex.planned = true;
  if (!ex.cap_stream) e = cudaStreamCreateWithFlags(&ex.cap_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess && !ex.body_stream) e = cudaStreamCreateWithFlags(&ex.body_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess && !ex.side_stream) e = cudaStreamCreateWithFlags(&ex.side_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess && !ex.ev_fork) e = cudaEventCreateWithFlags(&ex.ev_fork, cudaEventDisableTiming);
  if (e == cudaSuccess && !ex.ev_join) e = cudaEventCreateWithFlags(&ex.ev_join, cudaEventDisableTiming);
  if (e == cudaSuccess && !ex.host_flag) e = cudaMallocHost(&ex.host_flag, sizeof(double));
  return e;
}

void exec_destroy(Exec& ex) {
  if (ex.graph) cudaGraphExecDestroy(ex.graph);
  if (ex.planned) plan_destroy(&ex.plan);
  if (ex.cap_stream) cudaStreamDestroy(ex.cap_stream);
  if (ex.body_stream) cudaStreamDestroy(ex.body_stream);
  if (ex.side_stream) cudaStreamDestroy(ex.side_stream);
  if (ex.ev_fork) cudaEventDestroy(ex.ev_fork);
  if (ex.ev_join) cudaEventDestroy(ex.ev_join);
  if (ex.host_flag) cudaFreeHost(ex.host_flag);
  ex = Exec{};
}

// captures the step graph once (lazily) and counts its kernels
cudaError_t ensure_graph(Exec& ex, const mdbs_options& opt, Profiler& prof) {
  if (ex.graph) return cudaSuccess;
  const long long before = prof.launches;
  const bool was_on = prof.on;
  prof.on = false;
  cudaError_t e = cudaStreamBeginCapture(ex.cap_stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  cudaError_t rec = record_step(ex, opt, ex.cap_stream, true);
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(ex.cap_stream, &g);
  prof.on = was_on;
  const long long captured = prof.launches - before;
  prof.launches = before;
  if (rec != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return rec;
  }
  if (e != cudaSuccess) return e;
  e = cudaGraphInstantiate(&ex.graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    ex.graph = nullptr;
    return e;
  }
  ex.static_launches = captured - opt.n_corr * ex.body_launches;
  return cudaSuccess;
}

// n steps of the plan: eager when profiling (per-kernel events), else graph launches
cudaError_t exec_steps(Exec& ex, const mdbs_options& opt, Profiler& prof, cudaStream_t stream, int n) {
  if (prof.on) {
    for (int i = 0; i < n; i++) {
      cudaError_t e = record_step(ex, opt, stream, false);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  cudaError_t e = ensure_graph(ex, opt, prof);
  if (e != cudaSuccess) return e;
  for (int i = 0; i < n; i++) {
    e = cudaGraphLaunch(ex.graph, stream);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

const mdbs_tuning kDefaultTuning = {1, 4096, 0, 0, 1, 0, 0};

// whether a kernel of the plan reported a bounded wait that ran out (synchronous read)
bool plan_failed(const BatchPlan& B) {
  int h = 0;
  if (!B.err_flag) return false;
  if (cudaMemcpy(&h, B.err_flag, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return true;
  return h != 0;
}

bool valid_tuning(const mdbs_tuning* t) {
  return t && (t->smooth_rows == 1 || t->smooth_rows == 2 || t->smooth_rows == 4 || t->smooth_rows == 8) &&
         t->tail_cells >= 0 && t->tail_cells <= kTailCellsMax && (t->snake == 0 || t->snake == 1) &&
         (t->sweep_kz == 0 || t->sweep_kz == 4 || t->sweep_kz == 8 || t->sweep_kz == 16 || t->sweep_kz == 32) &&
         (t->tail_ctas == 1 || t->tail_ctas == 2 || t->tail_ctas == 4 || t->tail_ctas == 8) &&
         (t->coarse_coop == 0 || t->coarse_coop == 1) && (t->vec_sweeps == 0 || t->vec_sweeps == 1);
}

// (re)builds the batch-of-one plan of a simulation for its schedule
cudaError_t sim_exec_setup(mdbs_sim* s) {
  if (s->ex.graph) cudaGraphExecDestroy(s->ex.graph);
  s->ex.graph = nullptr;
  if (s->ex.planned) plan_destroy(&s->ex.plan);
  s->ex.planned = false;
  StepDom sd = step_view(s);
  CgDom cg;
  pressure_view(s->ps, s->F, s->tun.tail_cells, &cg);
  return exec_setup(s->ex, &sd, &cg, 1, s->precision != 0, s->tun);
}

cudaError_t batch_exec_setup(mdbs_batch* b) {
  if (b->ex.graph) cudaGraphExecDestroy(b->ex.graph);
  b->ex.graph = nullptr;
  if (b->ex.planned) plan_destroy(&b->ex.plan);
  b->ex.planned = false;
  const int n = (int)b->sims.size();
  std::vector<StepDom> sd(n);
  std::vector<CgDom> cg(n);
  for (int i = 0; i < n; i++) {
    sd[i] = step_view(b->sims[i]);
    pressure_view(b->sims[i]->ps, b->sims[i]->F, b->tun.tail_cells, &cg[i]);
  }
  return exec_setup(b->ex, sd.data(), cg.data(), n, b->sims[0]->precision != 0, b->tun);
}

// Device state of the simulations being tuned, copied aside so that every trial
// starts from it and the simulations end where they were.
struct Snapshot {
  struct Part {
    void* src;
    void* copy;
    size_t bytes;
  };
  std::vector<Part> parts;
  std::vector<mdbs_stats> st;
  std::vector<std::vector<double>> host_scal;
  ~Snapshot() {
    for (Part& p : parts)
      if (p.copy) cudaFree(p.copy);
  }
  cudaError_t take(const std::vector<mdbs_sim*>& sims, cudaStream_t stream) {
    for (mdbs_sim* s : sims) {
      void* pp;
      size_t pb;
      pressure_storage(s->ps, &pp, &pb);
      for (Part p : {Part{s->arena, nullptr, s->arena_bytes}, Part{pp, nullptr, pb}}) {
        cudaError_t e = cudaMalloc(&p.copy, p.bytes);
        if (e != cudaSuccess) return e;
        parts.push_back(p);
        e = cudaMemcpyAsync(p.copy, p.src, p.bytes, cudaMemcpyDeviceToDevice, stream);
        if (e != cudaSuccess) return e;
      }
      st.push_back(s->st);
      host_scal.emplace_back(s->host_scal, s->host_scal + kNumSlots);
    }
    return cudaStreamSynchronize(stream);
  }
  cudaError_t restore(cudaStream_t stream) const {
    for (const Part& p : parts) {
      cudaError_t e = cudaMemcpyAsync(p.src, p.copy, p.bytes, cudaMemcpyDeviceToDevice, stream);
      if (e != cudaSuccess) return e;
    }
    return cudaStreamSynchronize(stream);
  }
  void restore_host(const std::vector<mdbs_sim*>& sims) const {
    for (size_t i = 0; i < sims.size(); i++) {
      sims[i]->st = st[i];
      for (int k = 0; k < kNumSlots; k++) sims[i]->host_scal[k] = host_scal[i][k];
    }
  }
};

// Coordinate descent over the schedule (snake, then smooth_rows, then tail_cells):
// every trial restores the snapshot, rebuilds the plan, runs one untimed and
// `steps` timed graph steps.  setup(t) installs schedule t.
template <typename Setup>
int autotune_impl(const std::vector<mdbs_sim*>& sims, Exec& ex, const mdbs_options& opt, Profiler& prof,
                  cudaStream_t stream, mdbs_tuning& tun, Setup setup, int steps, double* trial_ms, int capacity,
                  int* ntrials, std::string& err, bool fp32_levels) {
  Snapshot snap;
  cudaError_t e = snap.take(sims, stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    err = std::string("autotune snapshot: ") + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? MDBS_ERR_OOM : MDBS_ERR_CUDA;
  }
  const bool was_on = prof.on;
  const long long launches = prof.launches;
  prof.on = false;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  cudaEventCreate(&ev0);
  cudaEventCreate(&ev1);
  int count = 0;
  auto trial = [&](const mdbs_tuning& t, double* ms) -> cudaError_t {
    cudaError_t r = setup(t);
    if (r == cudaSuccess) r = snap.restore(stream);
    if (r == cudaSuccess) r = exec_steps(ex, opt, prof, stream, 1);
    if (r == cudaSuccess) r = cudaEventRecord(ev0, stream);
    if (r == cudaSuccess) r = exec_steps(ex, opt, prof, stream, steps);
    if (r == cudaSuccess) r = cudaEventRecord(ev1, stream);
    if (r == cudaSuccess) r = cudaEventSynchronize(ev1);
    float f = 0.f;
    if (r == cudaSuccess) r = cudaEventElapsedTime(&f, ev0, ev1);
    *ms = (double)f / steps;
    if (r == cudaSuccess) {
      if (trial_ms && count < capacity) trial_ms[count] = *ms;
      count++;
    }
    return r;
  };
  mdbs_tuning best = tun;
  double best_ms = 0.0;
  e = trial(best, &best_ms);
  // axes in order; smooth_rows only matters for split half sweeps (sweep_kz == 0), and
  // fused sweeps only exist for FP32 levels
  const int snakes[] = {0, 1};
  const int kzs[] = {0, 4, 8, 16, 32};
  const int rows[] = {1, 2, 4, 8};
  const int coops[] = {0, 1};
  const int vecs[] = {0, 1};
  // (tail_cells, tail_ctas): larger tails want more CTAs
  // (1024: a 2-D grid's 32^2 level; the 64^2 fracture case measured 1.18 against 1.35 ms per
  // step with its whole V-cycle in one CTA)
  const int tails[][2] = {{0, 1}, {512, 1}, {1024, 1}, {4096, 1}, {4096, 4}, {32768, 4}, {32768, 8}, {262144, 8}};
  for (int axis = 0; axis < 6 && e == cudaSuccess; axis++) {
    if (axis == 2 && best.sweep_kz > 0 && fp32_levels) continue;
    if (axis == 1 && !fp32_levels) continue;
    const int nv = axis == 0 ? 2 : axis == 1 ? 5 : axis == 2 ? 4 : axis == 3 ? 2 : axis == 4 ? 8 : 2;
    const mdbs_tuning base = best;
    for (int v = 0; v < nv && e == cudaSuccess; v++) {
      mdbs_tuning t = base;
      if (axis == 0) t.snake = snakes[v];
      if (axis == 1) t.sweep_kz = kzs[v];
      if (axis == 2) t.smooth_rows = rows[v];
      if (axis == 3) t.coarse_coop = coops[v];
      if (axis == 4) {
        t.tail_cells = tails[v][0];
        t.tail_ctas = tails[v][1];
      }
      if (axis == 5) t.vec_sweeps = vecs[v];
      if (t.snake == base.snake && t.sweep_kz == base.sweep_kz && t.smooth_rows == base.smooth_rows &&
          t.tail_cells == base.tail_cells && t.tail_ctas == base.tail_ctas && t.coarse_coop == base.coarse_coop &&
          t.vec_sweeps == base.vec_sweeps)
        continue;
      double ms = 0.0;
      e = trial(t, &ms);
      if (e == cudaSuccess && ms < best_ms) {
        best = t;
        best_ms = ms;
      }
    }
  }
  if (e == cudaSuccess) e = setup(best);
  if (e == cudaSuccess) e = snap.restore(stream);
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
  snap.restore_host(sims);
  prof.on = was_on;
  prof.launches = launches;
  if (ntrials) *ntrials = count;
  if (e != cudaSuccess) {
    err = std::string("autotune: ") + cudaGetErrorString(e);
    return MDBS_ERR_CUDA;
  }
  tun = best;
  return MDBS_OK;
}

bool same_solver_options(const mdbs_options& a, const mdbs_options& b) {
  return a.n_corr == b.n_corr && a.mom_sweeps == b.mom_sweeps && a.p_tol == b.p_tol && a.max_cg == b.max_cg &&
         a.mg_nu1 == b.mg_nu1 && a.mg_nu2 == b.mg_nu2 && a.mg_coarse_sweeps == b.mg_coarse_sweeps &&
         (a.precision == 0) == (b.precision == 0);
}

}  // namespace

extern "C" {

size_t mdbs_bytes_required(const mdbs_grid* grid, int32_t precision) {
  if (!grid || grid->nx < 1 || grid->ny < 1 || grid->nz < 1) return 0;
  Layout L = layout_of(grid);
  int n[3] = {grid->nx, grid->ny, grid->nz};
  return carve(nullptr, L, nullptr) + pressure_bytes(n, precision < 0 || precision > 2 ? 1 : precision);
}

int mdbs_create(const mdbs_grid* grid, const double* porosity, const double* permeability,
                const mdbs_fluids* fl, double contact_angle_deg, const mdbs_closures* cl,
                const mdbs_options* op, mdbs_sim** out) {
  mdbs_sim* s = nullptr;
  if (!out) return fail(s, MDBS_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!grid || !porosity || !permeability || !fl || !cl || !op) return fail(s, MDBS_ERR_ARG, "NULL argument");
  if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1 || !(grid->h > 0.0))
    return fail(s, MDBS_ERR_ARG, "grid sizes must be >= 1 and h > 0");
  // kernels decode indices in 32 bits: every face array must stay below 2^31 entries
  if ((long long)(grid->nx + 1) * (grid->ny + 1) * (long long)(grid->nz + 1) >= (1ll << 31))
    return fail(s, MDBS_ERR_ARG, "grid too large (more than 2^31 faces per direction)");
  const long long cells = (long long)grid->nx * grid->ny * grid->nz;
  for (long long c = 0; c < cells; c++) {
    const double ph = porosity[c];
    if (!(ph > 0.0 && ph <= 1.0)) return fail(s, MDBS_ERR_ARG, "porosity must lie in (0, 1]");
    if (ph < 1.0 && !(permeability[c] > 0.0 && isfinite(permeability[c])))
      return fail(s, MDBS_ERR_ARG, "permeability must be > 0 where porosity < 1");
  }
  bool outlet = false;
  for (int i = 0; i < 6; i++) {
    if (op->bc[i] < 0 || op->bc[i] > 2) return fail(s, MDBS_ERR_ARG, "bc must be 0, 1 or 2");
    if (grid->nz == 1 && i >= 4) continue;
    outlet |= op->bc[i] == MDBS_BC_OUTLET;
  }
  if (!outlet) return fail(s, MDBS_ERR_ARG, "at least one side must be an outlet");
  if (op->n_corr < 1 || op->n_corr > 8 || op->mom_sweeps < 0 || op->max_cg < 1 || op->mg_nu1 < 0 ||
      op->mg_nu2 < 0 || op->mg_coarse_sweeps < 0 || op->precision < 0 || op->precision > 2 || !(op->dt > 0.0))
    return fail(s, MDBS_ERR_ARG, "invalid options");
  if (cl->kr_model < 0 || cl->kr_model > 1 || cl->pc_model < 0 || cl->pc_model > 1 ||
      cl->porous_density < 0 || cl->porous_density > 1)
    return fail(s, MDBS_ERR_ARG, "invalid closure model");

  s = new (std::nothrow) mdbs_sim();
  if (!s) return fail(nullptr, MDBS_ERR_OOM, "host allocation failed");
  s->tun = kDefaultTuning;
  Prm& P = s->P;
  P.n[0] = grid->nx;
  P.n[1] = grid->ny;
  P.n[2] = grid->nz;
  Layout L = layout_of(grid);
  P.dim = L.dim;
  P.dn0 = make_fastdiv((unsigned)grid->nx);
  P.dn1 = make_fastdiv((unsigned)grid->ny);
  P.dn0p = make_fastdiv((unsigned)grid->nx + 1);
  P.dn1p = make_fastdiv((unsigned)grid->ny + 1);
  P.cells = L.cells;
  for (int d = 0; d < 3; d++) P.nf[d] = L.nf[d];
  P.h = grid->h;
  P.A = grid->h * grid->h;
  P.V = grid->h * grid->h * grid->h;
  for (int i = 0; i < 6; i++) P.bc[i] = op->bc[i];
  P.inlet_u = op->inlet_u;
  P.inlet_alpha = op->inlet_alpha;
  P.rho_l = fl->rho_l;
  P.mu_l = fl->mu_l;
  P.rho_g = fl->rho_g;
  P.mu_g = fl->mu_g;
  P.sigma = fl->sigma;
  for (int e = 0; e < 3; e++) P.g[e] = fl->g[e];
  P.kr_model = cl->kr_model;
  P.pc_model = cl->pc_model;
  P.kr_m = cl->kr_m;
  P.a_l_irr = cl->a_l_irr;
  P.a_g_irr = cl->a_g_irr;
  P.pc0 = cl->pc0;
  P.pc_beta = cl->pc_beta;
  P.pc_m = cl->pc_m;
  P.a_pc_irr = cl->a_pc_irr;
  P.a_pc_max = cl->a_pc_max;
  P.pc_eps = cl->pc_eps;
  P.porous_density = cl->porous_density;
  const double th = contact_angle_deg * M_PI / 180.0;
  P.cos_t = cos(th);
  P.sin_t = sin(th);
  P.c_alpha = op->c_alpha;
  P.inv_h = 1.0 / grid->h;
  P.half_inv_h = 0.5 / grid->h;
  P.inv_mu_l = 1.0 / P.mu_l;
  P.inv_mu_g = 1.0 / P.mu_g;
  P.inv_ae_den = 1.0 / (1.0 - P.a_g_irr - P.a_l_irr);
  P.inv_s_den = 1.0 / (P.a_pc_max - P.a_pc_irr);
  P.reg_m = 1e-8 / grid->h;
  P.inv_h2 = 1.0 / (grid->h * grid->h);
  for (int d = 0; d < 3; d++) P.drho_g[d] = (P.rho_l - P.rho_g) * P.g[d];
  P.kr_m_int = (cl->kr_m >= 1.0 && cl->kr_m <= 8.0 && cl->kr_m == floor(cl->kr_m)) ? (int)cl->kr_m : 0;
  P.cfl = op->cfl;
  P.dt_max = op->dt_max;
  s->opt = *op;
  s->precision = op->precision;
  s->stream = nullptr;

  s->arena_bytes = carve(nullptr, L, nullptr);
  cudaError_t e = dev_block_alloc(&s->arena_mem, s->arena_bytes);
  if (e != cudaSuccess) {
    int code = e == cudaErrorMemoryAllocation ? MDBS_ERR_OOM
               : e == cudaErrorInvalidValue  ? MDBS_ERR_ARG
                                              : MDBS_ERR_CUDA;
    fail(nullptr, code, std::string("device arena: ") +
                            (e == cudaErrorInvalidValue ? "the allocator hook returned memory not aligned to 256 bytes"
                                                        : cudaGetErrorString(e)));
    cudaGetLastError();
    delete s;
    return code;
  }
  s->arena = s->arena_mem.ptr;
  cudaMemset(s->arena, 0, s->arena_bytes);
  carve(s, L, (char*)s->arena);
  e = cudaMallocHost(&s->host_scal, kNumSlots * sizeof(double));
  if (e == cudaSuccess) s->ps = pressure_create(P, s->precision, &e);
  if (e != cudaSuccess) {
    int code = e == cudaErrorMemoryAllocation ? MDBS_ERR_OOM : MDBS_ERR_CUDA;
    fail(nullptr, code, std::string("pressure solver: ") + cudaGetErrorString(e));
    cudaGetLastError();
    if (s->host_scal) cudaFreeHost(s->host_scal);
    dev_block_free(&s->arena_mem);
    delete s;
    return code;
  }
  e = cudaMemcpy((void*)s->F.phi, porosity, cells * 8, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy((void*)s->F.k0, permeability, cells * 8, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    // this simulation alone as a batch of one
    StepDom sd = step_view(s);
    CgDom cg;
    pressure_view(s->ps, s->F, s->tun.tail_cells, &cg);
    e = exec_setup(s->ex, &sd, &cg, 1, s->precision != 0, s->tun);
  }
  if (e == cudaSuccess) {
    Activate act(s);
    launch_static_geometry(s->ex.plan, nullptr);
    launch_set_boundary_velocities(s->ex.plan, nullptr);
    e = cudaDeviceSynchronize();
  }
  if (e != cudaSuccess) {
    fail(nullptr, MDBS_ERR_CUDA, std::string("setup: ") + cudaGetErrorString(e));
    mdbs_destroy(s);
    return MDBS_ERR_CUDA;
  }
  *out = s;
  return MDBS_OK;
}

// 1 in *flag if any of the n values lies outside [lo, hi] (NaN fails both comparisons)
__global__ void k_check_range(const double* __restrict__ a, long long n, double lo, double hi, double* flag) {
  int bad = 0;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
    const double v = a[c];
    bad |= !(v >= lo && v <= hi);
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) *flag = 1.0;
}

int mdbs_set_fields(mdbs_sim* s, const double* alpha, const double* ux, const double* uy, const double* uz,
                    const double* p) {
  if (!s) return MDBS_ERR_ARG;
  if (!alpha || !ux || !uy || !p || (s->P.dim == 3 && !uz)) return fail(s, MDBS_ERR_ARG, "NULL field");
  Activate act(s);
  // New input must lie in [0, 1] to 1e-9 (round-off of an earlier computation).  State
  // this simulation produced itself must survive a get_fields / set_fields round trip:
  // transport through a velocity field divergence-free only to the pressure tolerance
  // moves alpha outside [0, 1] by dt |div(A u)| / (phi V) per step, so the range also
  // admits the extremes its own steps have reached.
  // The check runs on the device: alpha goes to the low-order saturation scratch (which
  // the next step overwrites), a kernel flags any value out of range, and only an
  // accepted field is copied into place, so a rejected call leaves the state unchanged.
  const double lo = std::min(-1e-9, s->alpha_lo_seen), hi = std::max(1.0 + 1e-9, s->alpha_hi_seen);
  double* stage = s->F.aL;
  CK(cudaMemcpyAsync(stage, alpha, s->P.cells * 8, cudaMemcpyHostToDevice, s->stream));
  CK(cudaMemsetAsync(s->scal + kSlotCheck, 0, sizeof(double), s->stream));
  {
    const long long blocks = std::min<long long>((s->P.cells + 255) / 256, 4096);
    k_check_range<<<(unsigned)blocks, 256, 0, s->stream>>>(stage, s->P.cells, lo, hi, s->scal + kSlotCheck);
    CK(cudaGetLastError());
  }
  CK(cudaMemcpyAsync(s->host_scal + kSlotCheck, s->scal + kSlotCheck, sizeof(double), cudaMemcpyDeviceToHost,
                     s->stream));
  CK(cudaStreamSynchronize(s->stream));
  if (s->host_scal[kSlotCheck] != 0.0)
    return fail(s, MDBS_ERR_ARG,
                "alpha must lie in [0, 1] (to 1e-9, or within the extremes this simulation reached)");
  const double* src[3] = {ux, uy, uz};
  CK(cudaMemcpyAsync(s->F.alpha, stage, s->P.cells * 8, cudaMemcpyDeviceToDevice, s->stream));
  CK(cudaMemcpyAsync(s->F.p, p, s->P.cells * 8, cudaMemcpyHostToDevice, s->stream));
  for (int d = 0; d < s->P.dim; d++)
    CK(cudaMemcpyAsync(s->F.u[d], src[d], s->P.nf[d] * 8, cudaMemcpyHostToDevice, s->stream));
  launch_set_boundary_velocities(s->ex.plan, s->stream);
  // the step's saturation phase reads the closures of the new alpha; normals and
  // curvature are formed again from alpha^{k+1} before the momentum assembly reads them
  launch_closures(s->ex.plan, s->stream);
  for (int i = 0; i < kNumSlots; i++) s->host_scal[i] = 0.0;
  s->host_scal[kSlotDt] = s->opt.dt;
  CK(cudaMemcpyAsync(s->scal, s->host_scal, kNumSlots * sizeof(double), cudaMemcpyHostToDevice, s->stream));
  launch_field_stats(s->ex.plan, s->stream);
  CK(cudaGetLastError());
  memset(&s->st, 0, sizeof(s->st));
  s->prof.launches = 0;
  s->fields_set = true;
  return refresh_stats(s);
}

int mdbs_step(mdbs_sim* s, int32_t n) {
  if (!s) return MDBS_ERR_ARG;
  if (n < 1) return fail(s, MDBS_ERR_ARG, "n must be >= 1");
  if (!s->fields_set) return fail(s, MDBS_ERR_ARG, "mdbs_set_fields has not been called");
  if (s->in_batch) return fail(s, MDBS_ERR_ARG, "the simulation belongs to a batch: step the batch");
  Activate act(s);
  const double it0 = s->host_scal[kSlotItersTotal];
  const double nc0 = s->host_scal[kSlotNotConverged];
  const bool eager = s->prof.on;
  CK(exec_steps(s->ex, s->opt, s->prof, s->stream, n));
  s->st.steps += n;
  int rc = refresh_stats(s);
  if (plan_failed(s->ex.plan)) return fail(s, MDBS_ERR_CUDA, "a device wait for staged data timed out");
  // kernels launched by the graphs: the fixed part of every step plus the CG bodies run
  if (!eager)
    s->prof.launches += (long long)n * s->ex.static_launches +
                        (long long)(s->host_scal[kSlotItersTotal] - it0) * s->ex.body_launches;
  s->st.kernel_launches = s->prof.launches;
  if (rc == MDBS_OK) rc = convergence_check(s, nc0);
  return rc;
}

int mdbs_get_fields(const mdbs_sim* cs, double* alpha, double* ux, double* uy, double* uz, double* p) {
  mdbs_sim* s = const_cast<mdbs_sim*>(cs);
  if (!s) return MDBS_ERR_ARG;
  double* dst[3] = {ux, uy, uz};
  if (alpha) CK(cudaMemcpyAsync(alpha, s->F.alpha, s->P.cells * 8, cudaMemcpyDeviceToHost, s->stream));
  if (p) CK(cudaMemcpyAsync(p, s->F.p, s->P.cells * 8, cudaMemcpyDeviceToHost, s->stream));
  for (int d = 0; d < s->P.dim; d++)
    if (dst[d]) CK(cudaMemcpyAsync(dst[d], s->F.u[d], s->P.nf[d] * 8, cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  return MDBS_OK;
}

void mdbs_destroy(mdbs_sim* s) {
  if (!s) return;
  if (s->stream) cudaStreamSynchronize(s->stream);
  cudaDeviceSynchronize();
  exec_destroy(s->ex);
  pressure_destroy(s->ps);
  if (s->host_scal) cudaFreeHost(s->host_scal);
  dev_block_free(&s->arena_mem);
  delete s;
}

int mdbs_get_stats(const mdbs_sim* s, mdbs_stats* out) {
  if (!s || !out) return MDBS_ERR_ARG;
  *out = s->st;
  return MDBS_OK;
}

const char* mdbs_last_error(const mdbs_sim* s) { return s ? s->err.c_str() : g_create_error.c_str(); }

int mdbs_set_stream(mdbs_sim* s, void* stream) {
  if (!s) return MDBS_ERR_ARG;
  s->stream = (cudaStream_t)stream;
  return MDBS_OK;
}

// ---------------------------------------------------------------- batches
int mdbs_batch_create(mdbs_sim* const* sims, int32_t n, mdbs_batch** out) {
  if (!out) return fail(nullptr, MDBS_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!sims || n < 1) return fail(nullptr, MDBS_ERR_ARG, "a batch needs at least one simulation");
  for (int i = 0; i < n; i++) {
    if (!sims[i]) return fail(nullptr, MDBS_ERR_ARG, "NULL simulation");
    if (sims[i]->in_batch) return fail(nullptr, MDBS_ERR_ARG, "a simulation already belongs to a batch");
    if (!sims[i]->fields_set) return fail(nullptr, MDBS_ERR_ARG, "mdbs_set_fields has not been called");
    if (!same_solver_options(sims[i]->opt, sims[0]->opt))
      return fail(nullptr, MDBS_ERR_ARG, "batched simulations need the same solver options and precision class");
    for (int j = 0; j < i; j++)
      if (sims[j] == sims[i]) return fail(nullptr, MDBS_ERR_ARG, "a simulation appears twice");
  }
  mdbs_batch* b = new (std::nothrow) mdbs_batch();
  if (!b) return fail(nullptr, MDBS_ERR_OOM, "host allocation failed");
  b->sims.assign(sims, sims + n);
  b->opt = sims[0]->opt;
  b->stream = nullptr;
  b->tun = sims[0]->tun;
  cudaError_t e = batch_exec_setup(b);
  if (e == cudaSuccess) e = cudaMalloc(&b->gather, (size_t)n * kNumSlots * sizeof(double));
  if (e == cudaSuccess) e = cudaMallocHost(&b->host_gather, (size_t)n * kNumSlots * sizeof(double));
  if (e != cudaSuccess) {
    int code = e == cudaErrorMemoryAllocation ? MDBS_ERR_OOM : MDBS_ERR_CUDA;
    fail(nullptr, code, std::string("batch: ") + cudaGetErrorString(e));
    cudaGetLastError();
    mdbs_batch_destroy(b);
    return code;
  }
  for (int i = 0; i < n; i++) sims[i]->in_batch = true;
  *out = b;
  return MDBS_OK;
}

// ---------------------------------------------------------------- schedule
int mdbs_set_tuning(mdbs_sim* s, const mdbs_tuning* t) {
  if (!s) return MDBS_ERR_ARG;
  if (!valid_tuning(t)) return fail(s, MDBS_ERR_ARG, "invalid tuning");
  if (s->in_batch) return fail(s, MDBS_ERR_ARG, "the simulation belongs to a batch: tune the batch");
  CK(cudaStreamSynchronize(s->stream));
  const mdbs_tuning old = s->tun;
  s->tun = *t;
  cudaError_t e = sim_exec_setup(s);
  if (e != cudaSuccess) {
    s->tun = old;
    cudaGetLastError();
    sim_exec_setup(s);
    return cuda_fail(s, e, "set_tuning");
  }
  return MDBS_OK;
}

int mdbs_get_tuning(const mdbs_sim* s, mdbs_tuning* out) {
  if (!s || !out) return MDBS_ERR_ARG;
  *out = s->tun;
  return MDBS_OK;
}

int mdbs_batch_set_tuning(mdbs_batch* b, const mdbs_tuning* t) {
  if (!b) return MDBS_ERR_ARG;
  if (!valid_tuning(t)) {
    b->err = "invalid tuning";
    return MDBS_ERR_ARG;
  }
  cudaError_t e = cudaStreamSynchronize(b->stream);
  const mdbs_tuning old = b->tun;
  b->tun = *t;
  if (e == cudaSuccess) e = batch_exec_setup(b);
  if (e != cudaSuccess) {
    b->tun = old;
    cudaGetLastError();
    batch_exec_setup(b);
    b->err = std::string("set_tuning: ") + cudaGetErrorString(e);
    return MDBS_ERR_CUDA;
  }
  return MDBS_OK;
}

int mdbs_batch_get_tuning(const mdbs_batch* b, mdbs_tuning* out) {
  if (!b || !out) return MDBS_ERR_ARG;
  *out = b->tun;
  return MDBS_OK;
}

int mdbs_autotune(mdbs_sim* s, int32_t trial_steps, mdbs_tuning* chosen, double* trial_ms, int32_t capacity,
                  int32_t* trials) {
  if (!s) return MDBS_ERR_ARG;
  if (trial_steps < 1 || capacity < 0) return fail(s, MDBS_ERR_ARG, "trial_steps must be >= 1");
  if (!s->fields_set) return fail(s, MDBS_ERR_ARG, "mdbs_set_fields has not been called");
  if (s->in_batch) return fail(s, MDBS_ERR_ARG, "the simulation belongs to a batch: tune the batch");
  Activate act(s);
  CK(cudaStreamSynchronize(s->stream));
  auto setup = [&](const mdbs_tuning& t) {
    s->tun = t;
    return sim_exec_setup(s);
  };
  std::vector<mdbs_sim*> one{s};
  mdbs_tuning tun = s->tun;
  int nt = 0;
  const int rc = autotune_impl(one, s->ex, s->opt, s->prof, s->stream, tun, setup, trial_steps, trial_ms, capacity,
                               &nt, s->err, s->precision != 0);
  if (trials) *trials = nt;
  if (rc == MDBS_OK && chosen) *chosen = s->tun;
  return rc;
}

int mdbs_batch_autotune(mdbs_batch* b, int32_t trial_steps, mdbs_tuning* chosen, double* trial_ms,
                        int32_t capacity, int32_t* trials) {
  if (!b) return MDBS_ERR_ARG;
  if (trial_steps < 1 || capacity < 0) {
    b->err = "trial_steps must be >= 1";
    return MDBS_ERR_ARG;
  }
  Activate act(b);
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) {
    b->err = "stream error before autotune";
    return MDBS_ERR_CUDA;
  }
  auto setup = [&](const mdbs_tuning& t) {
    b->tun = t;
    return batch_exec_setup(b);
  };
  mdbs_tuning tun = b->tun;
  int nt = 0;
  const int rc = autotune_impl(b->sims, b->ex, b->opt, b->prof, b->stream, tun, setup, trial_steps, trial_ms,
                               capacity, &nt, b->err, b->sims[0]->precision != 0);
  if (trials) *trials = nt;
  if (rc == MDBS_OK && chosen) *chosen = b->tun;
  return rc;
}

int mdbs_batch_set_stream(mdbs_batch* b, void* stream) {
  if (!b) return MDBS_ERR_ARG;
  b->stream = (cudaStream_t)stream;
  return MDBS_OK;
}

int mdbs_batch_step(mdbs_batch* b, int32_t n) {
  if (!b) return MDBS_ERR_ARG;
  if (n < 1) {
    b->err = "n must be >= 1";
    return MDBS_ERR_ARG;
  }
  Activate act(b);
  const int nd = (int)b->sims.size();
  const bool eager = b->prof.on;
  double it0 = 0.0;
  std::vector<double> nc0(nd);
  for (int i = 0; i < nd; i++) {
    it0 += b->sims[i]->host_scal[kSlotItersTotal];
    nc0[i] = b->sims[i]->host_scal[kSlotNotConverged];
  }
  cudaError_t e = exec_steps(b->ex, b->opt, b->prof, b->stream, n);
  // gather every member's scalars, then one copy to the host
  for (int i = 0; i < nd && e == cudaSuccess; i++)
    e = cudaMemcpyAsync(b->gather + (size_t)i * kNumSlots, b->sims[i]->scal, kNumSlots * sizeof(double),
                        cudaMemcpyDeviceToDevice, b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->host_gather, b->gather, (size_t)nd * kNumSlots * sizeof(double), cudaMemcpyDeviceToHost,
                        b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) {
    b->err = std::string("batch step: ") + cudaGetErrorString(e);
    return MDBS_ERR_CUDA;
  }
  if (plan_failed(b->ex.plan)) {
    b->err = "a device wait for staged data timed out";
    return MDBS_ERR_CUDA;
  }
  int rc = MDBS_OK;
  double it1 = 0.0;
  for (int i = 0; i < nd; i++) {
    mdbs_sim* s = b->sims[i];
    const double* h = b->host_gather + (size_t)i * kNumSlots;
    for (int k = 0; k < kNumSlots; k++) s->host_scal[k] = h[k];
    s->st.steps += n;
    it1 += h[kSlotItersTotal];
    int r = stats_from(s, h);
    if (r == MDBS_OK) r = convergence_check(s, nc0[i]);
    // a diverged member outranks one whose solves stopped at max_cg
    if (r != MDBS_OK && (rc == MDBS_OK || (rc == MDBS_ERR_NOT_CONVERGED && r != MDBS_ERR_NOT_CONVERGED))) {
      rc = r;
      b->err = "domain " + std::to_string(i) + ": " + s->err;
    }
  }
  // the CG loop runs while any member iterates: per corrector, the slowest member's count
  // (exact for n == 1)
  if (!eager) {
    long long iters = 0;
    for (int c = 0; c < b->opt.n_corr && c < 8; c++) {
      int mx = 0;
      for (mdbs_sim* s : b->sims) mx = std::max(mx, (int)s->st.cg_iters[c]);
      iters += mx;
    }
    b->prof.launches += (long long)n * (b->ex.static_launches + iters * b->ex.body_launches);
  }
  (void)it0;
  (void)it1;
  return rc;
}

const char* mdbs_batch_last_error(const mdbs_batch* b) { return b ? b->err.c_str() : g_create_error.c_str(); }

int mdbs_batch_add(mdbs_batch* b, mdbs_sim* s) {
  if (!b) return fail(nullptr, MDBS_ERR_ARG, "batch is NULL");
  auto bad = [&](const char* m) {
    b->err = m;
    return MDBS_ERR_ARG;
  };
  if (!s) return bad("NULL simulation");
  if (s->in_batch) return bad("the simulation already belongs to a batch");
  if (!s->fields_set) return bad("mdbs_set_fields has not been called");
  if (!same_solver_options(s->opt, b->sims[0]->opt))
    return bad("batched simulations need the same solver options and precision class");
  if (b->stream) cudaStreamSynchronize(b->stream);
  cudaDeviceSynchronize();
  const size_t n = b->sims.size() + 1;
  double *g = nullptr, *hg = nullptr;
  cudaError_t e = cudaMalloc(&g, n * kNumSlots * sizeof(double));
  if (e == cudaSuccess) e = cudaMallocHost(&hg, n * kNumSlots * sizeof(double));
  if (e == cudaSuccess) {
    b->sims.push_back(s);
    e = batch_exec_setup(b);
    if (e != cudaSuccess) {  // back to the previous members
      b->sims.pop_back();
      cudaGetLastError();
      batch_exec_setup(b);
    }
  }
  if (e != cudaSuccess) {
    if (g) cudaFree(g);
    if (hg) cudaFreeHost(hg);
    b->err = std::string("batch add: ") + cudaGetErrorString(e);
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? MDBS_ERR_OOM : MDBS_ERR_CUDA;
  }
  cudaFree(b->gather);
  cudaFreeHost(b->host_gather);
  b->gather = g;
  b->host_gather = hg;
  s->in_batch = true;
  return MDBS_OK;
}

int mdbs_batch_remove(mdbs_batch* b, mdbs_sim* s) {
  if (!b) return fail(nullptr, MDBS_ERR_ARG, "batch is NULL");
  size_t at = 0;
  while (at < b->sims.size() && b->sims[at] != s) at++;
  if (!s || at == b->sims.size()) {
    b->err = "the simulation is not a member of this batch";
    return MDBS_ERR_ARG;
  }
  if (b->sims.size() == 1) {
    b->err = "a batch keeps at least one member";
    return MDBS_ERR_ARG;
  }
  if (b->stream) cudaStreamSynchronize(b->stream);
  cudaDeviceSynchronize();
  b->sims.erase(b->sims.begin() + at);
  cudaError_t e = batch_exec_setup(b);
  if (e != cudaSuccess) {  // back to the previous members
    b->sims.insert(b->sims.begin() + at, s);
    cudaGetLastError();
    batch_exec_setup(b);
    b->err = std::string("batch remove: ") + cudaGetErrorString(e);
    return MDBS_ERR_CUDA;
  }
  s->in_batch = false;
  return MDBS_OK;
}

void mdbs_batch_destroy(mdbs_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  cudaDeviceSynchronize();
  exec_destroy(b->ex);
  if (b->gather) cudaFree(b->gather);
  if (b->host_gather) cudaFreeHost(b->host_gather);
  for (mdbs_sim* s : b->sims) s->in_batch = false;
  delete b;
}

int mdbs_profile_enable(mdbs_sim* s, int32_t enable, int32_t only_id) {
  if (!s || only_id < -1 || only_id >= K_COUNT) return MDBS_ERR_ARG;
  if (s->prof.on) s->prof.resolve();
  s->prof.on = enable != 0;
  s->prof.only = only_id;
  s->prof.reset();
  return MDBS_OK;
}

int32_t mdbs_profile_count(void) { return K_COUNT; }

int mdbs_profile_read(const mdbs_sim* s, int32_t id, const char** name, double* total_ms, int64_t* launches) {
  if (id < 0 || id >= K_COUNT) return MDBS_ERR_ARG;
  if (name) *name = kKernelNames[id];
  if (total_ms) *total_ms = s ? s->prof.ms[id] : 0.0;
  if (launches) *launches = s ? s->prof.count[id] : 0;
  return MDBS_OK;
}

int mdbs_check_bounded_wait(double* waited_s) {
  if (!waited_s) return fail(nullptr, MDBS_ERR_ARG, "waited_s is NULL");
  int status = 0;
  cudaError_t e = bounded_wait_selftest(&status, waited_s);
  if (e != cudaSuccess) return fail(nullptr, MDBS_ERR_CUDA, std::string("bounded wait: ") + cudaGetErrorString(e));
  if (status != 1) return fail(nullptr, MDBS_ERR_CUDA, "the bounded wait did not give up as designed");
  return MDBS_OK;
}

int64_t mdbs_debug_array(const mdbs_sim* cs, const char* name, double* out, int64_t capacity) {
  mdbs_sim* s = const_cast<mdbs_sim*>(cs);
  if (!s || !name) return MDBS_ERR_ARG;
  const Fld& F = s->F;
  const long long nc = s->P.cells;
  struct Ent {
    const char* nm;
    const double* a;
    long long n;
  } tab[] = {
      {"rho", F.rho, nc},          {"mu", F.mu, nc},
      {"drag", F.drag, nc},        {"pc", F.pc, nc},            {"cf", F.cf, nc},
      {"Ml", F.Ml, nc},            {"Mg", F.Mg, nc},            {"kappa", F.kappa, nc},
      {"mx", F.m[0], nc},          {"my", F.m[1], nc},          {"mz", F.m[2], nc},
      {"Tx", F.T[0], nc},          {"Ty", F.T[1], nc},          {"Tz", F.T[2], nc},
      {"Dd", F.Dd, nc},            {"b", F.b, nc},              {"aL", F.aL, nc},
      {"Rp", F.Rp, nc},            {"Rm", F.Rm, nc},            {"nwx", F.nw[0], nc},
      {"nwy", F.nw[1], nc},        {"nwz", F.nw[2], nc},        {"aPx", F.aP[0], s->P.nf[0]},
      {"aPy", F.aP[1], s->P.nf[1]}, {"aPz", F.aP[2], s->P.nf[2]}, {"rhs0x", F.rhs0[0], s->P.nf[0]},
      {"rhs0y", F.rhs0[1], s->P.nf[1]}, {"rhs0z", F.rhs0[2], s->P.nf[2]}, {"Bx", F.B[0], s->P.nf[0]},
      {"By", F.B[1], s->P.nf[1]},  {"Bz", F.B[2], s->P.nf[2]},  {"hbyax", F.hbya[0], s->P.nf[0]},
      {"hbyay", F.hbya[1], s->P.nf[1]}, {"hbyaz", F.hbya[2], s->P.nf[2]}, {"FLOx", F.FLO[0], s->P.nf[0]},
      {"FLOy", F.FLO[1], s->P.nf[1]}, {"FLOz", F.FLO[2], s->P.nf[2]}, {"AFx", F.AF[0], s->P.nf[0]},
      {"AFy", F.AF[1], s->P.nf[1]}, {"AFz", F.AF[2], s->P.nf[2]},
  };
  for (const Ent& e : tab) {
    if (strcmp(e.nm, name) != 0) continue;
    long long n = e.n;
    if (s->P.dim == 2 && (name[strlen(name) - 1] == 'z') && strcmp(name, "mz") != 0 && strcmp(name, "Tz") != 0 &&
        strcmp(name, "nwz") != 0)
      n = 0;
    if (out && capacity > 0) {
      long long m = n < capacity ? n : capacity;
      // the pressure system (T, D, b) is stored x-split: even cells of each row, then
      // odd ones; the copy returns natural x-fastest order
      const bool xsplit = e.a == F.T[0] || e.a == F.T[1] || e.a == F.T[2] || e.a == F.Dd || e.a == F.b;
      if (m > 0 && xsplit) {
        std::vector<double> dev((size_t)n);
        cudaError_t er = cudaMemcpyAsync(dev.data(), e.a, n * 8, cudaMemcpyDeviceToHost, s->stream);
        if (er == cudaSuccess) er = cudaStreamSynchronize(s->stream);
        if (er != cudaSuccess) return cuda_fail(s, er, "debug copy");
        const long long n0 = s->P.n[0], he = (n0 + 1) / 2;
        for (long long c = 0; c < m; c++) {
          const long long row = c / n0, i = c - row * n0;
          out[c] = dev[(size_t)(row * n0 + ((i & 1) ? he + i / 2 : i / 2))];
        }
      } else if (m > 0) {
        cudaError_t er = cudaMemcpyAsync(out, e.a, m * 8, cudaMemcpyDeviceToHost, s->stream);
        if (er == cudaSuccess) er = cudaStreamSynchronize(s->stream);
        if (er != cudaSuccess) return cuda_fail(s, er, "debug copy");
        // the a_P arrays hold reciprocals on the device (fixed faces hold 1)
        if (name[0] == 'a' && name[1] == 'P')
          for (long long i = 0; i < m; i++) out[i] = 1.0 / out[i];
      }
    }
    return n;
  }
  return fail(s, MDBS_ERR_ARG, std::string("unknown array ") + name);
}

}  // extern "C"
