// mdbs_internal.cuh -- device-side data structures shared by the CUDA
// translation units of libmdbs (sm_103a).  Not part of the public ABI.
//
// Execution model.  Every kernel runs over a *batch* of domains (a single
// simulation is a batch of one).  A Work table maps a flat block index to
// (domain, local block) through a prefix table of per-domain block counts, and
// kernels walk the blocks with a grid-stride loop over a grid sized to the GPU
// (persistent launch).  Per-domain views (StepDom, CgDom) live in device tables
// so one launch per phase advances every domain of the batch.
#pragma once
#include <cuda.h>  // CUtensorMap (type only; the encoder is fetched through the runtime)
#include <cuda_runtime.h>
#include <stdint.h>

namespace mdbs {

constexpr int kWall = 0, kInlet = 1, kOutlet = 2;
constexpr int kMaxLevels = 16;
constexpr int kBlock = 256;
constexpr int kRepBig = 8;  // rows of kBlock per work item in the cell and face spaces

// slots of the per-domain device scalar array
constexpr int kSlotMass = 0, kSlotAmin = 1, kSlotAmax = 2, kSlotBad = 3, kSlotUmax = 4, kSlotInflow = 5,
              kSlotDt = 6, kSlotTime = 7, kSlotIters = 8 /* 8 correctors */, kSlotResid = 16 /* 8 */,
              kSlotItersTotal = 24, kSlotNotConverged = 25, kSlotCheck = 26, kNumSlots = 32;

// Division by a divisor fixed for a level, without a hardware divide: for
// 0 <= t < 2^31, t / d == (t * m) >> s with s = 31 + ceil(log2 d) and
// m = ceil(2^s / d) < 2^32 (Granlund and Montgomery, "Division by invariant
// integers using multiplication", 1994).
struct FastDiv {
  unsigned m;
  unsigned s;
};
inline FastDiv make_fastdiv(unsigned d) {
  unsigned l = 0;
  while ((1ull << l) < d) l++;
  const unsigned long long num = 1ull << (31 + l);
  return FastDiv{(unsigned)((num + d - 1) / d), 31 + l};
}
__device__ __forceinline__ unsigned fastdiv(unsigned t, FastDiv f) {
  return (unsigned)(((unsigned long long)t * f.m) >> f.s);
}

// Geometry and physical parameters of one domain.
struct Prm {
  int n[3];  // cells per axis
  int dim;   // 2 or 3
  long long cells;
  long long nf[3];  // faces per direction
  double h, A, V;
  int bc[6];
  double inlet_u, inlet_alpha;
  double rho_l, mu_l, rho_g, mu_g, sigma, g[3];
  int kr_model, pc_model;
  double kr_m, a_l_irr, a_g_irr, pc0, pc_beta, pc_m, a_pc_irr, a_pc_max, pc_eps;
  int porous_density;   // 0: mobility-weighted rho* (Eq. 45), 1: Appendix B
  double cos_t, sin_t;  // contact angle
  double c_alpha;
  double inv_h, half_inv_h;  // 1/h and 1/(2h)
  // reciprocals of run-time constants (the kernels multiply; GB300's FP64 division is slow)
  double inv_mu_l, inv_mu_g;  // 1/mu_l, 1/mu_g
  double inv_ae_den;          // 1/(1 - a_g_irr - a_l_irr), effective saturation
  double inv_s_den;           // 1/(a_pc_max - a_pc_irr), capillary saturation
  double reg_m;               // 1e-8/h, regularisation of |grad alpha| in the interface normal
  double inv_h2;              // 1/h^2
  double drho_g[3];           // (rho_l - rho_g) g_d, the buoyancy drive of the porous relative flux
  int kr_m_int;              // kr exponent when it is an integer in [1, 8], else 0
  double cfl, dt_max;        // adaptive time step (cfl > 0)
  FastDiv dn0, dn1;          // division by n[0] and by n[1]
  FastDiv dn0p, dn1p;        // division by n[0] + 1 and by n[1] + 1 (face arrays)
};

// Device arrays of one domain.
struct Fld {
  // static
  const double* phi;
  const double* k0;
  const uint8_t* is_free;
  const double* nw[3];  // wall normal (zero outside contact cells)
  const double* iphi2;  // phi^-2 (porosity-gradient part of the convection)
  const double* iphiV;  // 1 / (phi V) (saturation updates)
  const double* iphif[3];  // 1 / phi_f, phi_f the mean porosity of a face's two cells
  const double* gphi[3];   // grad(phi^-2) at a face: component e of direction-d faces at e * nf[d] + f
                           // (the components across the face's normal carry a factor 1/4)
  // state
  double* alpha;
  double* p;
  double* u[3];
  // properties
  double *Ml, *Mg, *fw, *pc, *cf, *rho, *mu, *drag, *m[3], *kappa;  // fw = M_l / M
  // edge viscosities (mean of the four cells around an edge) of the axis pairs (0,1),
  // (0,2), (1,2): extent n + 1 along the pair's axes, natural x-fastest order
  double* muE[3];
  // saturation step
  double *FLO[3], *AF[3], *aL, *Rp, *Rm;
  // momentum
  double *aP[3], *anb[3], *rhs0[3], *B[3], *hbya[3], *utmp[3];  // aP holds 1 / a_P
  // pressure system (level 0)
  double *T[3], *Dd, *diag, *dinv, *b;
};

// One multigrid level (T is stored per cell for the face towards +axis).  In the
// FP32 hierarchy of MDBS_MIXED_BF16 the coarse levels (l >= 1) keep T as BF16 bit
// patterns in Tb (T is then NULL); every reader widens them to FP32.
template <typename R>
struct Level {
  int n[3];
  int cz[3];  // axis coarsened relative to the finer level
  long long cells;
  FastDiv dhalf, dn0, dn1;  // division by ceil(n[0] / 2), by n[0] and by n[1]
  R* T[3];
  uint16_t* Tb[3];
  R* Dd;
  R* diag;
  R* dinv;  // 1 / diag (multiplied in the smoothers instead of dividing)
  R* x;
  R* x2;    // second iterate buffer of the fused red-black sweeps (read one, write the other)
  R* b;
};

// ---------------------------------------------------------------- batches
struct Work {
  const int* blk;  // device table, ndom + 1 entries: first item of each domain, then the total
  int ndom;
  int total;       // work items; item i of a domain covers elements [i*rep*blockDim, (i+1)*rep*blockDim)
  int rep;         // blockDim-sized rows per work item
};

// domain owning flat block b: the largest d with blk[d] <= b (empty domains are skipped)
__device__ __forceinline__ int work_domain(const Work& w, int b) {
  int lo = 0, hi = w.ndom - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (w.blk[mid] <= b)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// per-domain view of the step kernels
struct StepDom {
  Prm P;
  Fld F;
  double* scal;      // step scalars (kSlot*)
  double* partials;  // reduction partials: 4 channels of pcap values
  long long pcap;    // partials per channel (>= work items of the largest space)
};

// per-domain view of the pressure solver
struct CgDom {
  Level<double> ld[kMaxLevels];  // FP64 hierarchy (level 0 arrays point into Fld)
  Level<float> lf[kMaxLevels];   // FP32 hierarchy (mixed precision)
  int nlev;
  int first;  // first level handled by the single-CTA tail
  double *r, *z, *dv, *q;
  double* partials;  // 2 channels of pcap values
  long long pcap;
  double* scal;      // CG scalars
  double* cinv_d;    // inverse of the coarsest operator
  float* cinv_f;
  // TMA descriptors of the FP32 levels (kTmaMaps per level: x, x2, b, 1/diag, T_x, T_y,
  // T_z); bit l of tma_levels set when level l has them
  const CUtensorMap* tmaps;
  unsigned tma_levels;
};

// ---------------------------------------------------------------- helpers
__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

__device__ __forceinline__ long long cell_index(const int n[3], int i, int j, int k) {
  return i + (long long)n[0] * (j + (long long)n[1] * k);
}

// face index of direction d at face coordinates (i, j, k), c[d] in [0, n[d]]
__device__ __forceinline__ long long face_index(const int n[3], int d, int i, int j, int k) {
  long long fx = n[0] + (d == 0), fy = n[1] + (d == 1);
  return i + fx * (j + fy * k);
}

// read with zero-gradient ghost cells (coordinates clamped into the grid)
__device__ __forceinline__ double ghost_read(const double* __restrict__ a, const int n[3], int i, int j,
                                             int k) {
  i = clampi(i, 0, n[0] - 1);
  j = clampi(j, 0, n[1] - 1);
  k = clampi(k, 0, n[2] - 1);
  return a[cell_index(n, i, j, k)];
}

// warp + block sum; result valid in thread 0
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double warp_part[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) warp_part[w] = v;
  __syncthreads();
  int nw = (blockDim.x + 31) >> 5;
  v = (threadIdx.x < nw) ? warp_part[threadIdx.x] : 0.0;
  if (w == 0)
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// warp + block minimum / maximum (order-independent); result valid in thread 0
template <bool MAX>
__device__ __forceinline__ double block_minmax(double v) {
  __shared__ double warp_part[32];
  for (int o = 16; o > 0; o >>= 1) {
    const double u = __shfl_down_sync(0xffffffffu, v, o);
    v = MAX ? fmax(v, u) : fmin(v, u);
  }
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) warp_part[w] = v;
  __syncthreads();
  int nw = (blockDim.x + 31) >> 5;
  v = (threadIdx.x < nw) ? warp_part[threadIdx.x] : (MAX ? -INFINITY : INFINITY);
  if (w == 0)
    for (int o = 16; o > 0; o >>= 1) {
      const double u = __shfl_down_sync(0xffffffffu, v, o);
      v = MAX ? fmax(v, u) : fmin(v, u);
    }
  return v;
}

// ---------------------------------------------------------------- launch accounting
// Every kernel launch goes through MDBS_LAUNCH: it counts the launch for the
// active simulation and, when profiling is on, brackets it with CUDA events on
// the launch stream.
enum KernelId {
  K_ALPHA_FLUX, K_ALPHA_LO, K_ALPHA_LIMIT, K_ALPHA_UPDATE, K_FINALIZE, K_PROPERTIES, K_NORMALS,
  K_CURVATURE, K_MOM_ASSEMBLE, K_JACOBI, K_HBYA, K_CORRECT, K_BOUNDARY, K_STATS, K_CFL, K_STATIC,
  K_ASSEMBLE, K_DIAG, K_CONVERT, K_COARSEN, K_SMOOTH0, K_SMOOTHC, K_ZERO, K_RESTRICT0, K_RESTRICTC,
  K_PROLONG0, K_PROLONGC, K_RESID0, K_SPMV_DOT, K_UPDATE_XR, K_DOTS, K_UPDATE_D, K_TAIL, K_COOP, K_EDGE_MU, K_COUNT
};
extern const char* const kKernelNames[K_COUNT];
void prof_begin(int id, cudaStream_t s);
void prof_end(int id, cudaStream_t s);
// the first error a kernel launch returned on this thread since the last take
void set_launch_error(cudaError_t e);
cudaError_t take_launch_error();
long long launch_count();  // kernels launched so far by the active simulation

//
// Launches are programmatic dependent launches: a kernel may be scheduled while
// its predecessor in the stream drains, and every kernel begins with
// MDBS_DEPENDENT_ENTRY(), which waits until the predecessor grid has completed and
// its memory is visible (griddepcontrol.wait) before touching any data, then lets
// its own successor start launching (griddepcontrol.launch_dependents).  The
// order of all memory effects is therefore the plain stream order; only the launch
// latency between dependent kernels overlaps (also inside captured graphs).
#define MDBS_DEPENDENT_ENTRY()                                    \
  do {                                                            \
    asm volatile("griddepcontrol.wait;\n" ::: "memory");          \
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); \
  } while (0)

#define MDBS_LAUNCH_SMEM(ID, GRID, BLOCK, SMEM, STREAM, KERNEL, ...)                                \
  do {                                                                                             \
    ::mdbs::prof_begin((ID), (STREAM));                                                            \
    cudaLaunchConfig_t cfg_ = {};                                                                  \
    cfg_.gridDim = dim3(GRID);                                                                     \
    cfg_.blockDim = dim3(BLOCK);                                                                   \
    cfg_.dynamicSmemBytes = (SMEM);                                                                \
    cfg_.stream = (STREAM);                                                                        \
    cudaLaunchAttribute at_[1];                                                                    \
    at_[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;                                \
    at_[0].val.programmaticStreamSerializationAllowed = 1;                                         \
    cfg_.attrs = at_;                                                                              \
    cfg_.numAttrs = 1;                                                                             \
    const cudaError_t le_ = cudaLaunchKernelEx(&cfg_, KERNEL, __VA_ARGS__);                        \
    if (le_ != cudaSuccess) ::mdbs::set_launch_error(le_);                                         \
    ::mdbs::prof_end((ID), (STREAM));                                                              \
  } while (0)

#define MDBS_LAUNCH(ID, GRID, BLOCK, STREAM, KERNEL, ...) \
  MDBS_LAUNCH_SMEM(ID, GRID, BLOCK, 0, STREAM, KERNEL, __VA_ARGS__)

// ---------------------------------------------------------------- host-side batch plan
// Block tables of one batch for every iteration space, uploaded once per
// batch composition.
struct BatchPlan {
  int ndom;
  int grid_cap;               // persistent grid: SMs x resident blocks
  Work cells, faces, dom;     // per-domain cells, faces (one row per item), one block per domain
  Work rcells, rfaces;        // the same with kRepBig rows per item: kernels with block reductions
  Work lcells[kMaxLevels];    // level-l cells of domains that have level l
  Work lhalf[kMaxLevels];     // level-l red/black half cells of domains whose level l precedes the tail
  Work lfine[kMaxLevels];     // level-l cells of the same domains (prolongation)
  Work lcoarse[kMaxLevels];   // level-(l+1) cells of the same domains (restriction)
  Work lsweep[kMaxLevels];    // fused-sweep tiles (kSweepTX x kSweepTY columns x sweep_kz planes) of the same domains
  Work lvec[kMaxLevels];      // vector half sweeps: kBlock threads x (2 FP64 / 4 FP32) half cells per item
  unsigned vec_levels;        // bit l: every domain's level l (before its tail) allows vector half sweeps
  int vec_sweeps;             // use them (schedule)
  int max_first;              // largest tail start over the domains
  long long tail_words;       // largest x + b element count of a domain's tail levels
  int tail_ctas;              // CTAs (one cluster) per domain in the tail kernel
  int max_levels;             // largest level count over the domains
  int flexible;               // FP32 V-cycle inside flexible CG
  int any_cfl;                // some domain uses the adaptive time step
  int snake;                  // alternate the traversal direction of consecutive level kernels
  int sweep_kz;               // > 0: fused red-black sweeps (FP32 levels) over chunks of this many planes
  int coarse_coop;            // levels between the finest and the tail in one cooperative launch
  int coop_grid;              // CTAs of that launch (all resident)
  unsigned long long* coop_ctr;  // device: arrival counter of its grid barriers
  StepDom* sd;                // device tables (ndom entries)
  CgDom* cg;
  int* table_storage;         // device memory of every block table
  int* any_flag;              // device: some domain still iterating (CG WHILE condition)
  int* err_flag;              // device: a kernel's bounded wait ran out (the batch's results are invalid)
};

inline int grid_of(const BatchPlan& B, const Work& w) {
  return w.total < B.grid_cap ? (w.total > 0 ? w.total : 1) : B.grid_cap;
}

// ---------------------------------------------------------------- launchers
// step_kernels.cu (dt, time and the statistics live in each domain's scalar array)
void launch_alpha_step(const BatchPlan& B, cudaStream_t s);
void launch_properties(const BatchPlan& B, cudaStream_t s);
// the closures alone (no normals or curvature): all the saturation step reads
void launch_closures(const BatchPlan& B, cudaStream_t s);
void launch_momentum_assemble(const BatchPlan& B, cudaStream_t s);
void launch_jacobi_sweeps(const BatchPlan& B, int sweeps, cudaStream_t s);  // result in F.u
void launch_hbya(const BatchPlan& B, cudaStream_t s);
void launch_correct(const BatchPlan& B, cudaStream_t s);
void launch_set_boundary_velocities(const BatchPlan& B, cudaStream_t s);
void launch_field_stats(const BatchPlan& B, cudaStream_t s);
void launch_time_advance(const BatchPlan& B, cudaStream_t s);
void launch_static_geometry(const BatchPlan& B, cudaStream_t s);

// capi.cu: bulk device allocations through the mdbs_set_allocator hook (or the
// CUDA runtime); a DevBlock remembers the hook that allocated it
struct DevBlock {
  void* ptr = nullptr;
  void (*free_fn)(void*, void*) = nullptr;  // nullptr: cudaFree
  void* ctx = nullptr;
};
cudaError_t dev_block_alloc(DevBlock* b, size_t bytes);
void dev_block_free(DevBlock* b);

// pressure.cu
struct PressureSolver;
PressureSolver* pressure_create(const Prm& P, int precision, cudaError_t* err);
void pressure_destroy(PressureSolver* ps);
size_t pressure_bytes(const int n[3], int precision);
// fills the per-domain solver view (level 0 of the FP64 hierarchy points into F);
// levels with at most tail_cells cells (and all coarser ones) go to the single-CTA tail
void pressure_view(const PressureSolver* ps, const Fld& F, int tail_cells, CgDom* out);
// the solver's single device allocation
void pressure_storage(const PressureSolver* ps, void** ptr, size_t* bytes);
constexpr int kTailCellsMax = 262144;
int pressure_precision(const PressureSolver* ps);
constexpr int kAsmMatrix = 1, kAsmRhs = 2;
void launch_pressure_matrix(const BatchPlan& B, int coarse_sweeps, cudaStream_t s);
void launch_pressure_rhs(const BatchPlan& B, cudaStream_t s);
// Enqueues the solve of A p = b for every domain of the batch by GMG-preconditioned
// CG.  Iterations and the final relative residual of corrector `corr` go to each
// domain's step scalars.  capture == false: the CG loop is driven from the host
// (host_flag: pinned scratch); capture == true: s is capturing a graph and the loop
// becomes a conditional WHILE node evaluated on the device (body captured on
// body_stream).  *body_launches receives the kernels of one CG iteration.
cudaError_t pressure_solve(const BatchPlan& B, double tol, int max_it, int nu1, int nu2, int coarse_sweeps, int corr,
                           bool capture, cudaStream_t s, cudaStream_t body_stream, double* host_flag,
                           long long* body_launches);

// batch.cu
// builds the block tables and device views of a batch of domains
// Fused red-black sweep tiles (FP32 levels): a CTA of kSweepBX x kSweepBY threads,
// each owning two adjacent cells of a row, covers kSweepCX x kSweepBY cells: the
// interior kSweepTX x kSweepTY plus a one-cell halo ring and spare columns.  Every
// array of a plane is staged as the natural x range [i0 - 8, i0 + 64) of kBoxY
// rows from j0 - 2: in the x-split storage that is one box of kBoxHX even cells
// and one of kBoxHX odd cells per row (i0 a multiple of 8 keeps both box starts
// on 16-byte boundaries when n_x is a multiple of 8).
constexpr int kSweepBX = 32, kSweepBY = 8, kSweepCX = 2 * kSweepBX;
constexpr int kSweepTX = kSweepCX - 8, kSweepTY = kSweepBY - 2;
constexpr int kBoxHX = (kSweepCX + 8) / 2, kBoxY = kSweepBY + 2;
constexpr int kSweepDepth = 1;  // planes staged ahead of use
constexpr int kTmaMaps = 7;
// opts the fused-sweep and tail kernels into their shared-memory sizes (current device)
cudaError_t sweep_kernel_setup();
// runs one bounded mbarrier wait that cannot complete; *status 1: it gave up as designed
cudaError_t bounded_wait_selftest(int* status, double* waited_s);

// smooth_rows: kBlock rows per work item of the finest-level half sweeps (1, 2, 4, 8);
// sweep_kz: planes per fused-sweep chunk (0: half sweeps); tail_ctas: CTAs per domain
// in the tail kernel (1, 2, 4, 8: one cluster)
// coarse_coop: run the levels between the finest and the tail in one cooperative launch
cudaError_t plan_create(const StepDom* sd, const CgDom* cg, int ndom, int flexible, int smooth_rows, int snake,
                        int sweep_kz, int tail_ctas, int coarse_coop, int vec_sweeps, BatchPlan* out);
// CTAs of the cooperative coarse-level kernel that are resident at once on this device
cudaError_t coop_grid_size(int flexible, long long tail_words, int* grid);
void plan_destroy(BatchPlan* B);

}  // namespace mdbs
