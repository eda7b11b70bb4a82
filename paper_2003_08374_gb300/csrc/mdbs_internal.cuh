// mdbs_internal.cuh -- device-side data structures shared by the CUDA
// translation units of libmdbs (sm_103a).  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace mdbs {

constexpr int kWall = 0, kInlet = 1, kOutlet = 2;
constexpr int kMaxLevels = 16;
constexpr int kBlock = 256;
constexpr int kMaxPartials = 2048;  // blocks per deterministic reduction

// slots of the per-simulation device scalar array
constexpr int kSlotMass = 0, kSlotAmin = 1, kSlotAmax = 2, kSlotBad = 3, kSlotUmax = 4, kSlotInflow = 5,
              kSlotDt = 6, kSlotTime = 7, kSlotIters = 8 /* 8 correctors */, kSlotResid = 16 /* 8 */,
              kSlotItersTotal = 24, kSlotNotConverged = 25, kNumSlots = 32;

// Geometry and physical parameters, passed by value to every kernel.
struct Prm {
  int n[3];      // cells per axis
  int dim;       // 2 or 3
  long long cells;
  long long nf[3];  // faces per direction
  double h, A, V;
  int bc[6];
  double inlet_u, inlet_alpha;
  double rho_l, mu_l, rho_g, mu_g, sigma, g[3];
  int kr_model, pc_model;
  double kr_m, a_l_irr, a_g_irr, pc0, pc_beta, pc_m, a_pc_irr, a_pc_max, pc_eps;
  double cos_t, sin_t;  // contact angle
  double c_alpha;
  double inv_h, half_inv_h;  // 1/h and 1/(2h)
  int kr_m_int;              // kr exponent when it is an integer in [1, 8], else 0
};

// Device arrays of one simulation.
struct Fld {
  // static
  const double* phi;
  const double* k0;
  const uint8_t* is_free;
  const double* nw[3];  // wall normal (zero outside contact cells)
  // state
  double* alpha;
  double* p;
  double* u[3];
  // properties
  double *Ml, *Mg, *pc, *cf, *rho, *rho_old, *mu, *drag, *m[3], *kappa;
  // saturation step
  double *FLO[3], *AF[3], *aL, *Rp, *Rm;
  // momentum
  double *aP[3], *anb[3], *rhs0[3], *B[3], *hbya[3], *utmp[3];  // aP holds 1 / a_P
  // pressure system (level 0)
  double *T[3], *Dd, *diag, *dinv, *b;
};

// One multigrid level (T is stored per cell for the face towards +axis).
template <typename R>
struct Level {
  int n[3];
  int cz[3];  // axis coarsened relative to the finer level
  long long cells;
  R* T[3];
  R* Dd;
  R* diag;
  R* dinv;  // 1 / diag (multiplied in the smoothers instead of dividing)
  R* x;
  R* b;
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

// ---------------------------------------------------------------- launch accounting
// Every kernel launch goes through MDBS_LAUNCH: it counts the launch for the
// active simulation and, when profiling is on, brackets it with CUDA events on
// the launch stream.
enum KernelId {
  K_ALPHA_FLUX, K_ALPHA_LO, K_ALPHA_LIMIT, K_ALPHA_UPDATE, K_FINALIZE, K_PROPERTIES, K_NORMALS,
  K_CURVATURE, K_MOM_ASSEMBLE, K_JACOBI, K_HBYA, K_CORRECT, K_BOUNDARY, K_STATS, K_CFL, K_STATIC,
  K_ASSEMBLE, K_DIAG, K_CONVERT, K_COARSEN, K_SMOOTH0, K_SMOOTHC, K_ZERO, K_RESTRICT0, K_RESTRICTC,
  K_PROLONG0, K_PROLONGC, K_RESID0, K_SPMV_DOT, K_UPDATE_XR, K_DOTS, K_UPDATE_D, K_TAIL, K_COUNT
};
extern const char* const kKernelNames[K_COUNT];
void prof_begin(int id, cudaStream_t s);
void prof_end(int id, cudaStream_t s);
long long launch_count();  // kernels launched so far by the active simulation

#define MDBS_LAUNCH(ID, GRID, BLOCK, STREAM, KERNEL, ...)   \
  do {                                                     \
    ::mdbs::prof_begin((ID), (STREAM));                    \
    KERNEL<<<(GRID), (BLOCK), 0, (STREAM)>>>(__VA_ARGS__); \
    ::mdbs::prof_end((ID), (STREAM));                      \
  } while (0)

// ---------------------------------------------------------------- launchers
// step_kernels.cu
// (dt, time and the statistics live in the device scalar array, see kSlot*)
void launch_alpha_step(const Prm& P, const Fld& F, double* partials, double* scal, cudaStream_t s);
void launch_properties(const Prm& P, const Fld& F, cudaStream_t s);
void launch_momentum_assemble(const Prm& P, const Fld& F, const double* scal, cudaStream_t s);
void launch_jacobi_sweeps(const Prm& P, const Fld& F, int sweeps, cudaStream_t s);  // result in F.u
void launch_hbya(const Prm& P, const Fld& F, cudaStream_t s);
void launch_correct(const Prm& P, const Fld& F, cudaStream_t s);
void launch_set_boundary_velocities(const Prm& P, const Fld& F, cudaStream_t s);
void launch_field_stats(const Prm& P, const Fld& F, double* partials, double* scal, cudaStream_t s);
void launch_time_advance(const Prm& P, const Fld& F, double cfl, double dt_max, double* partials, double* scal,
                         cudaStream_t s);
void launch_static_geometry(const Prm& P, const double* phi, uint8_t* is_free, double* nw[3], cudaStream_t s);

// pressure.cu
struct PressureSolver;
PressureSolver* pressure_create(const Prm& P, int precision, cudaError_t* err);
void pressure_destroy(PressureSolver* ps);
size_t pressure_bytes(const int n[3], int precision);
void launch_pressure_assemble(const Prm& P, const Fld& F, cudaStream_t s);
// Enqueues the solve of A p = b (level-0 arrays of F) by GMG-preconditioned CG on s.
// Iterations and the final relative residual of corrector `corr` go to
// step_scal[kSlotIters + corr] / [kSlotResid + corr] (totals accumulate).
// capture == false: the CG loop is driven from the host (one sync per iteration);
// capture == true: s is capturing a graph and the loop becomes a conditional
// WHILE node evaluated on the device.  Returns a CUDA error code.
cudaError_t pressure_solve(PressureSolver* ps, const Prm& P, const Fld& F, double tol, int max_it, int nu1,
                           int nu2, int coarse_sweeps, double* step_scal, int corr, bool capture,
                           cudaStream_t s);
// kernels in one CG iteration, as counted during the last capture
long long pressure_body_launches(const PressureSolver* ps);

}  // namespace mdbs
