// pressure.cu -- pressure equation of the PISO corrector (Eq. 53) on sm_103a:
// assembly of the 7-point (5-point in 2-D) variable-coefficient operator,
// geometric multigrid V-cycle (red-black Gauss-Seidel, cell-centred 2:1
// coarsening with series/parallel transmissibilities) and preconditioned CG in
// FP64 with deterministic block reductions.  In mixed precision the V-cycle
// runs in FP32 inside a flexible (Polak-Ribiere) FP64 CG.
#include <math.h>

#include <new>

#include "mdbs_internal.cuh"

namespace mdbs {

namespace {

int grid_for(long long n, int cap = 1 << 30) {
  long long b = (n + kBlock - 1) / kBlock;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (int)b;
}

__device__ __forceinline__ void decode3(const int n[3], long long c, int& i, int& j, int& k) {
  const unsigned uc = (unsigned)c;  // arrays stay below 2^31 entries
  i = (int)(uc % (unsigned)n[0]);
  const unsigned r = uc / (unsigned)n[0];
  j = (int)(r % (unsigned)n[1]);
  k = (int)(r / (unsigned)n[1]);
}

// ------------------------------------------------------------------ assembly
// T_f = A^2 / a_P,f between cells, 2 A^2 / a_P,f on outlet faces (Dirichlet
// through the ghost p_ghost = -p), b = -sum_f s_f A ubar_f with ubar = HbyA on
// unknown faces and the fixed velocity on wall / inlet faces.
__global__ void k_assemble(Prm P, Fld F) {
  long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= P.cells) return;
  int q[3];
  decode3(P.n, c, q[0], q[1], q[2]);
  const double A = P.A, A2 = P.A * P.A;
  double div = 0.0, Dd = 0.0;
  for (int d = 0; d < 3; d++) {
    if (d >= P.dim) {
      F.T[d][c] = 0.0;
      continue;
    }
    const int di = (d == 0), dj = (d == 1), dk = (d == 2);
    const long long flo = face_index(P.n, d, q[0], q[1], q[2]);
    const long long fhi = face_index(P.n, d, q[0] + di, q[1] + dj, q[2] + dk);
    F.T[d][c] = (q[d] + 1 < P.n[d]) ? A2 * F.aP[d][fhi] : 0.0;  // aP holds 1 / a_P
    const bool lo_bnd = q[d] == 0, hi_bnd = q[d] + 1 == P.n[d];
    if (lo_bnd && P.bc[2 * d] == kOutlet) Dd += 2.0 * A2 * F.aP[d][flo];
    if (hi_bnd && P.bc[2 * d + 1] == kOutlet) Dd += 2.0 * A2 * F.aP[d][fhi];
    const bool lo_fixed = lo_bnd && P.bc[2 * d] != kOutlet;
    const bool hi_fixed = hi_bnd && P.bc[2 * d + 1] != kOutlet;
    const double ulo = lo_fixed ? F.u[d][flo] : F.hbya[d][flo];
    const double uhi = hi_fixed ? F.u[d][fhi] : F.hbya[d][fhi];
    div += A * uhi - A * ulo;
  }
  F.Dd[c] = Dd;
  F.b[c] = -div;
}

template <typename R>
__device__ __forceinline__ R coef_lo(const Level<R>& L, int d, const int q[3], long long c) {
  if (q[d] == 0) return R(0);
  long long o = d == 0 ? 1 : (d == 1 ? (long long)L.n[0] : (long long)L.n[0] * L.n[1]);
  return L.T[d][c - o];
}

template <typename R>
__global__ void k_diag(Level<R> L) {
  long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= L.cells) return;
  int q[3];
  decode3(L.n, c, q[0], q[1], q[2]);
  R dg = R(0);
  for (int d = 0; d < 3; d++) {
    dg += L.T[d][c];
    if (q[d] > 0) dg += coef_lo(L, d, q, c);
  }
  const R dgt = dg + L.Dd[c];
  L.diag[c] = dgt;
  L.dinv[c] = R(1) / dgt;
}

__global__ void k_to_float(const double* __restrict__ a, float* __restrict__ b, long long n) {
  long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c < n) b[c] = (float)a[c];
}

__global__ void k_reciprocal_f(const float* __restrict__ a, float* __restrict__ b, long long n) {
  long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c < n) b[c] = 1.0f / a[c];
}

// coarse transmissibilities: fine rows across a coarse face in parallel, along a
// row half of each coarse cell's interior link and the crossing link in series
template <typename R>
__global__ void k_coarsen(Level<R> Fi, Level<R> Co) {
  long long ci = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (ci >= Co.cells) return;
  int Q[3];
  decode3(Co.n, ci, Q[0], Q[1], Q[2]);
  int lo[3], hi[3];
  for (int a = 0; a < 3; a++) {
    lo[a] = Co.cz[a] ? 2 * Q[a] : Q[a];
    hi[a] = Co.cz[a] ? (2 * Q[a] + 1 < Fi.n[a] ? 2 * Q[a] + 1 : 2 * Q[a]) : Q[a];
  }
  for (int d = 0; d < 3; d++) {
    if (Q[d] + 1 >= Co.n[d]) {
      Co.T[d][ci] = R(0);
      continue;
    }
    const R* Tf = Fi.T[d];
    int rl[3] = {lo[0], lo[1], lo[2]}, rh[3] = {hi[0], hi[1], hi[2]};
    rl[d] = rh[d] = 0;
    R sum = R(0);
    for (int z = rl[2]; z <= rh[2]; z++)
      for (int y = rl[1]; y <= rh[1]; y++)
        for (int x = rl[0]; x <= rh[0]; x++) {
          int fc[3] = {x, y, z};
          R inv;
          if (Co.cz[d]) {
            fc[d] = 2 * Q[d] + 1;
            const R tface = Tf[cell_index(Fi.n, fc[0], fc[1], fc[2])];
            fc[d] = 2 * Q[d];
            const R tin_l = Tf[cell_index(Fi.n, fc[0], fc[1], fc[2])];
            inv = R(1) / tface + R(1) / (R(2) * tin_l);
            if (2 * Q[d] + 3 < Fi.n[d]) {
              fc[d] = 2 * Q[d] + 2;
              inv += R(1) / (R(2) * Tf[cell_index(Fi.n, fc[0], fc[1], fc[2])]);
            }
          } else {
            fc[d] = Q[d];
            inv = R(1) / Tf[cell_index(Fi.n, fc[0], fc[1], fc[2])];
          }
          sum += R(1) / inv;
        }
    Co.T[d][ci] = sum;
  }
  R dd = R(0);
  for (int z = lo[2]; z <= hi[2]; z++)
    for (int y = lo[1]; y <= hi[1]; y++)
      for (int x = lo[0]; x <= hi[0]; x++) dd += R(0.5) * Fi.Dd[cell_index(Fi.n, x, y, z)];
  Co.Dd[ci] = dd;
}

// sum_nb T x_nb at cell c of level L (order x-, x+, y-, y+, z-, z+)
template <typename R>
__device__ __forceinline__ R neighbour_sum(const Level<R>& L, const R* __restrict__ x, const int q[3],
                                           long long c) {
  R v = R(0);
  long long o = 1;
  for (int d = 0; d < 3; d++) {
    if (q[d] > 0) v += L.T[d][c - o] * x[c - o];
    if (q[d] + 1 < L.n[d]) v += L.T[d][c] * x[c + o];
    o *= L.n[d];
  }
  return v;
}

// red-black Gauss-Seidel half sweep of colour col; zero: x is taken as 0
template <typename R>
__global__ void k_smooth(Level<R> L, int col, int zero) {
  const unsigned half = (L.n[0] + 1) >> 1;
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned rows = (unsigned)L.n[1] * (unsigned)L.n[2];
  if (t >= rows * half) return;
  const int ti = (int)(t % half);
  const unsigned row = t / half;
  const int j = (int)(row % (unsigned)L.n[1]), k = (int)(row / (unsigned)L.n[1]);
  const int i = ((j + k + col) & 1) + 2 * ti;
  if (i >= L.n[0]) return;
  const long long c = i + (long long)L.n[0] * row;
  if (zero) {
    L.x[c] = L.b[c] * L.dinv[c];
    return;
  }
  const int q[3] = {i, j, k};
  R v = L.b[c] + neighbour_sum(L, L.x, q, c);
  L.x[c] = v * L.dinv[c];
}

template <typename R>
__global__ void k_zero(R* x, long long n) {
  long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c < n) x[c] = R(0);
}

// coarse b = sum of the fine residuals b - A x over the covered fine cells
template <typename R>
__global__ void k_resid_restrict(Level<R> Fi, Level<R> Co) {
  long long ci = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (ci >= Co.cells) return;
  int Q[3];
  decode3(Co.n, ci, Q[0], Q[1], Q[2]);
  int lo[3], hi[3];
  for (int a = 0; a < 3; a++) {
    lo[a] = Co.cz[a] ? 2 * Q[a] : Q[a];
    hi[a] = Co.cz[a] ? (2 * Q[a] + 1 < Fi.n[a] ? 2 * Q[a] + 1 : 2 * Q[a]) : Q[a];
  }
  R s = R(0);
  for (int z = lo[2]; z <= hi[2]; z++)
    for (int y = lo[1]; y <= hi[1]; y++)
      for (int x = lo[0]; x <= hi[0]; x++) {
        const int q[3] = {x, y, z};
        const long long c = cell_index(Fi.n, x, y, z);
        const R ax = Fi.diag[c] * Fi.x[c] - neighbour_sum(Fi, Fi.x, q, c);
        s += Fi.b[c] - ax;
      }
  Co.b[ci] = s;
}

template <typename R>
__global__ void k_prolong(Level<R> Fi, Level<R> Co) {
  long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= Fi.cells) return;
  int q[3];
  decode3(Fi.n, c, q[0], q[1], q[2]);
  int Q[3];
  for (int a = 0; a < 3; a++) Q[a] = Co.cz[a] ? q[a] / 2 : q[a];
  Fi.x[c] += Co.x[cell_index(Co.n, Q[0], Q[1], Q[2])];
}

// ------------------------------------------------------------------ coarsest level
// The coarsest level has at most 4 x 4 x 4 cells.  Once per assembly its dense
// operator is inverted in one CTA (Gauss-Jordan in shared memory, no pivoting:
// the matrix is symmetric positive definite) and symmetrised; the V-cycle then
// solves it exactly with one dense product.
constexpr int kCoarseMax = 64;

template <typename R>
__global__ void k_coarse_inverse(Level<R> C, R* __restrict__ inv) {
  __shared__ R M[kCoarseMax * kCoarseMax];
  const int n = (int)C.cells;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) M[e] = R(0);
  __syncthreads();
  for (int c = threadIdx.x; c < n; c += blockDim.x) {
    int q[3];
    q[0] = c % C.n[0];
    q[1] = (c / C.n[0]) % C.n[1];
    q[2] = c / (C.n[0] * C.n[1]);
    M[c * n + c] = C.diag[c];
    int o = 1;
    for (int d = 0; d < 3; d++) {
      if (q[d] + 1 < C.n[d]) {
        M[c * n + c + o] = -C.T[d][c];
        M[(c + o) * n + c] = -C.T[d][c];
      }
      o *= C.n[d];
    }
  }
  __syncthreads();
  for (int k = 0; k < n; k++) {
    const R pinv = R(1) / M[k * n + k];
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += blockDim.x)
      if (j != k) M[k * n + j] *= pinv;
    __syncthreads();
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
      const int i = e / n, j = e % n;
      if (i != k && j != k) M[e] -= M[i * n + k] * M[k * n + j];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x)
      if (i != k) M[i * n + k] = -M[i * n + k] * pinv;
    if (threadIdx.x == 0) M[k * n + k] = pinv;
    __syncthreads();
  }
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e % n;
    inv[e] = R(0.5) * (M[i * n + j] + M[j * n + i]);
  }
}

// ------------------------------------------------------------------ tail V-cycle
// The small levels (and the coarsest solve) of a V-cycle in one CTA: the same
// per-cell arithmetic, in the same order, as the per-level kernels above, with
// __syncthreads() between phases instead of kernel boundaries.
constexpr int kTailCells = 4096;
constexpr int kTailThreads = 1024;

template <typename R>
struct Tail {
  Level<R> lv[kMaxLevels];
  int first, nlev, nu1, nu2, cs;
  const R* cinv;  // inverse of the coarsest operator (used when cs == 0)
};

template <typename R>
__device__ void tail_smooth(const Level<R>& L, int col, int zero) {
  const unsigned half = (L.n[0] + 1) >> 1;
  const unsigned total = half * (unsigned)L.n[1] * (unsigned)L.n[2];
  for (unsigned t = threadIdx.x; t < total; t += blockDim.x) {
    const unsigned ti = t % half, row = t / half;
    const int j = (int)(row % (unsigned)L.n[1]), k = (int)(row / (unsigned)L.n[1]);
    const int i = ((j + k + col) & 1) + 2 * (int)ti;
    if (i >= L.n[0]) continue;
    const long long c = i + (long long)L.n[0] * row;
    if (zero) {
      L.x[c] = L.b[c] * L.dinv[c];
    } else {
      const int q[3] = {i, j, k};
      R v = L.b[c] + neighbour_sum(L, L.x, q, c);
      L.x[c] = v * L.dinv[c];
    }
  }
  __syncthreads();
}

template <typename R>
__device__ void tail_pair(const Level<R>& L, int first_col, bool zero_first) {
  tail_smooth(L, first_col, zero_first ? 1 : 0);
  tail_smooth(L, 1 - first_col, 0);
}

template <typename R>
__device__ void tail_zero(const Level<R>& L) {
  for (unsigned c = threadIdx.x; c < (unsigned)L.cells; c += blockDim.x) L.x[c] = R(0);
  __syncthreads();
}

template <typename R>
__device__ void tail_restrict(const Level<R>& Fi, const Level<R>& Co) {
  for (unsigned ci = threadIdx.x; ci < (unsigned)Co.cells; ci += blockDim.x) {
    int Q[3];
    Q[0] = (int)(ci % (unsigned)Co.n[0]);
    const unsigned r = ci / (unsigned)Co.n[0];
    Q[1] = (int)(r % (unsigned)Co.n[1]);
    Q[2] = (int)(r / (unsigned)Co.n[1]);
    int lo[3], hi[3];
    for (int a = 0; a < 3; a++) {
      lo[a] = Co.cz[a] ? 2 * Q[a] : Q[a];
      hi[a] = Co.cz[a] ? (2 * Q[a] + 1 < Fi.n[a] ? 2 * Q[a] + 1 : 2 * Q[a]) : Q[a];
    }
    R s = R(0);
    for (int z = lo[2]; z <= hi[2]; z++)
      for (int y = lo[1]; y <= hi[1]; y++)
        for (int x = lo[0]; x <= hi[0]; x++) {
          const int q[3] = {x, y, z};
          const long long c = cell_index(Fi.n, x, y, z);
          const R ax = Fi.diag[c] * Fi.x[c] - neighbour_sum(Fi, Fi.x, q, c);
          s += Fi.b[c] - ax;
        }
    Co.b[ci] = s;
  }
  __syncthreads();
}

template <typename R>
__device__ void tail_prolong(const Level<R>& Fi, const Level<R>& Co) {
  for (unsigned c = threadIdx.x; c < (unsigned)Fi.cells; c += blockDim.x) {
    int q[3];
    q[0] = (int)(c % (unsigned)Fi.n[0]);
    const unsigned r = c / (unsigned)Fi.n[0];
    q[1] = (int)(r % (unsigned)Fi.n[1]);
    q[2] = (int)(r / (unsigned)Fi.n[1]);
    int Q[3];
    for (int a = 0; a < 3; a++) Q[a] = Co.cz[a] ? q[a] / 2 : q[a];
    Fi.x[c] += Co.x[cell_index(Co.n, Q[0], Q[1], Q[2])];
  }
  __syncthreads();
}

template <typename R>
__global__ void __launch_bounds__(kTailThreads) k_tail_vcycle(Tail<R> t) {
  for (int l = t.first; l < t.nlev - 1; l++) {
    if (t.nu1 == 0) tail_zero(t.lv[l]);
    for (int it = 0; it < t.nu1; it++) tail_pair(t.lv[l], 0, it == 0);
    tail_restrict(t.lv[l], t.lv[l + 1]);
  }
  const Level<R>& C = t.lv[t.nlev - 1];
  if (t.cs == 0) {
    const int n = (int)C.cells;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      R v = R(0);
      for (int j = 0; j < n; j++) v += t.cinv[i * n + j] * C.b[j];
      C.x[i] = v;
    }
    __syncthreads();
  }
  for (int it = 0; it < t.cs; it++) tail_pair(C, 0, it == 0);
  for (int it = 0; it < t.cs; it++) tail_pair(C, 1, false);
  for (int l = t.nlev - 2; l >= t.first; l--) {
    tail_prolong(t.lv[l], t.lv[l + 1]);
    for (int it = 0; it < t.nu2; it++) tail_pair(t.lv[l], 1, false);
  }
}

// ------------------------------------------------------------------ CG kernels (FP64)
__device__ __forceinline__ double apply_A0(const Fld& F, const Prm& P, const double* __restrict__ x, long long c,
                                           const int q[3]) {
  double v = F.diag[c] * x[c];
  long long o = 1;
  for (int d = 0; d < 3; d++) {
    if (q[d] > 0) v -= F.T[d][c - o] * x[c - o];
    if (q[d] + 1 < P.n[d]) v -= F.T[d][c] * x[c + o];
    o *= P.n[d];
  }
  return v;
}

// r = b - A x; partial sums of r.r and b.b
__global__ void k_resid0(Prm P, Fld F, const double* __restrict__ x, double* __restrict__ r,
                         double* __restrict__ partials, int nb) {
  double rr = 0.0, bb = 0.0;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < P.cells;
       c += (long long)gridDim.x * blockDim.x) {
    int q[3];
    decode3(P.n, c, q[0], q[1], q[2]);
    const double bc = F.b[c];
    const double rc = bc - apply_A0(F, P, x, c, q);
    r[c] = rc;
    rr += rc * rc;
    bb += bc * bc;
  }
  rr = block_sum(rr);
  if (threadIdx.x == 0) partials[blockIdx.x] = rr;
  bb = block_sum(bb);
  if (threadIdx.x == 0) partials[nb + blockIdx.x] = bb;
}

// q = A d; partial d.q
__global__ void k_spmv_dot(Prm P, Fld F, const double* __restrict__ dv, double* __restrict__ q,
                           double* __restrict__ partials) {
  double s = 0.0;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < P.cells;
       c += (long long)gridDim.x * blockDim.x) {
    int qq[3];
    decode3(P.n, c, qq[0], qq[1], qq[2]);
    const double v = apply_A0(F, P, dv, c, qq);
    q[c] = v;
    s += dv[c] * v;
  }
  s = block_sum(s);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// x += alpha d; r -= alpha q; partial r.r   (alpha = scal[5])
__global__ void k_update_xr(long long n, const double* __restrict__ scal, double* __restrict__ x,
                            double* __restrict__ r, const double* __restrict__ dv, const double* __restrict__ q,
                            double* __restrict__ partials) {
  const double al = scal[5];
  double s = 0.0;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
       c += (long long)gridDim.x * blockDim.x) {
    x[c] += al * dv[c];
    const double rc = r[c] - al * q[c];
    r[c] = rc;
    s += rc * rc;
  }
  s = block_sum(s);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// partial r.z and z.q
__global__ void k_dots_rz(long long n, const double* __restrict__ r, const double* __restrict__ z,
                          const double* __restrict__ q, double* __restrict__ partials, int nb, int with_zq) {
  double rz = 0.0, zq = 0.0;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
       c += (long long)gridDim.x * blockDim.x) {
    rz += r[c] * z[c];
    if (with_zq) zq += z[c] * q[c];
  }
  rz = block_sum(rz);
  if (threadIdx.x == 0) partials[blockIdx.x] = rz;
  if (with_zq) {
    zq = block_sum(zq);
    if (threadIdx.x == 0) partials[nb + blockIdx.x] = zq;
  }
}

// CG scalars on the device
constexpr int kBB = 0, kRR = 1, kRZ = 2, kDQ = 3, kZQ = 4, kAlpha = 5, kCond = 6, kRZold = 7, kIt = 8;

// d = z + beta d; the first iteration (counter 0) takes d = z
__global__ void k_update_d(long long n, const double* __restrict__ scal, const double* __restrict__ z,
                           double* __restrict__ dv, int flexible) {
  const bool first = scal[kIt] == 0.0;
  double be = 0.0;
  if (!first) be = flexible ? -scal[kAlpha] * scal[kZQ] / scal[kRZold] : scal[kRZ] / scal[kRZold];
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
       c += (long long)gridDim.x * blockDim.x)
    dv[c] = first ? z[c] : z[c] + be * dv[c];
}

// Scalar finalizers (one block, fixed summation order).  The loop condition
// "not converged, below max_it, finite" is written to scal[kCond] and, inside a
// captured graph, to the WHILE node's conditional handle.
// mode 0: rr, bb after the initial residual; iteration counter = 0
// mode 1: dq, alpha = rz / dq
// mode 2: rr after the update; counter += 1
// mode 3: rz_old = rz; rz (and zq when two channels)
__global__ void k_finalize(const double* __restrict__ partials, int nb, double* scal, int mode, int two,
                           double tol, int max_it, cudaGraphConditionalHandle handle, int use_handle) {
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    a += partials[i];
    if (two) b += partials[nb + i];
  }
  a = block_sum(a);
  if (two) b = block_sum(b);
  if (threadIdx.x != 0) return;
  if (mode == 1) {
    scal[kDQ] = a;
    scal[kAlpha] = scal[kRZ] / a;
    return;
  }
  if (mode == 3) {
    scal[kRZold] = scal[kRZ];
    scal[kRZ] = a;
    scal[kZQ] = two ? b : 0.0;
    return;
  }
  double it;
  if (mode == 0) {
    scal[kRR] = a;
    scal[kBB] = b;
    it = 0.0;
  } else {
    scal[kRR] = a;
    it = scal[kIt] + 1.0;
  }
  scal[kIt] = it;
  const double bb = scal[kBB];
  const bool done = bb == 0.0 || sqrt(a) <= tol * sqrt(bb) || it >= (double)max_it || !(a == a);
  scal[kCond] = done ? 0.0 : 1.0;
  if (use_handle) cudaGraphSetConditional(handle, done ? 0u : 1u);
}

// b = 0 has the solution p = 0 whatever the initial guess
__global__ void k_zero_if_b0(long long n, const double* __restrict__ scal, double* __restrict__ x) {
  if (scal[kBB] != 0.0) return;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
       c += (long long)gridDim.x * blockDim.x)
    x[c] = 0.0;
}

// iterations and relative residual of corrector corr into the step scalars
__global__ void k_record(const double* __restrict__ scal, double* step, int corr, double tol) {
  if (threadIdx.x != 0) return;
  const double bb = scal[kBB];
  const double res = bb == 0.0 ? 0.0 : sqrt(scal[kRR] / bb);
  step[kSlotIters + corr] = scal[kIt];
  step[kSlotResid + corr] = res;
  step[kSlotItersTotal] += scal[kIt];
  if (!(res <= tol)) step[kSlotNotConverged] += 1.0;
}

__global__ void k_copy_d2f(const double* __restrict__ a, float* __restrict__ b, long long n) {
  long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c < n) b[c] = (float)a[c];
}
__global__ void k_copy_f2d(const float* __restrict__ a, double* __restrict__ b, long long n) {
  long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c < n) b[c] = (double)a[c];
}

}  // namespace

// ------------------------------------------------------------------ solver object
struct PressureSolver {
  int precision;
  int nlev;
  Level<double> ld[kMaxLevels];  // FP64 hierarchy (level 0 arrays are borrowed)
  Level<float> lf[kMaxLevels];   // FP32 hierarchy (mixed precision)
  double *r, *z, *dv, *q;
  double* partials;
  double* scal;
  double* host_scal;  // pinned
  double* cinv_d;     // inverse of the coarsest operator (FP64 hierarchy)
  float* cinv_f;      // (FP32 hierarchy)
  void* block;        // single device allocation
  cudaStream_t body_stream;  // captures the body of the CG WHILE node
  long long body_launches;   // kernels per CG iteration (counted while capturing)
};

long long pressure_body_launches(const PressureSolver* ps) { return ps->body_launches; }

static int plan_levels(const int n0[3], int dims[kMaxLevels][3], int cz[kMaxLevels][3]) {
  int nlev = 1;
  for (int a = 0; a < 3; a++) {
    dims[0][a] = n0[a];
    cz[0][a] = 0;
  }
  while (nlev < kMaxLevels) {
    int changed = 0;
    for (int a = 0; a < 3; a++) {
      if (dims[nlev - 1][a] > 4) {
        dims[nlev][a] = (dims[nlev - 1][a] + 1) / 2;
        cz[nlev][a] = 1;
        changed = 1;
      } else {
        dims[nlev][a] = dims[nlev - 1][a];
        cz[nlev][a] = 0;
      }
    }
    if (!changed) break;
    nlev++;
  }
  return nlev;
}

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

static size_t solver_layout(const int n[3], int precision, PressureSolver* ps, char* base) {
  int dims[kMaxLevels][3], cz[kMaxLevels][3];
  const int nlev = plan_levels(n, dims, cz);
  size_t off = 0;
  auto take = [&](size_t bytes) -> char* {
    char* p = base ? base + off : nullptr;
    off += align256(bytes);
    return p;
  };
  const long long n0 = (long long)n[0] * n[1] * n[2];
  if (ps) ps->nlev = nlev;
  double* r = (double*)take(n0 * 8);
  double* z = (double*)take(n0 * 8);
  double* dv = (double*)take(n0 * 8);
  double* q = (double*)take(n0 * 8);
  double* partials = (double*)take(2 * kMaxPartials * 8);
  double* scal = (double*)take(16 * 8);
  double* cinv_d = (double*)take(kCoarseMax * kCoarseMax * 8);
  float* cinv_f = (float*)take(kCoarseMax * kCoarseMax * 4);
  if (ps) {
    ps->r = r;
    ps->z = z;
    ps->dv = dv;
    ps->q = q;
    ps->partials = partials;
    ps->scal = scal;
    ps->cinv_d = cinv_d;
    ps->cinv_f = cinv_f;
  }
  for (int l = 0; l < nlev; l++) {
    const long long nc = (long long)dims[l][0] * dims[l][1] * dims[l][2];
    if (precision == 0) {
      Level<double> L{};
      for (int a = 0; a < 3; a++) {
        L.n[a] = dims[l][a];
        L.cz[a] = cz[l][a];
      }
      L.cells = nc;
      if (l > 0) {
        for (int a = 0; a < 3; a++) L.T[a] = (double*)take(nc * 8);
        L.Dd = (double*)take(nc * 8);
        L.diag = (double*)take(nc * 8);
        L.dinv = (double*)take(nc * 8);
        L.x = (double*)take(nc * 8);
        L.b = (double*)take(nc * 8);
      }
      if (ps) ps->ld[l] = L;
    } else {
      Level<float> L{};
      for (int a = 0; a < 3; a++) {
        L.n[a] = dims[l][a];
        L.cz[a] = cz[l][a];
      }
      L.cells = nc;
      for (int a = 0; a < 3; a++) L.T[a] = (float*)take(nc * 4);
      L.Dd = (float*)take(nc * 4);
      L.diag = (float*)take(nc * 4);
      L.dinv = (float*)take(nc * 4);
      L.x = (float*)take(nc * 4);
      L.b = (float*)take(nc * 4);
      if (ps) ps->lf[l] = L;
    }
  }
  return off;
}

size_t pressure_bytes(const int n[3], int precision) { return solver_layout(n, precision, nullptr, nullptr); }

PressureSolver* pressure_create(const Prm& P, int precision, cudaError_t* err) {
  PressureSolver* ps = new (std::nothrow) PressureSolver();
  if (!ps) {
    *err = cudaErrorMemoryAllocation;
    return nullptr;
  }
  ps->precision = precision == 0 ? 0 : 1;
  {
    int dims[kMaxLevels][3], cz[kMaxLevels][3];
    const int nl = plan_levels(P.n, dims, cz);
    if ((long long)dims[nl - 1][0] * dims[nl - 1][1] * dims[nl - 1][2] > kCoarseMax) {
      *err = cudaErrorInvalidValue;  // coarsest level larger than the dense solver handles
      delete ps;
      return nullptr;
    }
  }
  size_t bytes = solver_layout(P.n, ps->precision, nullptr, nullptr);
  *err = cudaMalloc(&ps->block, bytes);
  if (*err != cudaSuccess) {
    delete ps;
    return nullptr;
  }
  *err = cudaMallocHost(&ps->host_scal, 16 * sizeof(double));
  if (*err != cudaSuccess) {
    cudaFree(ps->block);
    delete ps;
    return nullptr;
  }
  *err = cudaStreamCreateWithFlags(&ps->body_stream, cudaStreamNonBlocking);
  if (*err != cudaSuccess) {
    cudaFreeHost(ps->host_scal);
    cudaFree(ps->block);
    delete ps;
    return nullptr;
  }
  solver_layout(P.n, ps->precision, ps, (char*)ps->block);
  return ps;
}

void pressure_destroy(PressureSolver* ps) {
  if (!ps) return;
  cudaStreamDestroy(ps->body_stream);
  cudaFree(ps->block);
  cudaFreeHost(ps->host_scal);
  delete ps;
}

void launch_pressure_assemble(const Prm& P, const Fld& F, cudaStream_t s) {
  MDBS_LAUNCH(K_ASSEMBLE, grid_for(P.cells), kBlock, s, k_assemble, P, F);
  Level<double> L0{};
  for (int a = 0; a < 3; a++) {
    L0.n[a] = P.n[a];
    L0.T[a] = F.T[a];
  }
  L0.cells = P.cells;
  L0.Dd = F.Dd;
  L0.diag = F.diag;
  L0.dinv = F.dinv;
  MDBS_LAUNCH(K_DIAG, grid_for(P.cells), kBlock, s, k_diag<double>, L0);
}

template <typename R>
static void build_hierarchy(Level<R>* lv, int nlev, R* cinv, bool direct, cudaStream_t s) {
  for (int l = 1; l < nlev; l++) {
    MDBS_LAUNCH(K_COARSEN, grid_for(lv[l].cells), kBlock, s, k_coarsen<R>, lv[l - 1], lv[l]);
    MDBS_LAUNCH(K_DIAG, grid_for(lv[l].cells), kBlock, s, k_diag<R>, lv[l]);
  }
  if (direct) MDBS_LAUNCH(K_COARSEN, 1, 256, s, k_coarse_inverse<R>, lv[nlev - 1], cinv);
}

template <typename R>
static void smooth_pair(const Level<R>& L, int first_col, bool zero_first, bool finest, cudaStream_t s) {
  const int id = finest ? K_SMOOTH0 : K_SMOOTHC;
  const long long threads = (long long)((L.n[0] + 1) >> 1) * L.n[1] * L.n[2];
  MDBS_LAUNCH(id, grid_for(threads), kBlock, s, k_smooth<R>, L, first_col, zero_first ? 1 : 0);
  MDBS_LAUNCH(id, grid_for(threads), kBlock, s, k_smooth<R>, L, 1 - first_col, 0);
}

// symmetric V-cycle, x of level 0 receives M b of level 0; the levels from the
// first one with at most kTailCells cells run in the single-CTA tail kernel
template <typename R>
static void vcycle(Level<R>* lv, int nlev, int nu1, int nu2, int cs, const R* cinv, cudaStream_t s) {
  int first = nlev - 1;
  while (first > 0 && lv[first - 1].cells <= kTailCells) first--;
  for (int l = 0; l < first; l++) {
    if (nu1 == 0) MDBS_LAUNCH(K_ZERO, grid_for(lv[l].cells), kBlock, s, k_zero<R>, lv[l].x, lv[l].cells);
    for (int it = 0; it < nu1; it++) smooth_pair(lv[l], 0, it == 0, l == 0, s);
    MDBS_LAUNCH(l == 0 ? K_RESTRICT0 : K_RESTRICTC, grid_for(lv[l + 1].cells), kBlock, s, k_resid_restrict<R>, lv[l], lv[l + 1]);
  }
  Tail<R> t;
  for (int l = 0; l < nlev; l++) t.lv[l] = lv[l];
  t.first = first;
  t.nlev = nlev;
  t.nu1 = nu1;
  t.nu2 = nu2;
  t.cs = cs;
  t.cinv = cinv;
  MDBS_LAUNCH(K_TAIL, 1, kTailThreads, s, k_tail_vcycle<R>, t);
  for (int l = first - 1; l >= 0; l--) {
    MDBS_LAUNCH(l == 0 ? K_PROLONG0 : K_PROLONGC, grid_for(lv[l].cells), kBlock, s, k_prolong<R>, lv[l], lv[l + 1]);
    for (int it = 0; it < nu2; it++) smooth_pair(lv[l], 1, false, l == 0, s);
  }
}

cudaError_t pressure_solve(PressureSolver* ps, const Prm& P, const Fld& F, double tol, int max_it, int nu1,
                           int nu2, int cs, double* step_scal, int corr, bool capture, cudaStream_t s) {
  const long long n = P.cells;
  const int nb = grid_for(n, kMaxPartials);
  const int flexible = ps->precision != 0;
  double* x = F.p;
  // hierarchy for this assembly
  if (!flexible) {
    Level<double>& L0 = ps->ld[0];
    for (int a = 0; a < 3; a++) L0.T[a] = F.T[a];
    L0.Dd = F.Dd;
    L0.diag = F.diag;
    L0.dinv = F.dinv;
    L0.b = ps->r;
    L0.x = ps->z;
    build_hierarchy(ps->ld, ps->nlev, ps->cinv_d, cs == 0, s);
  } else {
    Level<float>& L0 = ps->lf[0];
    const int g = grid_for(n);
    for (int a = 0; a < 3; a++) MDBS_LAUNCH(K_CONVERT, g, kBlock, s, k_to_float, F.T[a], L0.T[a], n);
    MDBS_LAUNCH(K_CONVERT, g, kBlock, s, k_to_float, F.Dd, L0.Dd, n);
    MDBS_LAUNCH(K_CONVERT, g, kBlock, s, k_to_float, F.diag, L0.diag, n);
    MDBS_LAUNCH(K_CONVERT, g, kBlock, s, k_reciprocal_f, L0.diag, L0.dinv, n);
    build_hierarchy(ps->lf, ps->nlev, ps->cinv_f, cs == 0, s);
  }
  cudaGraphConditionalHandle handle = 0;
  cudaGraph_t graph = nullptr;
  if (capture) {
    cudaStreamCaptureStatus st;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    cudaError_t e = cudaStreamGetCaptureInfo(s, &st, nullptr, &graph, &deps, nullptr, &ndeps);
    if (e != cudaSuccess) return e;
    if (st != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureInvalidated;
    e = cudaGraphConditionalHandleCreate(&handle, graph, 0, 0);
    if (e != cudaSuccess) return e;
  }
  const int use = capture ? 1 : 0;
  // initial residual and loop condition
  MDBS_LAUNCH(K_RESID0, nb, kBlock, s, k_resid0, P, F, x, ps->r, ps->partials, nb);
  MDBS_LAUNCH(K_FINALIZE, 1, 1024, s, k_finalize, ps->partials, nb, ps->scal, 0, 1, tol, max_it, handle, use);
  MDBS_LAUNCH(K_ZERO, nb, kBlock, s, k_zero_if_b0, n, ps->scal, x);
  // one CG iteration, preconditioner first; the last finalizer decides whether to continue
  auto body = [&](cudaStream_t bs) {
    if (!flexible) {
      vcycle(ps->ld, ps->nlev, nu1, nu2, cs, (const double*)ps->cinv_d, bs);
    } else {
      const int g = grid_for(n);
      MDBS_LAUNCH(K_CONVERT, g, kBlock, bs, k_copy_d2f, ps->r, ps->lf[0].b, n);
      vcycle(ps->lf, ps->nlev, nu1, nu2, cs, (const float*)ps->cinv_f, bs);
      MDBS_LAUNCH(K_CONVERT, g, kBlock, bs, k_copy_f2d, ps->lf[0].x, ps->z, n);
    }
    MDBS_LAUNCH(K_DOTS, nb, kBlock, bs, k_dots_rz, n, ps->r, ps->z, ps->q, ps->partials, nb, flexible);
    MDBS_LAUNCH(K_FINALIZE, 1, 1024, bs, k_finalize, ps->partials, nb, ps->scal, 3, flexible, tol, max_it,
                handle, use);
    MDBS_LAUNCH(K_UPDATE_D, nb, kBlock, bs, k_update_d, n, ps->scal, ps->z, ps->dv, flexible);
    MDBS_LAUNCH(K_SPMV_DOT, nb, kBlock, bs, k_spmv_dot, P, F, ps->dv, ps->q, ps->partials);
    MDBS_LAUNCH(K_FINALIZE, 1, 1024, bs, k_finalize, ps->partials, nb, ps->scal, 1, 0, tol, max_it, handle, use);
    MDBS_LAUNCH(K_UPDATE_XR, nb, kBlock, bs, k_update_xr, n, ps->scal, x, ps->r, ps->dv, ps->q, ps->partials);
    MDBS_LAUNCH(K_FINALIZE, 1, 1024, bs, k_finalize, ps->partials, nb, ps->scal, 2, 0, tol, max_it, handle, use);
  };
  if (capture) {
    cudaStreamCaptureStatus st;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    cudaError_t e = cudaStreamGetCaptureInfo(s, &st, nullptr, &graph, &deps, nullptr, &ndeps);
    if (e != cudaSuccess) return e;
    cudaGraphNodeParams prm = {};
    prm.type = cudaGraphNodeTypeConditional;
    prm.conditional.handle = handle;
    prm.conditional.type = cudaGraphCondTypeWhile;
    prm.conditional.size = 1;
    cudaGraphNode_t node;
    e = cudaGraphAddNode(&node, graph, deps, nullptr, ndeps, &prm);
    if (e != cudaSuccess) return e;
    cudaGraph_t body_graph = prm.conditional.phGraph_out[0];
    e = cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
    if (e != cudaSuccess) return e;
    e = cudaStreamBeginCaptureToGraph(ps->body_stream, body_graph, nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    const long long c0 = launch_count();
    body(ps->body_stream);
    ps->body_launches = launch_count() - c0;
    cudaGraph_t out = nullptr;
    e = cudaStreamEndCapture(ps->body_stream, &out);
    if (e != cudaSuccess) return e;
  } else {
    for (;;) {
      cudaError_t e = cudaMemcpyAsync(ps->host_scal, ps->scal + kCond, sizeof(double), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) return e;
      if (ps->host_scal[0] == 0.0) break;
      body(s);
    }
  }
  MDBS_LAUNCH(K_FINALIZE, 1, 32, s, k_record, ps->scal, step_scal, corr, tol);
  return cudaGetLastError();
}

}  // namespace mdbs
