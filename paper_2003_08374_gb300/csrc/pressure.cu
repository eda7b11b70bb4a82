// pressure.cu -- pressure equation of the PISO corrector (Eq. 53) on sm_103a:
// assembly of the 7-point (5-point in 2-D) variable-coefficient operator,
// geometric multigrid V-cycle (red-black Gauss-Seidel, cell-centred 2:1
// coarsening with halved Galerkin transmissibilities) and preconditioned CG in
// FP64 with deterministic block reductions.  In mixed precision the V-cycle
// runs in FP32 inside a flexible (Polak-Ribiere) FP64 CG.  Every kernel runs over
// all domains of a batch (see mdbs_internal.cuh); per-domain CG scalars and
// convergence flags let converged domains drop out of the remaining iterations.
#include <cudaTypedefs.h>  // PFN_cuTensorMapEncodeTiled
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <new>
#include <type_traits>
#include <vector>

#include "mdbs_internal.cuh"

namespace mdbs {

namespace {



// ------------------------------------------------------------------ x-split storage
// Every array of the pressure system (the assembled coefficients and right-hand
// side, the CG vectors and every multigrid level) stores each x-row with its even
// cells first and its odd cells after them: cell (i, j, k) sits at
// n0 (j + n1 k) + (i even ? i / 2 : he + i / 2), he = ceil(n0 / 2).  One colour of a
// red-black sweep and all its neighbours are then contiguous runs (a natural
// layout makes every sweep read stride-2, wasting half of each sector).  The
// pressure field p keeps the natural x-fastest order.
__device__ __forceinline__ unsigned xs_px(unsigned he, int i) {
  return (i & 1) ? he + (unsigned)(i >> 1) : (unsigned)(i >> 1);
}
__device__ __forceinline__ unsigned lpos(const int n[3], int i, int j, int k) {
  return (unsigned)n[0] * ((unsigned)j + (unsigned)n[1] * (unsigned)k) + xs_px((unsigned)(n[0] + 1) >> 1, i);
}
// storage position -> cell, with the divisions by n[0] and n[1] done by multiplication
__device__ __forceinline__ void decode_pos(const int n[3], FastDiv dn0, FastDiv dn1, long long c, int& i, int& j,
                                           int& k) {
  const unsigned uc = (unsigned)c, n0 = (unsigned)n[0];
  const unsigned row = fastdiv(uc, dn0), r = uc - row * n0, he = (n0 + 1) >> 1;
  i = (int)(r < he ? 2 * r : 2 * (r - he) + 1);
  const unsigned kk = fastdiv(row, dn1);
  j = (int)(row - kk * (unsigned)n[1]);
  k = (int)kk;
}
template <typename R>
__device__ __forceinline__ void decode_pos(const Level<R>& L, long long c, int& i, int& j, int& k) {
  decode_pos(L.n, L.dn0, L.dn1, c, i, j, k);
}
__device__ __forceinline__ void decode_pos(const Prm& P, long long c, int& i, int& j, int& k) {
  decode_pos(P.n, P.dn0, P.dn1, c, i, j, k);
}
__device__ __forceinline__ void decode_pos(const int n[3], long long c, int& i, int& j, int& k) {
  const unsigned uc = (unsigned)c, n0 = (unsigned)n[0];
  const unsigned row = uc / n0, r = uc - row * n0, he = (n0 + 1) >> 1;
  i = (int)(r < he ? 2 * r : 2 * (r - he) + 1);
  j = (int)(row % (unsigned)n[1]);
  k = (int)(row / (unsigned)n[1]);
}
// position of the neighbour of cell q (at position c) one cell down / up along d
__device__ __forceinline__ unsigned lo_pos(const int n[3], const int q[3], unsigned c, int d) {
  return d == 0 ? lpos(n, q[0] - 1, q[1], q[2]) : (d == 1 ? c - (unsigned)n[0] : c - (unsigned)n[0] * (unsigned)n[1]);
}
__device__ __forceinline__ unsigned hi_pos(const int n[3], const int q[3], unsigned c, int d) {
  return d == 0 ? lpos(n, q[0] + 1, q[1], q[2]) : (d == 1 ? c + (unsigned)n[0] : c + (unsigned)n[0] * (unsigned)n[1]);
}

// the FP64 or FP32 hierarchy of a domain
template <typename R>
__device__ __forceinline__ const Level<R>* levels_of(const CgDom& C);
template <>
__device__ __forceinline__ const Level<double>* levels_of<double>(const CgDom& C) { return C.ld; }
template <>
__device__ __forceinline__ const Level<float>* levels_of<float>(const CgDom& C) { return C.lf; }

// ---------------------------------------------------------------- coefficient storage
// FP32 / FP64 coefficients, or BF16 bit patterns widened exactly to FP32 on load.
template <typename R>
struct CoefF {
  const R* __restrict__ p;
  __device__ __forceinline__ R operator[](unsigned i) const { return p[i]; }
};
struct CoefH {
  const uint16_t* __restrict__ p;
  __device__ __forceinline__ float operator[](unsigned i) const { return __uint_as_float((unsigned)p[i] << 16); }
};

// coefficient d of level L at cell i, whatever its storage
template <typename R>
__device__ __forceinline__ R tcoef(const Level<R>& L, int d, unsigned i) {
  if constexpr (std::is_same<R, float>::value)
    if (L.Tb[d]) return __uint_as_float((unsigned)L.Tb[d][i] << 16);
  return L.T[d][i];
}

// stores coefficient d of level L at cell i (BF16: rounded to nearest even)
template <typename R>
__device__ __forceinline__ void tstore(const Level<R>& L, int d, unsigned i, R v) {
  if constexpr (std::is_same<R, float>::value)
    if (L.Tb[d]) {
      L.Tb[d][i] = __bfloat16_as_ushort(__float2bfloat16_rn(v));
      return;
    }
  L.T[d][i] = v;
}

// calls f with the three coefficient readers of level L
template <typename R, typename F>
__device__ __forceinline__ void with_coefs(const Level<R>& L, F&& f) {
  if constexpr (std::is_same<R, float>::value)
    if (L.Tb[0]) {
      f(CoefH{L.Tb[0]}, CoefH{L.Tb[1]}, CoefH{L.Tb[2]});
      return;
    }
  f(CoefF<R>{L.T[0]}, CoefF<R>{L.T[1]}, CoefF<R>{L.T[2]});
}

// CG scalars on the device
constexpr int kBB = 0, kRR = 1, kRZ = 2, kDQ = 3, kZQ = 4, kAlpha = 5, kCond = 6, kRZold = 7, kIt = 8;

#define FOR_WORK(W)                                   \
  for (int b_ = blockIdx.x; b_ < (W).total; b_ += gridDim.x) { \
    const int dm = work_domain((W), b_);              \
    const int lb = b_ - (W).blk[dm];

// The same walk with the item order reversed when REV != 0.  Consecutive kernels
// over one level alternate direction, so that each starts on the cache lines the
// previous one touched last (still in L2).  Every item computes the same values,
// and writes the same partial, in either order.
#define FOR_WORK_DIR(W, REV)                                              \
  for (int i_ = blockIdx.x; i_ < (W).total; i_ += gridDim.x) {            \
    const int b_ = (REV) ? (W).total - 1 - i_ : i_;                        \
    const int dm = work_domain((W), b_);                                  \
    const int lb = b_ - (W).blk[dm];

// ------------------------------------------------------------------ assembly
// T_f = A^2 / a_P,f between cells, 2 A^2 / a_P,f on outlet faces (Dirichlet
// through the ghost p_ghost = -p), b = -sum_f s_f A ubar_f with ubar = HbyA on
// unknown faces and the fixed velocity on wall / inlet faces.
// what: kAsmMatrix (coefficients T, Dd) and / or kAsmRhs (right-hand side b)
__device__ __forceinline__ void b_assemble(const Prm& P, const Fld& F, long long c, int what) {
  const bool matrix = what & kAsmMatrix;
  int q[3];
  decode_pos(P, c, q[0], q[1], q[2]);  // c: storage position of the cell
  const double A = P.A, A2 = P.A * P.A;
  double div = 0.0, Dd = 0.0;
  for (int d = 0; d < 3; d++) {
    if (d >= P.dim) {
      if (matrix) F.T[d][c] = 0.0;
      continue;
    }
    const int di = (d == 0), dj = (d == 1), dk = (d == 2);
    const long long flo = face_index(P.n, d, q[0], q[1], q[2]);
    const long long fhi = face_index(P.n, d, q[0] + di, q[1] + dj, q[2] + dk);
    if (matrix) F.T[d][c] = (q[d] + 1 < P.n[d]) ? A2 * F.aP[d][fhi] : 0.0;  // aP holds 1 / a_P
    const bool lo_bnd = q[d] == 0, hi_bnd = q[d] + 1 == P.n[d];
    if (lo_bnd && P.bc[2 * d] == kOutlet) Dd += 2.0 * A2 * F.aP[d][flo];
    if (hi_bnd && P.bc[2 * d + 1] == kOutlet) Dd += 2.0 * A2 * F.aP[d][fhi];
    const bool lo_fixed = lo_bnd && P.bc[2 * d] != kOutlet;
    const bool hi_fixed = hi_bnd && P.bc[2 * d + 1] != kOutlet;
    const double ulo = lo_fixed ? F.u[d][flo] : F.hbya[d][flo];
    const double uhi = hi_fixed ? F.u[d][fhi] : F.hbya[d][fhi];
    div += A * uhi - A * ulo;
  }
  if (matrix) F.Dd[c] = Dd;
  if (what & kAsmRhs) F.b[c] = -div;
}

__global__ void k_assemble(const StepDom* __restrict__ D, Work w, int what) {
  MDBS_DEPENDENT_ENTRY();
  FOR_WORK(w)
    const StepDom& S = D[dm];
    for (int r = 0; r < w.rep; r++) {
      const long long c = ((long long)lb * w.rep + r) * blockDim.x + threadIdx.x;
      if (c < S.P.cells) b_assemble(S.P, S.F, c, what);
    }
  }
}

template <typename R>
__device__ __forceinline__ R coef_lo(const Level<R>& L, int d, const int q[3], long long c) {
  if (q[d] == 0) return R(0);
  return tcoef(L, d, lo_pos(L.n, q, (unsigned)c, d));
}

template <typename R>
__device__ __forceinline__ void b_diag(const Level<R>& L, long long c) {
  int q[3];
  decode_pos(L, c, q[0], q[1], q[2]);
  R dg = R(0);
  for (int d = 0; d < 3; d++) {
    dg += tcoef(L, d, (unsigned)c);
    if (q[d] > 0) dg += coef_lo(L, d, q, c);
  }
  const R dgt = dg + L.Dd[c];
  L.diag[c] = dgt;
  L.dinv[c] = R(1) / dgt;
}

template <typename R>
__global__ void k_diag(const CgDom* __restrict__ C, Work w, int l) {
  MDBS_DEPENDENT_ENTRY();
  FOR_WORK(w)
    const Level<R>& L = levels_of<R>(C[dm])[l];
    for (int r = 0; r < w.rep; r++) {
      const long long c = ((long long)lb * w.rep + r) * blockDim.x + threadIdx.x;
      if (c < L.cells) b_diag(L, c);
    }
  }
}

// FP32 copy of the level-0 operator (mixed precision), with its reciprocal diagonal
__global__ void k_level0_to_float(const CgDom* __restrict__ C, Work w) {
  MDBS_DEPENDENT_ENTRY();
  FOR_WORK(w)
    const Level<double>& Ld = C[dm].ld[0];
    const Level<float>& Lf = C[dm].lf[0];
    for (int r = 0; r < w.rep; r++) {
      const long long c = ((long long)lb * w.rep + r) * blockDim.x + threadIdx.x;
      if (c < Ld.cells) {
        for (int a = 0; a < 3; a++) Lf.T[a][c] = (float)Ld.T[a][c];
        Lf.Dd[c] = (float)Ld.Dd[c];
        const float dg = (float)Ld.diag[c];
        Lf.diag[c] = dg;
        Lf.dinv[c] = 1.0f / dg;
      }
    }
  }
}

// coarse transmissibilities: the sum of the fine links crossing the coarse face
// (the Galerkin operator of piecewise-constant transfer), halved when the face's
// normal axis is coarsened, where the 2h link spans twice the fine distance
template <typename R>
__device__ __forceinline__ void b_coarsen(const Level<R>& Fi, const Level<R>& Co, long long ci) {
  int Q[3];
  decode_pos(Co, ci, Q[0], Q[1], Q[2]);
  int lo[3], hi[3];
  for (int a = 0; a < 3; a++) {
    lo[a] = Co.cz[a] ? 2 * Q[a] : Q[a];
    hi[a] = Co.cz[a] ? (2 * Q[a] + 1 < Fi.n[a] ? 2 * Q[a] + 1 : 2 * Q[a]) : Q[a];
  }
  for (int d = 0; d < 3; d++) {
    if (Q[d] + 1 >= Co.n[d]) {
      tstore(Co, d, (unsigned)ci, R(0));
      continue;
    }
    int rl[3] = {lo[0], lo[1], lo[2]}, rh[3] = {hi[0], hi[1], hi[2]};
    rl[d] = rh[d] = Co.cz[d] ? 2 * Q[d] + 1 : Q[d];  // last fine cell of coarse cell Q
    R sum = R(0);
    for (int z = rl[2]; z <= rh[2]; z++)
      for (int y = rl[1]; y <= rh[1]; y++)
        for (int x = rl[0]; x <= rh[0]; x++) sum += tcoef(Fi, d, (unsigned)lpos(Fi.n, x, y, z));
    tstore(Co, d, (unsigned)ci, Co.cz[d] ? R(0.5) * sum : sum);
  }
  R dd = R(0);
  for (int z = lo[2]; z <= hi[2]; z++)
    for (int y = lo[1]; y <= hi[1]; y++)
      for (int x = lo[0]; x <= hi[0]; x++) dd += R(0.5) * Fi.Dd[lpos(Fi.n, x, y, z)];
  Co.Dd[ci] = dd;
}

template <typename R>
__global__ void k_coarsen(const CgDom* __restrict__ C, Work w, int l) {
  MDBS_DEPENDENT_ENTRY();
  FOR_WORK(w)
    const Level<R>* L = levels_of<R>(C[dm]);
    for (int r = 0; r < w.rep; r++) {
      const long long c = ((long long)lb * w.rep + r) * blockDim.x + threadIdx.x;
      if (c < L[l].cells) b_coarsen(L[l - 1], L[l], c);
    }
  }
}

// sum_nb T x_nb at cell c of level L (order x-, x+, y-, y+, z-, z+)
// Load of an iterate or right-hand side.  COH: through L2 (ld.global.cg), for the
// phases of the cooperative kernel, where other CTAs rewrote the value since this
// SM may last have read it (L2 is the point of coherence; a load that allocates in
// L1, or takes the read-only path, could return the old value).
template <bool COH, typename R>
__device__ __forceinline__ R ldc(const R* p) {
  if constexpr (COH)
    return __ldcg(p);
  else
    return *p;
}

template <typename R, bool COH = false>
__device__ __forceinline__ R neighbour_sum(const Level<R>& L, const R* x, const int q[3], long long c) {
  R v = R(0);
  for (int d = 0; d < 3; d++) {
    if (q[d] > 0) {
      const unsigned cl = lo_pos(L.n, q, (unsigned)c, d);
      v += tcoef(L, d, cl) * ldc<COH>(x + cl);
    }
    if (q[d] + 1 < L.n[d]) v += tcoef(L, d, (unsigned)c) * ldc<COH>(x + hi_pos(L.n, q, (unsigned)c, d));
  }
  return v;
}

// fused multiply-add of the level's precision (every smoother spells out the same
// fma chain, so no value depends on the compiler's contraction choices)
__device__ __forceinline__ double fma_r(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fma_r(float a, float b, float c) { return fmaf(a, b, c); }

// One red-black Gauss-Seidel update of cell c = (i, j, k):
// x_c = (b_c + sum_nb T x_nb) / diag_c, neighbours in the order x-, x+, y-, y+,
// z-, z+; zero: the other colour's x is taken as 0.  The batched sweeps and the
// tail share this function, so a cell's value does not depend on which of them
// updates it.
// c, cm, cp: storage positions of the cell and of its x neighbours i - 1, i + 1
template <typename R, typename CT, bool COH = false>
__device__ __forceinline__ void smooth_cell(const R* __restrict__ bb, const R* __restrict__ dinv,
                                            const R* __restrict__ xr, R* __restrict__ xw, CT Tx, CT Ty, CT Tz,
                                            int n0, int n1, int n2, int i, int j, int k, long long c, long long cm,
                                            long long cp, int zero) {
  if (zero) {
    xw[c] = ldc<COH>(bb + c) * dinv[c];
    return;
  }
  const long long sy = n0, sz = (long long)n0 * n1;
  R v = ldc<COH>(bb + c);
  if (i > 0) v = fma_r(Tx[cm], ldc<COH>(xr + cm), v);
  if (i + 1 < n0) v = fma_r(Tx[c], ldc<COH>(xr + cp), v);
  if (j > 0) v = fma_r(Ty[c - sy], ldc<COH>(xr + c - sy), v);
  if (j + 1 < n1) v = fma_r(Ty[c], ldc<COH>(xr + c + sy), v);
  if (k > 0) v = fma_r(Tz[c - sz], ldc<COH>(xr + c - sz), v);
  if (k + 1 < n2) v = fma_r(Tz[c], ldc<COH>(xr + c + sz), v);
  xw[c] = v * dinv[c];
}

// The first post-smoothing update of a level, with the coarse-grid correction of
// the piecewise-constant prolongation applied on the fly: every neighbour of a
// cell being updated has the other colour, and reads x_nb + e_parent(nb) -- the
// value the separate prolongation would have stored, rounded the same way.  The
// cells of the updated colour are overwritten and the other colour is
// overwritten by the next half sweep, so the corrected values need not be stored.
template <typename R, typename CT, bool COH = false>
__device__ __forceinline__ void smooth_cell_corr(const R* __restrict__ bb, const R* __restrict__ dinv,
                                                 const R* __restrict__ xr, R* __restrict__ xw, CT Tx, CT Ty, CT Tz,
                                                 int n0, int n1, int n2, int i, int j, int k, long long c,
                                                 long long cm, long long cp, const Level<R>& Co) {
  const R* __restrict__ ex = Co.x;
  auto e = [&](int a, int b, int d) -> R {
    return ldc<COH>(ex + lpos(Co.n, Co.cz[0] ? a >> 1 : a, Co.cz[1] ? b >> 1 : b, Co.cz[2] ? d >> 1 : d));
  };
  const long long sy = n0, sz = (long long)n0 * n1;
  R v = ldc<COH>(bb + c);
  if (i > 0) v = fma_r(Tx[cm], ldc<COH>(xr + cm) + e(i - 1, j, k), v);
  if (i + 1 < n0) v = fma_r(Tx[c], ldc<COH>(xr + cp) + e(i + 1, j, k), v);
  if (j > 0) v = fma_r(Ty[c - sy], ldc<COH>(xr + c - sy) + e(i, j - 1, k), v);
  if (j + 1 < n1) v = fma_r(Ty[c], ldc<COH>(xr + c + sy) + e(i, j + 1, k), v);
  if (k > 0) v = fma_r(Tz[c - sz], ldc<COH>(xr + c - sz) + e(i, j, k - 1), v);
  if (k + 1 < n2) v = fma_r(Tz[c], ldc<COH>(xr + c + sz) + e(i, j, k + 1), v);
  xw[c] = v * dinv[c];
}

// Red-black half sweep of colour col over REP rows of kBlock half-row cells per
// work item.  Skips domains whose CG has converged (the V-cycle only runs inside
// CG iterations).  The level's arrays go to restrict-qualified registers once per
// work item so that the REP rows of an item overlap their loads: the colour being
// written and the colour being read are disjoint cells of the same array.
// The REP rows of work item lb of a half sweep of colour col over level l of domain G,
// thread tid of kBlock (shared by the per-level launches and the cooperative kernel).
template <typename R, int REP, bool PRO, bool COH = false>
__device__ __forceinline__ void smooth_item_lv(const Level<R>& Lr, const Level<R>& Lc, int lb, unsigned tid, int col,
                                               int zero) {
  const int n0 = Lr.n[0], n1 = Lr.n[1], n2 = Lr.n[2];
  const R* __restrict__ bb = Lr.b;
  const R* __restrict__ dinv = Lr.dinv;
  R* __restrict__ x = Lr.x;
  const unsigned half = (n0 + 1) >> 1;
  const unsigned total = half * (unsigned)n1 * (unsigned)n2;
  const FastDiv dh = Lr.dhalf, dn = Lr.dn1;
  with_coefs(Lr, [&](auto Tx, auto Ty, auto Tz) {
#pragma unroll
    for (int r = 0; r < REP; r++) {
      const unsigned t = ((unsigned)lb * REP + r) * kBlock + tid;
      if (t >= total) continue;
      const unsigned row = fastdiv(t, dh);
      const int ti = (int)(t - row * half);
      const unsigned kk = fastdiv(row, dn);
      const int j = (int)(row - kk * (unsigned)n1), k = (int)kk;
      const int sh = (j + k + col) & 1, i = sh + 2 * ti;
      if (i >= n0) continue;
      // x-split positions: this colour's run, and the other colour's run for i -/+ 1
      const unsigned rb = (unsigned)n0 * row, c = rb + (sh ? half + ti : ti);
      const unsigned cm = sh ? rb + ti : rb + half + ti - 1, cp = sh ? rb + ti + 1 : rb + half + ti;
      if constexpr (PRO)
        smooth_cell_corr<R, decltype(Tx), COH>(bb, dinv, x, x, Tx, Ty, Tz, n0, n1, n2, i, j, k, c, cm, cp, Lc);
      else
        smooth_cell<R, decltype(Tx), COH>(bb, dinv, x, x, Tx, Ty, Tz, n0, n1, n2, i, j, k, c, cm, cp, zero);
    }
  });
}

// the same for domain G's level l (and l + 1, the coarse level of the prolongation)
template <typename R, int REP, bool PRO, bool COH = false>
__device__ __forceinline__ void smooth_item(const CgDom& G, int l, int lb, unsigned tid, int col, int zero) {
  const Level<R>* L = levels_of<R>(G);
  smooth_item_lv<R, REP, PRO, COH>(L[l], L[PRO ? l + 1 : l], lb, tid, col, zero);
}

template <typename R, int REP, bool PRO = false>
__global__ void __launch_bounds__(kBlock, REP == 1 ? 8 : 1)
    k_smooth(const CgDom* __restrict__ C, Work w, int l, int col, int zero, int rev) {
  MDBS_DEPENDENT_ENTRY();
  FOR_WORK_DIR(w, rev)
    const CgDom& G = C[dm];
    if (G.scal[kCond] == 0.0) continue;
    smooth_item<R, REP, PRO>(G, l, lb, threadIdx.x, col, zero);
  }
}

// ------------------------------------------------------------------ vector half sweeps
// A half sweep in which each thread updates kVec consecutive cells of one colour
// run of a row (2 in FP64, 4 in FP32: 16 bytes) with 128-bit loads and stores.  In
// the x-split storage a run of cells of one colour, their right-hand sides, 1/diag,
// their T_x, T_y, T_z and their y and z neighbours are all contiguous and, when n_x
// is a multiple of 2 kVec, 16-byte aligned; the x neighbours are the other colour's
// run shifted by one cell (one extra scalar load).  Each cell's arithmetic is
// smooth_cell's (the same fma chain in the same order), so values are bitwise those
// of the scalar sweep.  Levels of BF16 coefficients use the scalar sweep.
template <typename R>
struct VecOf;
template <>
struct VecOf<double> {
  using T = double2;
  static constexpr int N = 2;
};
template <>
struct VecOf<float> {
  using T = float4;
  static constexpr int N = 4;
};

template <typename R>
__device__ __forceinline__ void ld_vec(const R* __restrict__ p, R* o) {
  const typename VecOf<R>::T v = *reinterpret_cast<const typename VecOf<R>::T*>(p);
  if constexpr (VecOf<R>::N == 2) {
    o[0] = v.x;
    o[1] = v.y;
  } else {
    o[0] = v.x;
    o[1] = v.y;
    o[2] = v.z;
    o[3] = v.w;
  }
}
template <typename R>
__device__ __forceinline__ void st_vec(R* __restrict__ p, const R* o) {
  typename VecOf<R>::T v;
  if constexpr (VecOf<R>::N == 2) {
    v.x = o[0];
    v.y = o[1];
  } else {
    v.x = o[0];
    v.y = o[1];
    v.z = o[2];
    v.w = o[3];
  }
  *reinterpret_cast<typename VecOf<R>::T*>(p) = v;
}

template <typename R, bool PRO>
__global__ void __launch_bounds__(kBlock, 3)
    k_smooth_vec(const CgDom* __restrict__ C, Work w, int l, int col, int zero, int rev) {
  constexpr int V = VecOf<R>::N;
  MDBS_DEPENDENT_ENTRY();
  FOR_WORK_DIR(w, rev)
    const CgDom& G = C[dm];
    if (G.scal[kCond] == 0.0) continue;
    const Level<R>& Lr = levels_of<R>(G)[l];
    const int n0 = Lr.n[0], n1 = Lr.n[1], n2 = Lr.n[2];
    const unsigned half = (unsigned)n0 >> 1;  // both runs: n0 is a multiple of 2 V
    const unsigned total = half * (unsigned)n1 * (unsigned)n2;
    const unsigned t0 = ((unsigned)lb * kBlock + threadIdx.x) * V;  // first half cell of this thread
    if (t0 >= total) continue;
    const unsigned row = fastdiv(t0, Lr.dhalf), ti0 = t0 - row * half;
    const unsigned kk = fastdiv(row, Lr.dn1);
    const int j = (int)(row - kk * (unsigned)n1), k = (int)kk;
    const int sh = (j + k + col) & 1;
    const unsigned rb = (unsigned)n0 * row, c0 = rb + (sh ? half + ti0 : ti0);
    const R* __restrict__ bb = Lr.b;
    const R* __restrict__ dinv = Lr.dinv;
    R* __restrict__ x = Lr.x;
    const R* __restrict__ Tx = Lr.T[0];
    const R* __restrict__ Ty = Lr.T[1];
    const R* __restrict__ Tz = Lr.T[2];
    R acc[V], di[V];
    ld_vec(bb + c0, acc);
    ld_vec(dinv + c0, di);
    if (zero) {
      for (int v = 0; v < V; v++) acc[v] = acc[v] * di[v];
      st_vec(x + c0, acc);
      continue;
    }
    // x neighbours: the other colour's run, shifted by one cell to the left (even cells)
    // or to the right (odd cells); the coefficient of the low face sits at the low
    // neighbour, that of the high face at the cell itself
    R xm[V], xp[V], tm[V], tp[V], ta[V];
    if (sh == 0) {  // cells i = 2 (ti0 + v); i - 1 at rb + half + ti0 + v - 1, i + 1 at rb + half + ti0 + v
      ld_vec(x + rb + half + ti0, xp);
      ld_vec(Tx + rb + half + ti0, ta);
      ld_vec(Tx + c0, tp);
      const bool first = ti0 == 0;
      xm[0] = first ? R(0) : x[rb + half + ti0 - 1];
      tm[0] = first ? R(0) : Tx[rb + half + ti0 - 1];
      for (int v = 1; v < V; v++) {
        xm[v] = xp[v - 1];
        tm[v] = ta[v - 1];
      }
    } else {  // cells i = 2 (ti0 + v) + 1; i - 1 at rb + ti0 + v, i + 1 at rb + ti0 + v + 1
      ld_vec(x + rb + ti0, xm);
      ld_vec(Tx + rb + ti0, tm);
      ld_vec(Tx + c0, tp);
      for (int v = 0; v + 1 < V; v++) xp[v] = xm[v + 1];
      const bool last = ti0 + V == half;  // the last odd cell of the row has no x+ neighbour
      xp[V - 1] = last ? R(0) : x[rb + ti0 + V];
    }
    auto e = [&](int a, int b2, int d) -> R {
      const Level<R>& Co = levels_of<R>(G)[l + 1];
      return Co.x[lpos(Co.n, Co.cz[0] ? a >> 1 : a, Co.cz[1] ? b2 >> 1 : b2, Co.cz[2] ? d >> 1 : d)];
    };
    const unsigned sy = (unsigned)n0, sz = (unsigned)n0 * (unsigned)n1;
    R ym[V], yp[V], zm[V], zp[V], tym[V], typ[V], tzm[V], tzp[V];
    if (j > 0) {
      ld_vec(x + c0 - sy, ym);
      ld_vec(Ty + c0 - sy, tym);
    }
    if (j + 1 < n1) {
      ld_vec(x + c0 + sy, yp);
      ld_vec(Ty + c0, typ);
    }
    if (k > 0) {
      ld_vec(x + c0 - sz, zm);
      ld_vec(Tz + c0 - sz, tzm);
    }
    if (k + 1 < n2) {
      ld_vec(x + c0 + sz, zp);
      ld_vec(Tz + c0, tzp);
    }
#pragma unroll
    for (int v = 0; v < V; v++) {
      const int i = 2 * (int)(ti0 + v) + sh;
      R s = acc[v];
      if constexpr (PRO) {
        if (i > 0) s = fma_r(tm[v], xm[v] + e(i - 1, j, k), s);
        if (i + 1 < n0) s = fma_r(tp[v], xp[v] + e(i + 1, j, k), s);
        if (j > 0) s = fma_r(tym[v], ym[v] + e(i, j - 1, k), s);
        if (j + 1 < n1) s = fma_r(typ[v], yp[v] + e(i, j + 1, k), s);
        if (k > 0) s = fma_r(tzm[v], zm[v] + e(i, j, k - 1), s);
        if (k + 1 < n2) s = fma_r(tzp[v], zp[v] + e(i, j, k + 1), s);
      } else {
        if (i > 0) s = fma_r(tm[v], xm[v], s);
        if (i + 1 < n0) s = fma_r(tp[v], xp[v], s);
        if (j > 0) s = fma_r(tym[v], ym[v], s);
        if (j + 1 < n1) s = fma_r(typ[v], yp[v], s);
        if (k > 0) s = fma_r(tzm[v], zm[v], s);
        if (k + 1 < n2) s = fma_r(tzp[v], zp[v], s);
      }
      acc[v] = s * di[v];
    }
    st_vec(x + c0, acc);
  }
}

// ------------------------------------------------------------------ fused red-black sweep (FP32)
// One launch per sweep pair of an FP32 level: colour c1 everywhere, then the other
// colour.  A CTA owns an extended tile of kSweepCX x kSweepBY cells (the interior
// kSweepTX x kSweepTY, a one-cell halo ring, and spare columns); thread
// (tx, ty) owns the pair of cells 2 tx, 2 tx + 1 of row ty, so in each colour phase
// every lane of a warp updates exactly one cell (no checkerboard divergence).  The
// CTA marches over a chunk [z0, z1) of kz planes: at step k it updates the first
// colour on plane k of the extended tile from the old iterate, and the second
// colour on plane k - 2 of the interior from first-colour values of planes k - 3
// .. k - 1, all finished before the step's barrier (in-plane neighbours at the
// tile edge are the halo values).  One barrier per plane.  The first colour is
// computed more than once on the halo ring and the chunk's end planes z0 - 1 and
// z1, with identical inputs and arithmetic.  The iterate is read from one buffer
// and written to the other (x <-> x2): each array crosses HBM once per pair, half
// the traffic of two half sweeps, and each cell's arithmetic is smooth_cell's.
//
// Planes reach shared memory kSweepDepth planes ahead of use, in a ring of
// kSweepDepth + 4 stages (planes k - 2 .. k + 1 are read at step k).  A stage holds,
// per array (x, T_x, T_y, T_z, b, 1/diag), the natural x range [i0 - 8, i0 + 64) of
// kBoxY rows from j0 - 2, as two kBoxHX x kBoxY boxes of the x-split storage (even
// cells, odd cells): TMA tiled copies (cp.async.bulk.tensor) issued by one thread
// and completing on the stage's mbarrier when the level has tensor maps (FP32
// coefficients, n_x a multiple of 8), else per-element cp.async by every thread.
// Cells outside the domain or the plane range are zero-filled and never used.
// FP64 levels use the half sweeps: GB300's FP64 pipe, not HBM, bounds them.
constexpr int kBoxHalf = kBoxHX * kBoxY;               // cells per box (even or odd cells)
constexpr int kBoxHalfS = (kBoxHalf + 31) / 32 * 32;   // floats per box slot (128-byte aligned)
constexpr int kBoxN = 2 * kBoxHalf;                    // cells per staged array
constexpr int kBoxS = 2 * kBoxHalfS;                   // floats per staged array: even box, odd box
constexpr int kSweepThreads = kSweepBX * kSweepBY;
constexpr int kStage = 6 * kBoxS;                 // floats per stage
constexpr int kStages = kSweepDepth + 4;
constexpr int kRing = 4;                          // planes of first-colour values kept
constexpr unsigned kBoxBytes = kBoxHalf * 4u;  // one TMA box (even or odd cells)
enum { kBoxX_ = 0, kBoxTx = 1, kBoxTy = 2, kBoxTz = 3, kBoxB = 4, kBoxD = 5 };
static_assert(kBoxS * 4 % 128 == 0, "boxes must stay 128-byte aligned in shared memory");
static_assert(kSweepTX % 8 == 0, "tile origins must keep the box starts 16-byte aligned for TMA");

// index in a staged array of the cell at natural offset bx = i - (i0 - 8), row by
__device__ __forceinline__ int box_idx(int bx, int by) {
  return (bx & 1) * kBoxHalfS + by * kBoxHX + (bx >> 1);
}

__host__ __device__ constexpr size_t sweep_smem_bytes() {
  // 128 bytes of alignment slack, the stages, the first-colour ring, the mbarriers
  return 128 + (size_t)kStages * kStage * 4 + (size_t)kRing * kSweepThreads * 4 + (size_t)kStages * 8;
}

constexpr unsigned long long kWaitLimitNs = 1000000000ull;  // a stage that has not landed in 1 s is an error

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// asynchronous copy of one float into shared memory (zero-filled when !ok)
__device__ __forceinline__ void cp_async_f32(float* dst, const float* src, bool ok) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(ok ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(a), "r"(bytes) : "memory");
}
// waits for the phase with the given parity; false when it has not completed within kWaitLimitNs
__device__ __forceinline__ bool mbar_try(unsigned a, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(a), "r"(parity)
      : "memory");
  return done != 0;
}
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
  if (mbar_try(a, parity)) return true;  // the usual case: no clock read
  const unsigned long long t0 = global_ns();
  for (;;) {
    if (mbar_try(a, parity)) return true;
    if (global_ns() - t0 > kWaitLimitNs) return false;
  }
}
// one TMA tiled copy of the box at (x, y, z) of the tensor into shared memory
__device__ __forceinline__ void tma_box(float* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  const unsigned b = (unsigned)__cvta_generic_to_shared(bar);
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];\n" ::"r"(d),
      "l"(map), "r"(x), "r"(y), "r"(z), "r"(b)
      : "memory");
}

// one element of an array into a box: asynchronous for FP32 storage, a plain
// widening copy for BF16 storage (Tb != NULL)
__device__ __forceinline__ void stage_el(float* dst, const float* T, const uint16_t* Tb, unsigned g, bool ok) {
  if (Tb) {
    *dst = ok ? __uint_as_float((unsigned)Tb[g] << 16) : 0.0f;
    return;
  }
  cp_async_f32(dst, T + g, ok);
}

__global__ void __launch_bounds__(kSweepThreads, 2)
    k_smooth_fused(const CgDom* __restrict__ C, Work w, int l, int c1, int zero, int src, int kz, int* err) {
  MDBS_DEPENDENT_ENTRY();
  extern __shared__ unsigned char sweep_smem_raw[];
  float* const base =
      reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(sweep_smem_raw) + 127) & ~(uintptr_t)127);
  float* const s1 = base + kStages * kStage;  // first-colour values, slot plane % kRing, one per thread
  uint64_t* const bars = reinterpret_cast<uint64_t*>(s1 + kRing * kSweepThreads);
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * kSweepBX + tx;
  if (tid == 0) {
    for (int s = 0; s < kStages; s++) mbar_init(&bars[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  unsigned phases = 0;  // parity of the next wait on each stage's mbarrier
  bool failed = false;
  for (int b_ = blockIdx.x; b_ < w.total && !failed; b_ += gridDim.x) {
    const int dm = work_domain(w, b_);
    const int lb = b_ - w.blk[dm];
    const CgDom& G = C[dm];
    if (G.scal[kCond] == 0.0) continue;  // the same for the whole block
    const Level<float>& L = G.lf[l];
    // every pointer in registers: the copies' memory clobbers would otherwise reload
    // them from the domain table after each copy
    const int n0 = L.n[0], n1 = L.n[1], n2 = L.n[2];
    const float* const xin = src ? L.x2 : L.x;
    float* const xout = src ? L.x : L.x2;
    const float* const arr[6] = {xin, L.T[0], L.T[1], L.T[2], L.b, L.dinv};
    const uint16_t* const half[6] = {nullptr, L.Tb[0], L.Tb[1], L.Tb[2], nullptr, nullptr};
    const bool tma = (G.tma_levels >> l) & 1u;
    // the level's maps in the order x, x2, b, 1/diag, T_x, T_y, T_z; box a uses map_idx[a]
    const CUtensorMap* const maps = G.tmaps;
    const int mb = l * kTmaMaps;
    const int map_idx[6] = {mb + (src ? 1 : 0), mb + 4, mb + 5, mb + 6, mb + 2, mb + 3};
    const int ntx = (n0 + kSweepTX - 1) / kSweepTX, nty = (n1 + kSweepTY - 1) / kSweepTY;
    const int rr = lb / ntx;
    const int i0 = (lb - rr * ntx) * kSweepTX, j0 = (rr % nty) * kSweepTY;
    const int z0 = (rr / nty) * kz, z1 = min(z0 + kz, n2);
    const int ia = i0 - 1 + 2 * tx;  // first cell of this thread's pair
    const int j = j0 - 1 + ty;
    const bool row_in = j >= 0 && j < n1;
    const bool row_interior = row_in && ty >= 1 && ty <= kSweepTY;
    // 32-bit cell indices (levels stay below 2^31 cells)
    const unsigned sy = (unsigned)n0, sz = (unsigned)n0 * (unsigned)n1, he = (unsigned)(n0 + 1) >> 1;
    const int a0 = zero ? 1 : 0;  // the zero-guess sweep does not read x
    auto stage_of = [&](int p) { return base + ((p % kStages) + kStages) % kStages * kStage; };

    // stages plane p into stage p mod kStages
    auto issue = [&](int p) {
      const int s = ((p % kStages) + kStages) % kStages;
      float* st = base + s * kStage;
      if (tma) {
        if (tid == 0) {
          asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
          mbar_expect_tx(&bars[s], (6 - a0) * 2 * kBoxBytes);
#pragma unroll
          for (int a = 0; a < 6; a++)
            if (a >= a0) {
              tma_box(st + a * kBoxS, maps + map_idx[a], i0 / 2 - 4, j0 - 2, p, &bars[s]);  // even cells
              tma_box(st + a * kBoxS + kBoxHalfS, maps + map_idx[a], (int)he + i0 / 2 - 4, j0 - 2, p,
                      &bars[s]);  // odd cells
            }
        }
      } else {
        const bool pv = p >= 0 && p < n2;
        for (int e = tid; e < kBoxN; e += kSweepThreads) {
          const int par = e / kBoxHalf, rem = e - par * kBoxHalf;
          const int by = rem / kBoxHX, hx = rem - by * kBoxHX;
          const int ii = i0 - 8 + 2 * hx + par, jj = j0 - 2 + by;
          const bool ok = pv && ii >= 0 && ii < n0 && jj >= 0 && jj < n1;
          // the box holds cells in natural x order, gathered from x-split storage
          const unsigned g = ok ? xs_px(he, ii) + sy * (unsigned)jj + sz * (unsigned)p : 0u;
          const int slot = par * kBoxHalfS + rem;
#pragma unroll
          for (int a = 0; a < 6; a++)
            if (a >= a0) stage_el(st + a * kBoxS + slot, arr[a], half[a], g, ok);
        }
        cp_async_commit();
      }
    };
    // waits until plane p has landed in its stage (TMA path; the copy path waits by group count)
    auto land = [&](int p) -> bool {
      const int s = ((p % kStages) + kStages) % kStages;
      const bool ok = mbar_wait(&bars[s], (phases >> s) & 1u);
      phases ^= 1u << s;
      return ok;
    };

    for (int p = z0 - 2; p <= z0 - 1 + kSweepDepth; p++) issue(p);
    bool ok = true;
    if (tma) ok = land(z0 - 2) && land(z0 - 1);
    float tzmm = 0.0f;  // T_z on plane m - 1 of the cell that is second colour on plane m = k - 2
    int k = z0 - 1;
    for (; k <= z1 + 1 && ok; k++) {
      if (tma)
        ok = land(k + 1);
      else
        cp_async_wait<kSweepDepth - 1>();  // planes up to k + 1 (this thread's copies)
      // every thread's copies of plane k + 1 and first-colour values of plane k - 1 are
      // visible; nothing reads stage k - 3 any more
      if (__syncthreads_or(!ok)) {
        ok = false;
        break;
      }
      issue(k + kSweepDepth + 1);
      // first colour on plane k: the member of the pair with (i + j + k) % 2 == c1
      if (k <= z1) {
        const float* Sm = stage_of(k - 1);
        const float* Sk = stage_of(k);
        const float* Sp = stage_of(k + 1);
        const int e1 = 2 * tx + (((ia + j + k) & 1) == c1 ? 0 : 1);
        const int i1 = i0 - 1 + e1;
        const int b1 = e1 + 7;                 // natural offset of the cell from i0 - 8
        const int h1 = box_idx(b1, ty + 1);  // the cell in the staged arrays
        const int h1m = box_idx(b1 - 1, ty + 1), h1p = box_idx(b1 + 1, ty + 1);
        if (row_in && i1 >= 0 && i1 < n0 && k >= 0 && k < n2) {
          float v = Sk[kBoxB * kBoxS + h1];
          if (!zero) {
            const float* X = Sk;
            const float* TX = Sk + kBoxTx * kBoxS;
            const float* TY = Sk + kBoxTy * kBoxS;
            if (i1 > 0) v = fma_r(TX[h1m], X[h1m], v);
            if (i1 + 1 < n0) v = fma_r(TX[h1], X[h1p], v);
            if (j > 0) v = fma_r(TY[h1 - kBoxHX], X[h1 - kBoxHX], v);
            if (j + 1 < n1) v = fma_r(TY[h1], X[h1 + kBoxHX], v);
            if (k > 0) v = fma_r(Sm[kBoxTz * kBoxS + h1], Sm[h1], v);
            if (k + 1 < n2) v = fma_r(Sk[kBoxTz * kBoxS + h1], Sp[h1], v);
          }
          s1[((k + kRing) % kRing) * kSweepThreads + tid] = v * Sk[kBoxD * kBoxS + h1];
        }
      }
      // second colour on plane m = k - 2: the member of the pair that is not first colour
      const int m = k - 2;
      const int e2 = 2 * tx + (((ia + j + m) & 1) == c1 ? 1 : 0);
      const float* Sq = stage_of(m);
      if (row_interior && m >= z0 && m < z1) {
        const int h2 = box_idx(e2 + 7, ty + 1), h2m = box_idx(e2 + 6, ty + 1);
        const float* q = s1 + ((m + kRing) % kRing) * kSweepThreads;
        const int io = i0 - 1 + (e2 ^ 1);  // first-colour member of the pair on plane m
        if (io >= i0 && io < i0 + kSweepTX && io < n0) xout[xs_px(he, io) + sy * (unsigned)j + sz * (unsigned)m] = q[tid];
        const int i2 = i0 - 1 + e2;
        if (i2 >= i0 && i2 < i0 + kSweepTX && i2 < n0) {
          const float* TX = Sq + kBoxTx * kBoxS;
          const float* TY = Sq + kBoxTy * kBoxS;
          const float left = (e2 & 1) ? q[tid] : q[tid - 1];
          const float right = (e2 & 1) ? q[tid + 1] : q[tid];
          float v = Sq[kBoxB * kBoxS + h2];
          if (i2 > 0) v = fma_r(TX[h2m], left, v);
          if (i2 + 1 < n0) v = fma_r(TX[h2], right, v);
          if (j > 0) v = fma_r(TY[h2 - kBoxHX], q[tid - kSweepBX], v);
          if (j + 1 < n1) v = fma_r(TY[h2], q[tid + kSweepBX], v);
          if (m > 0) v = fma_r(tzmm, s1[((m + kRing - 1) % kRing) * kSweepThreads + tid], v);
          if (m + 1 < n2) v = fma_r(Sq[kBoxTz * kBoxS + h2], s1[((m + 1) % kRing) * kSweepThreads + tid], v);
          xout[xs_px(he, i2) + sy * (unsigned)j + sz * (unsigned)m] = v * Sq[kBoxD * kBoxS + h2];
        }
      }
      // T_z on plane m of the cell that is second colour on plane m + 1 (the next step's;
      // needed from m + 1 = z0 on, and plane m has landed from m = z0 - 2 on)
      if (m >= z0 - 1) {
        const int e2n = 2 * tx + (((ia + j + m + 1) & 1) == c1 ? 1 : 0);
        tzmm = Sq[kBoxTz * kBoxS + box_idx(e2n + 7, ty + 1)];
      }
    }
    // planes staged beyond the chunk: let them land before the stages are reused
    if (tma) {
      for (int p = k + 1; p <= k + kSweepDepth && ok; p++) ok = land(p);
    } else {
      cp_async_wait<0>();
    }
    if (__syncthreads_or(!ok)) {
      if (tid == 0) atomicExch(err, 1);
      failed = true;
    }
  }
  if (failed) {
    // an mbarrier wait ran out: wait (bounded) for the copies still in flight on every
    // stage before the block's shared memory is released
    for (int s = 0; s < kStages; s++) mbar_wait(&bars[s], (phases >> s) & 1u);
  }
}

template <typename R>
__global__ void k_zero(const CgDom* __restrict__ C, Work w, int l, int rev, int sel) {
  MDBS_DEPENDENT_ENTRY();
  FOR_WORK_DIR(w, rev)
    const CgDom& G = C[dm];
    if (G.scal[kCond] == 0.0) continue;
    const Level<R>& L = levels_of<R>(G)[l];
    R* __restrict__ x = sel ? L.x2 : L.x;
    for (int r = 0; r < w.rep; r++) {
      const long long c = ((long long)lb * w.rep + r) * blockDim.x + threadIdx.x;
      if (c < L.cells) x[c] = R(0);
    }
  }
}

// coarse b = sum of the fine residuals b - A x over the covered fine cells.  mask: the
// pre-smoothing ended with a half sweep of colour 1, which leaves the residual of every
// colour-1 cell at zero in exact arithmetic (x_c = (b_c + sum T x_nb) / diag_c), so
// only the colour-0 cells' residuals are formed and summed: half the FP64 work, the
// same V-cycle operator.
template <typename R, bool COH = false>
// fold: also store the coarse level's zero-guess colour-0 update x = b / diag (the
// first pre-smoothing half sweep of that level, which then is not launched)
__device__ __forceinline__ void b_resid_restrict(const Level<R>& Fi, const Level<R>& Co, long long ci, int mask,
                                                 int fold) {
  int Q[3];
  decode_pos(Co, ci, Q[0], Q[1], Q[2]);
  int lo[3], hi[3];
  for (int a = 0; a < 3; a++) {
    lo[a] = Co.cz[a] ? 2 * Q[a] : Q[a];
    hi[a] = Co.cz[a] ? (2 * Q[a] + 1 < Fi.n[a] ? 2 * Q[a] + 1 : 2 * Q[a]) : Q[a];
  }
  R s = R(0);
  for (int z = lo[2]; z <= hi[2]; z++)
    for (int y = lo[1]; y <= hi[1]; y++)
      for (int x = lo[0]; x <= hi[0]; x++) {
        if (mask && ((x + y + z) & 1)) continue;
        const int q[3] = {x, y, z};
        const long long c = lpos(Fi.n, x, y, z);
        const R ax = Fi.diag[c] * ldc<COH>(Fi.x + c) - neighbour_sum<R, COH>(Fi, Fi.x, q, c);
        s += ldc<COH>(Fi.b + c) - ax;
      }
  Co.b[ci] = s;
  if (fold && !((Q[0] + Q[1] + Q[2]) & 1)) Co.x[ci] = s * Co.dinv[ci];
}

template <typename R>
__global__ void k_resid_restrict(const CgDom* __restrict__ C, Work w, int l, int rev, int sel, int mask, int fold) {
  MDBS_DEPENDENT_ENTRY();
  FOR_WORK_DIR(w, rev)
    const CgDom& G = C[dm];
    if (G.scal[kCond] == 0.0) continue;
    const Level<R>* L = levels_of<R>(G);
    Level<R> Fi = L[l];
    if (sel) Fi.x = Fi.x2;  // the buffer holding the fine iterate
    for (int r = 0; r < w.rep; r++) {
      const long long c = ((long long)lb * w.rep + r) * blockDim.x + threadIdx.x;
      if (c < L[l + 1].cells) b_resid_restrict(Fi, L[l + 1], c, mask, fold);
    }
  }
}

template <typename R, bool COH = false>
__device__ __forceinline__ void b_prolong(const Level<R>& Fi, const Level<R>& Co, long long c) {
  int q[3];
  decode_pos(Fi, c, q[0], q[1], q[2]);
  int Q[3];
  for (int a = 0; a < 3; a++) Q[a] = Co.cz[a] ? q[a] / 2 : q[a];
  Fi.x[c] = ldc<COH>(Fi.x + c) + ldc<COH>(Co.x + lpos(Co.n, Q[0], Q[1], Q[2]));
}

template <typename R>
__global__ void k_prolong(const CgDom* __restrict__ C, Work w, int l, int rev, int sel) {
  MDBS_DEPENDENT_ENTRY();
  FOR_WORK_DIR(w, rev)
    const CgDom& G = C[dm];
    if (G.scal[kCond] == 0.0) continue;
    const Level<R>* L = levels_of<R>(G);
    Level<R> Fi = L[l];
    if (sel) Fi.x = Fi.x2;
    for (int r = 0; r < w.rep; r++) {
      const long long c = ((long long)lb * w.rep + r) * blockDim.x + threadIdx.x;
      if (c < L[l].cells) b_prolong(Fi, L[l + 1], c);
    }
  }
}

// ------------------------------------------------------------------ coarsest level
// The coarsest level has at most 4 x 4 x 4 cells.  Once per assembly its dense
// operator is inverted in one CTA (Gauss-Jordan in shared memory, no pivoting:
// the matrix is symmetric positive definite) and symmetrised; the V-cycle then
// solves it exactly with one dense product.
constexpr int kCoarseMax = 64;

template <typename R>
__device__ __forceinline__ R* coarse_inverse_of(const CgDom& G);
template <>
__device__ __forceinline__ double* coarse_inverse_of<double>(const CgDom& G) { return G.cinv_d; }
template <>
__device__ __forceinline__ float* coarse_inverse_of<float>(const CgDom& G) { return G.cinv_f; }

// one block per domain
template <typename R>
__global__ void k_coarse_inverse(const CgDom* __restrict__ CG) {
  MDBS_DEPENDENT_ENTRY();
  const CgDom& G = CG[blockIdx.x];
  const Level<R> C = levels_of<R>(G)[G.nlev - 1];
  R* __restrict__ inv = coarse_inverse_of<R>(G);
  __shared__ R M[kCoarseMax * kCoarseMax];
  const int n = (int)C.cells;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) M[e] = R(0);
  __syncthreads();
  for (int c = threadIdx.x; c < n; c += blockDim.x) {  // rows and columns in storage order
    int q[3];
    decode_pos(C.n, c, q[0], q[1], q[2]);
    M[c * n + c] = C.diag[c];
    for (int d = 0; d < 3; d++) {
      if (q[d] + 1 < C.n[d]) {
        const int u = (int)hi_pos(C.n, q, (unsigned)c, d);
        M[c * n + u] = -tcoef(C, d, (unsigned)c);
        M[u * n + c] = -tcoef(C, d, (unsigned)c);
      }
    }
  }
  // Gauss-Jordan elimination without pivoting (the matrix is symmetric positive
  // definite).  Each thread keeps the (row, column) of its entries (the launch has
  // 1024 threads); per pivot every thread reads what its entries need, a barrier,
  // all write, a barrier.  The thread that owns the next diagonal entry forms that
  // pivot's reciprocal from its new value before the first barrier (double buffered:
  // one FP64 division a pivot).
  constexpr int kPer = (kCoarseMax * kCoarseMax + 1023) / 1024;
  __shared__ R piv[2];
  int ei[kPer], ej[kPer];
  for (int t = 0; t < kPer; t++) {
    const int e = threadIdx.x + t * blockDim.x;
    ei[t] = e < n * n ? e / n : -1;
    ej[t] = e < n * n ? e - ei[t] * n : -1;
  }
  if (threadIdx.x == 0) piv[0] = R(1) / M[0];
  __syncthreads();
  for (int k = 0; k < n; k++) {
    const R pinv = piv[k & 1];
    R nv[kPer];
    for (int t = 0; t < kPer; t++) {
      const int i = ei[t], j = ej[t];
      if (i < 0) continue;
      if (i == k && j == k)
        nv[t] = pinv;
      else if (i == k)
        nv[t] = M[k * n + j] * pinv;
      else if (j == k)
        nv[t] = -M[i * n + k] * pinv;
      else
        nv[t] = M[i * n + j] - M[i * n + k] * (M[k * n + j] * pinv);
      if (i == k + 1 && j == k + 1) piv[(k + 1) & 1] = R(1) / nv[t];
    }
    __syncthreads();  // every read of this pivot's step is done
    for (int t = 0; t < kPer; t++)
      if (ei[t] >= 0) M[ei[t] * n + ej[t]] = nv[t];
    __syncthreads();  // the step's writes (and the next reciprocal) are visible
  }
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e % n;
    inv[e] = R(0.5) * (M[i * n + j] + M[j * n + i]);
  }
}

// ------------------------------------------------------------------ tail V-cycle
// The small levels (and the coarsest solve) of a V-cycle in one CTA, or in one
// thread-block cluster of up to 8 CTAs, per domain: the same per-cell arithmetic,
// in the same order, as the per-level kernels above, with a block or cluster
// barrier between phases instead of kernel boundaries.  The cluster barrier
// (release / acquire at cluster scope) orders the phases' global-memory writes.
constexpr int kTailThreads = 1024;
constexpr int kTailCtasMax = 8;

// this CTA's share of a phase: items rank * blockDim.x + threadIdx.x, step size * blockDim.x
struct TailPart {
  unsigned first, step;
  int size;
};

__device__ __forceinline__ void tail_barrier(const TailPart& tp) {
  if (tp.size > 1) {
    asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
    asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
  } else {
    __syncthreads();
  }
}

template <typename R>
__device__ void tail_smooth(const Level<R>& L, int col, int zero, const TailPart& tp) {
  const int n0 = L.n[0], n1 = L.n[1], n2 = L.n[2];
  const unsigned half = (n0 + 1) >> 1;
  const unsigned total = half * (unsigned)n1 * (unsigned)n2;
  with_coefs(L, [&](auto Tx, auto Ty, auto Tz) {
    for (unsigned t = tp.first; t < total; t += tp.step) {
      const unsigned row = fastdiv(t, L.dhalf), ti = t - row * half;
      const unsigned kk = fastdiv(row, L.dn1);
      const int j = (int)(row - kk * (unsigned)n1), k = (int)kk;
      const int sh = (j + k + col) & 1, i = sh + 2 * (int)ti;
      if (i >= n0) continue;
      const unsigned rb = (unsigned)n0 * row, c = rb + (sh ? half + ti : ti);
      const unsigned cm = sh ? rb + ti : rb + half + ti - 1, cp = sh ? rb + ti + 1 : rb + half + ti;
      smooth_cell<R>(L.b, L.dinv, L.x, L.x, Tx, Ty, Tz, n0, n1, n2, i, j, k, c, cm, cp, zero);
    }
  });
  tail_barrier(tp);
}

template <typename R>
__device__ void tail_pair(const Level<R>& L, int first_col, bool zero_first, const TailPart& tp) {
  tail_smooth(L, first_col, zero_first ? 1 : 0, tp);
  tail_smooth(L, 1 - first_col, 0, tp);
}

template <typename R>
__device__ void tail_zero(const Level<R>& L, const TailPart& tp) {
  for (unsigned c = tp.first; c < (unsigned)L.cells; c += tp.step) L.x[c] = R(0);
  tail_barrier(tp);
}

template <typename R>
__device__ void tail_restrict(const Level<R>& Fi, const Level<R>& Co, const TailPart& tp, int mask) {
  for (unsigned ci = tp.first; ci < (unsigned)Co.cells; ci += tp.step) {
    int Q[3];
    decode_pos(Co, ci, Q[0], Q[1], Q[2]);
    int lo[3], hi[3];
    for (int a = 0; a < 3; a++) {
      lo[a] = Co.cz[a] ? 2 * Q[a] : Q[a];
      hi[a] = Co.cz[a] ? (2 * Q[a] + 1 < Fi.n[a] ? 2 * Q[a] + 1 : 2 * Q[a]) : Q[a];
    }
    R s = R(0);
    for (int z = lo[2]; z <= hi[2]; z++)
      for (int y = lo[1]; y <= hi[1]; y++)
        for (int x = lo[0]; x <= hi[0]; x++) {
          if (mask && ((x + y + z) & 1)) continue;  // as b_resid_restrict
          const int q[3] = {x, y, z};
          const long long c = lpos(Fi.n, x, y, z);
          const R ax = Fi.diag[c] * Fi.x[c] - neighbour_sum(Fi, Fi.x, q, c);
          s += Fi.b[c] - ax;
        }
    Co.b[ci] = s;
  }
  tail_barrier(tp);
}

template <typename R>
__device__ void tail_prolong(const Level<R>& Fi, const Level<R>& Co, const TailPart& tp) {
  for (unsigned c = tp.first; c < (unsigned)Fi.cells; c += tp.step) {
    int q[3];
    decode_pos(Fi, c, q[0], q[1], q[2]);
    int Q[3];
    for (int a = 0; a < 3; a++) Q[a] = Co.cz[a] ? q[a] / 2 : q[a];
    Fi.x[c] += Co.x[lpos(Co.n, Q[0], Q[1], Q[2])];
  }
  tail_barrier(tp);
}

// One CTA or cluster of ctas CTAs per domain (domain = blockIdx.x / ctas): the
// domain's levels from its tail start down to the coarsest one and back.  With
// smem != 0 (single CTA only) the iterates and right-hand sides of those levels
// live in shared memory for the whole cycle (the coefficients, read-only here, stay
// in L1): b of the first tail level is copied in, its x copied out.
// The tail levels of domain G's V-cycle (called by every thread of the CTA, or of
// the cluster when tp.size > 1); lv: the CTA's shared copy of the level views.
template <typename R>
__device__ void tail_body(const CgDom& G, int nu1, int nu2, int cs, int smem, const TailPart& tp, Level<R>* lv,
                          unsigned char* tail_smem_raw) {
  const Level<R>* gl = levels_of<R>(G);
  const int first = G.first, nlev = G.nlev;
  __syncthreads();  // lv may still be read by the previous domain's last phase
  if (threadIdx.x == 0) {
    R* p = reinterpret_cast<R*>(tail_smem_raw);
    for (int l = first; l < nlev; l++) {
      lv[l] = gl[l];
      if (smem) {
        lv[l].x = p;
        p += lv[l].cells;
        lv[l].b = p;
        p += lv[l].cells;
      }
    }
  }
  __syncthreads();
  if (smem) {
    for (unsigned c = threadIdx.x; c < (unsigned)lv[first].cells; c += blockDim.x) lv[first].b[c] = gl[first].b[c];
    __syncthreads();
  }
  for (int l = first; l < nlev - 1; l++) {
    if (nu1 == 0) tail_zero(lv[l], tp);
    for (int it = 0; it < nu1; it++) tail_pair(lv[l], 0, it == 0, tp);
    tail_restrict(lv[l], lv[l + 1], tp, nu1 > 0 ? 1 : 0);
  }
  const Level<R>& C = lv[nlev - 1];
  if (cs == 0) {
    const R* cinv = coarse_inverse_of<R>(G);
    const int n = (int)C.cells;
    for (int i = (int)tp.first; i < n; i += (int)tp.step) {
      R v = R(0);
      for (int j = 0; j < n; j++) v += cinv[i * n + j] * C.b[j];
      C.x[i] = v;
    }
    tail_barrier(tp);
  }
  for (int it = 0; it < cs; it++) tail_pair(C, 0, it == 0, tp);
  for (int it = 0; it < cs; it++) tail_pair(C, 1, false, tp);
  for (int l = nlev - 2; l >= first; l--) {
    tail_prolong(lv[l], lv[l + 1], tp);
    for (int it = 0; it < nu2; it++) tail_pair(lv[l], 1, false, tp);
  }
  if (smem)
    for (unsigned c = threadIdx.x; c < (unsigned)lv[first].cells; c += blockDim.x) gl[first].x[c] = lv[first].x[c];
}

template <typename R>
__global__ void __launch_bounds__(kTailThreads)
    k_tail_vcycle(const CgDom* __restrict__ CG, int nu1, int nu2, int cs, int smem, int ctas) {
  MDBS_DEPENDENT_ENTRY();
  extern __shared__ __align__(16) unsigned char tail_smem_raw[];
  const CgDom& G = CG[blockIdx.x / ctas];
  if (G.scal[kCond] == 0.0) return;  // the same for the whole cluster
  const int rank = blockIdx.x % ctas;
  const TailPart tp{(unsigned)(rank * blockDim.x + threadIdx.x), (unsigned)(ctas * blockDim.x), ctas};
  __shared__ Level<R> lv[kMaxLevels];  // one copy of the level views per block
  tail_body<R>(G, nu1, nu2, cs, smem, tp, lv, tail_smem_raw);
}

// largest shared-memory footprint the tail takes (beyond it, it works in global memory)
constexpr size_t kTailSmemMax = 200 * 1024;

// ------------------------------------------------------------------ coarse levels in one cooperative launch
// The levels between the finest one and the tail, which per-level launches would
// run as about twenty small kernels per V-cycle (each a few microseconds of launch
// and ramp latency for a few MB that sit in L2), in ONE cooperative launch: every
// CTA is resident, and a grid-wide barrier separates the phases (half sweeps,
// restriction) that kernel boundaries separate otherwise.  Each phase walks the
// same work tables as the per-level launches (virtual blocks of kBlock threads)
// with the same per-cell arithmetic, so every value is bitwise the same.  Between
// the descending and the ascending levels each domain's tail runs in one CTA
// (domain d in CTA d mod grid), with block barriers.
constexpr int kCoopThreads = 1024;
constexpr int kCoopVB = kCoopThreads / kBlock;  // virtual blocks of kBlock threads per CTA

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];\n" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Grid-wide barrier on a monotonic arrival counter: the k-th barrier of a launch of G
// CTAs completes when the counter reaches (k + 1) G (counted across launches, so
// nothing needs resetting between graph replays).  Thread 0 of each CTA arrives after
// a block barrier and a gpu-scope fence (the CTA's writes become visible), spins
// with acquire loads, and fences again.  The wait is bounded: after kWaitLimitNs, or
// once another CTA has given up, it sets *err and returns false, and the caller
// returns (the step then reports MDBS_ERR_CUDA).
__device__ __forceinline__ bool coop_sync(unsigned long long* ctr, int* err) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 0;
    if (*(volatile int*)err == 0) {
      ok = 1;
      __threadfence();
      const unsigned long long g = gridDim.x;
      const unsigned long long target = (atomicAdd(ctr, 1ull) / g + 1) * g;
      if (ld_acquire_u64(ctr) < target) {
        const unsigned long long t0 = global_ns();
        unsigned spins = 0;
        while (ld_acquire_u64(ctr) < target) {
          if ((++spins & 255u) == 0) {
            if (*(volatile int*)err != 0) {
              ok = 0;
              break;
            }
            if (global_ns() - t0 > kWaitLimitNs) {
              atomicExch(err, 1);
              ok = 0;
              break;
            }
          }
        }
      }
      __threadfence();
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// work tables of the levels the cooperative kernel runs (first .. last - 1)
struct CoopWork {
  Work half[kMaxLevels];    // red / black half cells
  Work coarse[kMaxLevels];  // cells of level l + 1 (restriction)
  Work fine[kMaxLevels];    // cells of level l (zero guess without pre-smoothing, prolongation without post-smoothing)
  int first, last, ndom;
};

// domains whose level views and convergence flag the cooperative kernel keeps in
// shared memory for the whole launch (batches of more domains read them from global
// memory in every phase)
constexpr int kCoopCacheDoms = 4;

template <typename R>
__global__ void __launch_bounds__(kCoopThreads, 1)
    k_coarse_coop(const CgDom* __restrict__ C, CoopWork cw, int nu1, int nu2, int cs, int tail_smem,
                  unsigned long long* ctr, int* err) {
  extern __shared__ __align__(16) unsigned char tail_smem_raw[];
  __shared__ Level<R> lv[kMaxLevels];
  // Every grid barrier ends in an acquire that invalidates L1, so the per-domain data a
  // phase starts from (level views, convergence flag, block tables) would come from L2
  // again in every phase, a chain of dependent round trips; small batches keep them in
  // shared memory instead (they do not change during the launch).
  __shared__ Level<R> cl[kCoopCacheDoms][kMaxLevels];
  __shared__ int cact[kCoopCacheDoms];
  __shared__ int cblk[2][kMaxLevels][kCoopCacheDoms + 1];  // block tables of cw.half / cw.coarse
  const bool cached = cw.ndom <= kCoopCacheDoms;
  if (cached) {
    for (int t = threadIdx.x; t < cw.ndom * kMaxLevels; t += blockDim.x) {
      const int d = t / kMaxLevels, l = t % kMaxLevels;
      if (l < C[d].nlev) cl[d][l] = levels_of<R>(C[d])[l];
    }
    for (int d = threadIdx.x; d < cw.ndom; d += blockDim.x) cact[d] = C[d].scal[kCond] != 0.0;
    for (int t = threadIdx.x; t < 2 * kMaxLevels * (cw.ndom + 1); t += blockDim.x) {
      const int which = t / (kMaxLevels * (cw.ndom + 1)), r = t % (kMaxLevels * (cw.ndom + 1));
      const int l = r / (cw.ndom + 1), d = r % (cw.ndom + 1);
      const Work& w = which ? cw.coarse[l] : cw.half[l];
      cblk[which][l][d] = (l >= cw.first && l < cw.last) ? w.blk[d] : 0;
    }
    __syncthreads();
  }
  // virtual blocks dealt round-robin over the CTAs first, so that the few items of a
  // small level spread over many SMs (GB300's FP64 rate per SM is low)
  const unsigned vb0 = blockIdx.x + gridDim.x * (threadIdx.x / kBlock), vstep = gridDim.x * kCoopVB;
  const unsigned tid = threadIdx.x % kBlock;
  // domain and local item of flat item b of a level's table (which: 0 half, 1 coarse)
  auto locate = [&](const Work& w, int which, int l, unsigned b, int& dm, int& lb) -> bool {
    if (cached) {
      int d = 0;
      while (d + 1 < cw.ndom && cblk[which][l][d + 1] <= (int)b) d++;
      dm = d;
      lb = (int)b - cblk[which][l][d];
      return cact[d] != 0;
    }
    dm = work_domain(w, (int)b);
    lb = (int)b - w.blk[dm];
    return C[dm].scal[kCond] != 0.0;
  };
  auto level = [&](int dm, int l) -> const Level<R>& { return cached ? cl[dm][l] : levels_of<R>(C[dm])[l]; };
  // every phase walks the items of one level of every domain that has it
  auto half = [&](int l, int col, int zero, bool pro) {
    const Work& w = cw.half[l];
    for (unsigned b = vb0; b < (unsigned)w.total; b += vstep) {
      int dm, lb;
      if (!locate(w, 0, l, b, dm, lb)) continue;
      if (pro)
        smooth_item_lv<R, 1, true, true>(level(dm, l), level(dm, l + 1), lb, tid, col, 0);
      else
        smooth_item_lv<R, 1, false, true>(level(dm, l), level(dm, l), lb, tid, col, zero);
    }
  };
  auto cells = [&](const Work& w, int l, int what) {  // 0 restrict, 1 zero, 2 prolong
    for (unsigned b = vb0; b < (unsigned)w.total; b += vstep) {
      int dm, lb;
      if (what == 0) {
        if (!locate(w, 1, l, b, dm, lb)) continue;
      } else {
        dm = work_domain(w, (int)b);
        lb = (int)b - w.blk[dm];
        if (C[dm].scal[kCond] == 0.0) continue;
      }
      const Level<R>& Lf = level(dm, l);
      const Level<R>& Lc = level(dm, l + 1);
      for (int r = 0; r < w.rep; r++) {
        const long long c = ((long long)lb * w.rep + r) * kBlock + tid;
        if (what == 0) {
          if (c < Lc.cells) b_resid_restrict<R, true>(Lf, Lc, c, nu1 > 0 ? 1 : 0, 0);
        } else if (c < Lf.cells) {
          if (what == 1)
            Lf.x[c] = R(0);
          else
            b_prolong<R, true>(Lf, Lc, c);
        }
      }
    }
  };
  for (int l = cw.first; l < cw.last; l++) {
    if (nu1 == 0) {
      cells(cw.fine[l], l, 1);
      if (!coop_sync(ctr, err)) return;
    }
    for (int it = 0; it < nu1; it++) {
      half(l, 0, it == 0, false);
      if (!coop_sync(ctr, err)) return;
      half(l, 1, 0, false);
      if (!coop_sync(ctr, err)) return;
    }
    cells(cw.coarse[l], l, 0);
    if (!coop_sync(ctr, err)) return;
  }
  for (int d = blockIdx.x; d < cw.ndom; d += gridDim.x) {
    const CgDom& G = C[d];
    if (G.scal[kCond] == 0.0) continue;  // uniform over the CTA
    tail_body<R>(G, nu1, nu2, cs, tail_smem, TailPart{threadIdx.x, blockDim.x, 1}, lv, tail_smem_raw);
  }
  if (!coop_sync(ctr, err)) return;
  for (int l = cw.last - 1; l >= cw.first; l--) {
    const bool last_level = l == cw.first;
    if (nu2 == 0) {
      cells(cw.fine[l], l, 2);
      if (!last_level && !coop_sync(ctr, err)) return;
      continue;
    }
    // the first post-smoothing half sweep applies the prolongation (as the per-level path)
    for (int it = 0; it < nu2; it++) {
      half(l, 1, 0, it == 0);
      if (!coop_sync(ctr, err)) return;
      half(l, 0, 0, false);
      if (!(last_level && it == nu2 - 1) && !coop_sync(ctr, err)) return;
    }
  }
}

// ------------------------------------------------------------------ CG kernels (FP64)
// (A p) at the cell q stored at position c; p is in natural order
__device__ __forceinline__ double apply_A0(const Fld& F, const Prm& P, const double* __restrict__ p, unsigned c,
                                           const int q[3]) {
  const unsigned nc = (unsigned)q[0] + (unsigned)P.n[0] * ((unsigned)q[1] + (unsigned)P.n[1] * (unsigned)q[2]);
  double v = F.diag[c] * p[nc];
  unsigned o = 1;
  for (int d = 0; d < 3; d++) {
    if (q[d] > 0) v -= F.T[d][lo_pos(P.n, q, c, d)] * p[nc - o];
    if (q[d] + 1 < P.n[d]) v -= F.T[d][c] * p[nc + o];
    o *= (unsigned)P.n[d];
  }
  return v;
}

// r = b - A p; one partial of r.r and b.b per block
template <int REP>
__global__ void k_resid0(const StepDom* __restrict__ D, const CgDom* __restrict__ C, Work w, int narrow) {
  MDBS_DEPENDENT_ENTRY();
  FOR_WORK(w)
    const StepDom& S = D[dm];
    const CgDom& G = C[dm];
    double rr = 0.0, bb = 0.0;
    #pragma unroll
    for (int r = 0; r < REP; r++) {
      const long long c = ((long long)lb * REP + r) * blockDim.x + threadIdx.x;
      if (c < S.P.cells) {
        int q[3];
        decode_pos(S.P, c, q[0], q[1], q[2]);
        const double bc = S.F.b[c];
        const double rc = bc - apply_A0(S.F, S.P, S.F.p, (unsigned)c, q);
        G.r[c] = rc;
        if (narrow) G.lf[0].b[c] = (float)rc;  // the first FP32 V-cycle's right-hand side
        rr += rc * rc;
        bb += bc * bc;
      }
    }
    rr = block_sum(rr);
    if (threadIdx.x == 0) G.partials[lb] = rr;
    bb = block_sum(bb);
    if (threadIdx.x == 0) G.partials[G.pcap + lb] = bb;
  }
}

// q = A d; partial d.q
template <int REP>
__global__ void k_spmv_dot(const StepDom* __restrict__ D, const CgDom* __restrict__ C, Work w, int rev) {
  MDBS_DEPENDENT_ENTRY();
  FOR_WORK_DIR(w, rev)
    const CgDom& G = C[dm];
    if (G.scal[kCond] == 0.0) continue;
    const StepDom& S = D[dm];
    double s = 0.0;
    const int n0 = S.P.n[0], n1 = S.P.n[1], n2 = S.P.n[2];
    const long long n = S.P.cells, sy = n0, sz = (long long)n0 * n1;
    const double* __restrict__ dv = G.dv;
    double* __restrict__ qv = G.q;
    const double* __restrict__ dg = S.F.diag;
    const double* __restrict__ Tx = S.F.T[0];
    const double* __restrict__ Ty = S.F.T[1];
    const double* __restrict__ Tz = S.F.T[2];
    #pragma unroll 1
    for (int r = 0; r < REP; r++) {
      const long long c = ((long long)lb * REP + r) * blockDim.x + threadIdx.x;
      if (c < n) {
        int i, j, k;
        decode_pos(S.P, c, i, j, k);
        const unsigned rb = (unsigned)n0 * ((unsigned)j + (unsigned)n1 * (unsigned)k), he = (unsigned)(n0 + 1) >> 1;
        const unsigned cm = rb + xs_px(he, i - 1), cp = rb + xs_px(he, i + 1);
        const double dc = dv[c];
        double v = dg[c] * dc;
        if (i > 0) v -= Tx[cm] * dv[cm];
        if (i + 1 < n0) v -= Tx[c] * dv[cp];
        if (j > 0) v -= Ty[c - sy] * dv[c - sy];
        if (j + 1 < n1) v -= Ty[c] * dv[c + sy];
        if (k > 0) v -= Tz[c - sz] * dv[c - sz];
        if (k + 1 < n2) v -= Tz[c] * dv[c + sz];
        qv[c] = v;
        s += dc * v;
      }
    }
    s = block_sum(s);
    if (threadIdx.x == 0) G.partials[lb] = s;
  }
}

// p += alpha d; r -= alpha q; partial r.r
template <int REP>
__global__ void k_update_xr(const StepDom* __restrict__ D, const CgDom* __restrict__ C, Work w, int rev, int narrow) {
  MDBS_DEPENDENT_ENTRY();
  FOR_WORK_DIR(w, rev)
    const CgDom& G = C[dm];
    if (G.scal[kCond] == 0.0) continue;
    const StepDom& S = D[dm];
    const double al = G.scal[kAlpha];
    double s = 0.0;
    const long long n = S.P.cells;
    const unsigned n0 = (unsigned)S.P.n[0], he = (n0 + 1) >> 1;
    double* __restrict__ p = S.F.p;
    double* __restrict__ rv = G.r;
    const double* __restrict__ dv = G.dv;
    const double* __restrict__ qv = G.q;
    #pragma unroll
    for (int r = 0; r < REP; r++) {
      const long long c = ((long long)lb * REP + r) * blockDim.x + threadIdx.x;
      if (c < n) {
        // p is in natural order: the cell at x-split position c
        const unsigned row = fastdiv((unsigned)c, S.P.dn0), x = (unsigned)c - row * n0;
        p[row * n0 + (x < he ? 2 * x : 2 * (x - he) + 1)] += al * dv[c];
        const double rc = rv[c] - al * qv[c];
        rv[c] = rc;
        if (narrow) G.lf[0].b[c] = (float)rc;  // the next FP32 V-cycle's right-hand side
        s += rc * rc;
      }
    }
    s = block_sum(s);
    if (threadIdx.x == 0) G.partials[lb] = s;
  }
}

// partial r.z and (flexible) z.q
template <int REP>
__global__ void k_dots_rz(const StepDom* __restrict__ D, const CgDom* __restrict__ C, Work w, int with_zq, int rev) {
  MDBS_DEPENDENT_ENTRY();
  FOR_WORK_DIR(w, rev)
    const CgDom& G = C[dm];
    if (G.scal[kCond] == 0.0) continue;
    double rz = 0.0, zq = 0.0;
    const long long n = D[dm].P.cells;
    const double* __restrict__ rv = G.r;
    double* __restrict__ z = G.z;
    const double* __restrict__ qv = G.q;
    const float* __restrict__ zf = G.lf[0].x;
    #pragma unroll
    for (int r = 0; r < REP; r++) {
      const long long c = ((long long)lb * REP + r) * blockDim.x + threadIdx.x;
      if (c < n) {
        // flexible CG: z is the FP32 V-cycle's result, widened here (no separate pass)
        double zc;
        if (with_zq) {
          zc = (double)zf[c];
          z[c] = zc;
        } else {
          zc = z[c];
        }
        rz += rv[c] * zc;
        if (with_zq) zq += zc * qv[c];
      }
    }
    rz = block_sum(rz);
    if (threadIdx.x == 0) G.partials[lb] = rz;
    if (with_zq) {
      zq = block_sum(zq);
      if (threadIdx.x == 0) G.partials[G.pcap + lb] = zq;
    }
  }
}

// d = z + beta d; the first iteration (counter 0) takes d = z
template <int REP>
__global__ void k_update_d(const StepDom* __restrict__ D, const CgDom* __restrict__ C, Work w, int flexible, int rev) {
  MDBS_DEPENDENT_ENTRY();
  FOR_WORK_DIR(w, rev)
    const CgDom& G = C[dm];
    if (G.scal[kCond] == 0.0) continue;
    const double* scal = G.scal;
    const bool first = scal[kIt] == 0.0;
    double be = 0.0;
    if (!first) be = flexible ? -scal[kAlpha] * scal[kZQ] / scal[kRZold] : scal[kRZ] / scal[kRZold];
    const long long n = D[dm].P.cells;
    const double* __restrict__ z = G.z;
    double* __restrict__ dv = G.dv;
    #pragma unroll
    for (int r = 0; r < REP; r++) {
      const long long c = ((long long)lb * REP + r) * blockDim.x + threadIdx.x;
      if (c < n) dv[c] = first ? z[c] : z[c] + be * dv[c];
    }
  }
}

// Scalar finalizers, one block per domain, fixed summation order.  The loop
// condition "not converged, below max_it, finite" goes to scal[kCond].
// mode 0: rr, bb after the initial residual; iteration counter = 0
// mode 1: dq, alpha = rz / dq
// mode 2: rr after the update; counter += 1
// mode 3: rz_old = rz; rz (and zq when two channels)
__global__ void k_finalize(const CgDom* __restrict__ C, Work w, int mode, int two, double tol, int max_it) {
  MDBS_DEPENDENT_ENTRY();
  const CgDom& G = C[blockIdx.x];
  double* scal = G.scal;
  if (mode != 0 && scal[kCond] == 0.0) return;
  const int nb = w.blk[blockIdx.x + 1] - w.blk[blockIdx.x];
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    a += G.partials[i];
    if (two) b += G.partials[G.pcap + i];
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
}

// OR of the domains' conditions: the WHILE node's condition (captured graph) and a flag
// the host reads (eager loop)
__global__ void k_any(const CgDom* __restrict__ C, int ndom, int* flag, cudaGraphConditionalHandle handle,
                      int use_handle) {
  MDBS_DEPENDENT_ENTRY();
  int any = 0;
  for (int d = threadIdx.x; d < ndom; d += blockDim.x) any |= C[d].scal[kCond] != 0.0;
  any = __syncthreads_or(any);
  if (threadIdx.x == 0) {
    *flag = any;
    if (use_handle) cudaGraphSetConditional(handle, any ? 1u : 0u);
  }
}

// b = 0 has the solution p = 0 whatever the initial guess
__global__ void k_zero_if_b0(const StepDom* __restrict__ D, const CgDom* __restrict__ C, Work w) {
  MDBS_DEPENDENT_ENTRY();
  FOR_WORK(w)
    if (C[dm].scal[kBB] != 0.0) continue;
    for (int r = 0; r < w.rep; r++) {
      const long long c = ((long long)lb * w.rep + r) * blockDim.x + threadIdx.x;
      if (c < D[dm].P.cells) D[dm].F.p[c] = 0.0;
    }
  }
}

// iterations and relative residual of corrector corr into each domain's step scalars
__global__ void k_record(const StepDom* __restrict__ D, const CgDom* __restrict__ C, int corr, double tol) {
  MDBS_DEPENDENT_ENTRY();
  if (threadIdx.x != 0) return;
  const double* scal = C[blockIdx.x].scal;
  double* step = D[blockIdx.x].scal;
  const double bb = scal[kBB];
  const double res = bb == 0.0 ? 0.0 : sqrt(scal[kRR] / bb);
  step[kSlotIters + corr] = scal[kIt];
  step[kSlotResid + corr] = res;
  step[kSlotItersTotal] += scal[kIt];
  if (!(res <= tol)) step[kSlotNotConverged] += 1.0;
}

}  // namespace

namespace {
// One thread waits, through the same bounded wait the fused sweep uses, on an
// mbarrier that nothing ever completes: the wait must give up after kWaitLimitNs
// and the kernel return normally.
__global__ void k_wait_selftest(int* status, unsigned long long* waited_ns) {
  __shared__ uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  const unsigned long long t0 = global_ns();
  const bool landed = mbar_wait(&bar, 0);
  *waited_ns = global_ns() - t0;
  *status = landed ? 2 : 1;
}
}  // namespace

cudaError_t bounded_wait_selftest(int* status, double* waited_s) {
  int* d_status = nullptr;
  unsigned long long* d_ns = nullptr;
  cudaError_t e = cudaMalloc(&d_status, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&d_ns, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(d_status, 0, sizeof(int));
  if (e == cudaSuccess) {
    k_wait_selftest<<<1, 32>>>(d_status, d_ns);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  unsigned long long ns = 0;
  if (e == cudaSuccess) e = cudaMemcpy(status, d_status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(&ns, d_ns, sizeof(ns), cudaMemcpyDeviceToHost);
  // the context must still run work after the timed-out wait
  if (e == cudaSuccess) e = cudaMemset(d_status, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (d_status) cudaFree(d_status);
  if (d_ns) cudaFree(d_ns);
  *waited_s = (double)ns * 1e-9;
  return e;
}

cudaError_t sweep_kernel_setup() {
  cudaError_t e =
      cudaFuncSetAttribute(k_smooth_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sweep_smem_bytes());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_tail_vcycle<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTailSmemMax);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_tail_vcycle<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTailSmemMax);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_coarse_coop<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTailSmemMax);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_coarse_coop<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTailSmemMax);
  return e;
}

// dynamic shared memory of the tail (and of the cooperative kernel, which runs it):
// the tail levels' x and b when one CTA per domain runs them and they fit
static size_t tail_smem_bytes(const BatchPlan& B, size_t word, int ctas) {
  const size_t bytes = (size_t)B.tail_words * word;
  return ctas == 1 && bytes <= kTailSmemMax ? bytes : 0;
}

cudaError_t coop_grid_size(int flexible, long long tail_words, int* grid) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t word = flexible ? sizeof(float) : sizeof(double);
  const size_t bytes = (size_t)tail_words * word;
  const size_t smem = bytes <= kTailSmemMax ? bytes : 0;
  if (e == cudaSuccess)
    e = flexible ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_coarse_coop<float>, kCoopThreads, smem)
                 : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_coarse_coop<double>, kCoopThreads, smem);
  *grid = e == cudaSuccess ? sms * per_sm : 0;
  return e;
}

// ------------------------------------------------------------------ solver object
// Device storage of one domain's pressure solver.
struct PressureSolver {
  int precision;
  int nlev;
  Level<double> ld[kMaxLevels];  // FP64 hierarchy (level 0 arrays are borrowed from Fld)
  Level<float> lf[kMaxLevels];   // FP32 hierarchy (mixed precision)
  double *r, *z, *z2, *dv, *q;
  double* partials;
  long long pcap;
  double* scal;
  double* cinv_d;  // inverse of the coarsest operator (FP64 hierarchy)
  float* cinv_f;   // (FP32 hierarchy)
  CUtensorMap* tmaps;   // device: TMA descriptors of the FP32 levels (mixed precisions)
  unsigned tma_levels;  // levels that have them
  void* block;     // single device allocation
  DevBlock mem;    // its owner record (allocator hook)
  size_t bytes;
};

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
  const long long pcap = (n0 + kBlock * kRepBig - 1) / (kBlock * kRepBig);
  double* r = (double*)take(n0 * 8);
  double* z = (double*)take(n0 * 8);
  double* z2 = (double*)take(n0 * 8);
  double* dv = (double*)take(n0 * 8);
  double* q = (double*)take(n0 * 8);
  double* partials = (double*)take(2 * pcap * 8);
  double* scal = (double*)take(16 * 8);
  double* cinv_d = (double*)take(kCoarseMax * kCoarseMax * 8);
  float* cinv_f = (float*)take(kCoarseMax * kCoarseMax * 4);
  CUtensorMap* tmaps = precision != 0 ? (CUtensorMap*)take(kMaxLevels * kTmaMaps * sizeof(CUtensorMap)) : nullptr;
  if (ps) {
    ps->nlev = nlev;
    ps->r = r;
    ps->z = z;
    ps->z2 = z2;
    ps->dv = dv;
    ps->q = q;
    ps->partials = partials;
    ps->pcap = pcap;
    ps->scal = scal;
    ps->cinv_d = cinv_d;
    ps->cinv_f = cinv_f;
    ps->tmaps = tmaps;
  }
  for (int l = 0; l < nlev; l++) {
    const long long nc = (long long)dims[l][0] * dims[l][1] * dims[l][2];
    Level<double> Ld{};
    Level<float> Lf{};
    for (int a = 0; a < 3; a++) {
      Ld.n[a] = Lf.n[a] = dims[l][a];
      Ld.cz[a] = Lf.cz[a] = cz[l][a];
    }
    Ld.cells = Lf.cells = nc;
    Ld.dhalf = Lf.dhalf = make_fastdiv((unsigned)(dims[l][0] + 1) / 2);
    Ld.dn0 = Lf.dn0 = make_fastdiv((unsigned)dims[l][0]);
    Ld.dn1 = Lf.dn1 = make_fastdiv((unsigned)dims[l][1]);
    if (precision == 0) {
      if (l > 0) {
        for (int a = 0; a < 3; a++) Ld.T[a] = (double*)take(nc * 8);
        Ld.Dd = (double*)take(nc * 8);
        Ld.diag = (double*)take(nc * 8);
        Ld.dinv = (double*)take(nc * 8);
        Ld.x = (double*)take(nc * 8);
        Ld.x2 = (double*)take(nc * 8);
        Ld.b = (double*)take(nc * 8);
      }
    } else if (precision == 2 && l > 0) {
      for (int a = 0; a < 3; a++) Lf.Tb[a] = (uint16_t*)take(nc * 2);
      Lf.Dd = (float*)take(nc * 4);
      Lf.diag = (float*)take(nc * 4);
      Lf.dinv = (float*)take(nc * 4);
      Lf.x = (float*)take(nc * 4);
      Lf.x2 = (float*)take(nc * 4);
      Lf.b = (float*)take(nc * 4);
    } else {
      for (int a = 0; a < 3; a++) Lf.T[a] = (float*)take(nc * 4);
      Lf.Dd = (float*)take(nc * 4);
      Lf.diag = (float*)take(nc * 4);
      Lf.dinv = (float*)take(nc * 4);
      Lf.x = (float*)take(nc * 4);
      Lf.x2 = (float*)take(nc * 4);
      Lf.b = (float*)take(nc * 4);
    }
    if (ps) {
      ps->ld[l] = Ld;
      ps->lf[l] = Lf;
    }
  }
  return off;
}

size_t pressure_bytes(const int n[3], int precision) { return solver_layout(n, precision, nullptr, nullptr); }

// The tensor-map encoder of the driver, fetched through the runtime (no libcuda link).
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

// TMA descriptors (3-D tiled over the x-split storage, FP32, box kBoxHX x kBoxY x 1,
// zero fill outside) of every FP32 level whose x extent is a multiple of 8 (so the
// odd cells of a row start on a 16-byte boundary) and whose coefficients are stored
// in FP32; the other levels stage their planes with per-element copies.
static cudaError_t encode_level_maps(PressureSolver* ps) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  ps->tma_levels = 0;
  if (!enc) return cudaSuccess;
  std::vector<CUtensorMap> maps((size_t)kMaxLevels * kTmaMaps);
  memset(maps.data(), 0, maps.size() * sizeof(CUtensorMap));
  for (int l = 0; l < ps->nlev; l++) {
    const Level<float>& L = ps->lf[l];
    if (!L.T[0] || L.n[0] % 8 != 0) continue;
    const cuuint64_t dims[3] = {(cuuint64_t)L.n[0], (cuuint64_t)L.n[1], (cuuint64_t)L.n[2]};
    const cuuint64_t strides[2] = {(cuuint64_t)L.n[0] * 4, (cuuint64_t)L.n[0] * L.n[1] * 4};
    const cuuint32_t box[3] = {(cuuint32_t)kBoxHX, (cuuint32_t)kBoxY, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    float* const arrays[kTmaMaps] = {L.x, L.x2, L.b, L.dinv, L.T[0], L.T[1], L.T[2]};
    bool ok = true;
    for (int a = 0; a < kTmaMaps && ok; a++)
      ok = enc(&maps[(size_t)l * kTmaMaps + a], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, arrays[a], dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    if (ok) ps->tma_levels |= 1u << l;
  }
  return cudaMemcpy(ps->tmaps, maps.data(), maps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice);
}

PressureSolver* pressure_create(const Prm& P, int precision, cudaError_t* err) {
  PressureSolver* ps = new (std::nothrow) PressureSolver();
  if (!ps) {
    *err = cudaErrorMemoryAllocation;
    return nullptr;
  }
  ps->precision = precision;
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
  ps->bytes = bytes;
  *err = dev_block_alloc(&ps->mem, bytes);
  if (*err != cudaSuccess) {
    delete ps;
    return nullptr;
  }
  ps->block = ps->mem.ptr;
  *err = cudaMemset(ps->block, 0, bytes);
  solver_layout(P.n, ps->precision, ps, (char*)ps->block);
  if (*err == cudaSuccess && ps->tmaps) *err = encode_level_maps(ps);
  return ps;
}

void pressure_destroy(PressureSolver* ps) {
  if (!ps) return;
  dev_block_free(&ps->mem);
  delete ps;
}

int pressure_precision(const PressureSolver* ps) { return ps->precision; }

void pressure_storage(const PressureSolver* ps, void** ptr, size_t* bytes) {
  *ptr = ps->block;
  *bytes = ps->bytes;
}

void pressure_view(const PressureSolver* ps, const Fld& F, int tail_cells, CgDom* out) {
  CgDom& G = *out;
  for (int l = 0; l < kMaxLevels; l++) {
    G.ld[l] = l < ps->nlev ? ps->ld[l] : Level<double>{};
    G.lf[l] = l < ps->nlev ? ps->lf[l] : Level<float>{};
  }
  // the FP64 level 0 is the assembled system itself, preconditioning r into z
  Level<double>& L0 = G.ld[0];
  for (int a = 0; a < 3; a++) L0.T[a] = F.T[a];
  L0.Dd = F.Dd;
  L0.diag = F.diag;
  L0.dinv = F.dinv;
  L0.b = ps->r;
  L0.x = ps->z;
  L0.x2 = ps->z2;
  G.nlev = ps->nlev;
  int first = ps->nlev - 1;
  while (first > 0 && ps->ld[first - 1].cells <= tail_cells) first--;
  G.first = first;
  G.r = ps->r;
  G.z = ps->z;
  G.dv = ps->dv;
  G.q = ps->q;
  G.partials = ps->partials;
  G.pcap = ps->pcap;
  G.scal = ps->scal;
  G.cinv_d = ps->cinv_d;
  G.cinv_f = ps->cinv_f;
  G.tmaps = ps->tmaps;
  G.tma_levels = ps->tma_levels;
}

// ------------------------------------------------------------------ batched host sequencing
template <typename R>
static void build_hierarchy(const BatchPlan& B, bool direct, cudaStream_t s) {
  for (int l = 1; l < B.max_levels; l++) {
    MDBS_LAUNCH(K_COARSEN, grid_of(B, B.lcells[l]), kBlock, s, k_coarsen<R>, B.cg, B.lcells[l], l);
    MDBS_LAUNCH(K_DIAG, grid_of(B, B.lcells[l]), kBlock, s, k_diag<R>, B.cg, B.lcells[l], l);
  }
  if (direct) MDBS_LAUNCH(K_COARSEN, B.ndom, 1024, s, k_coarse_inverse<R>, B.cg);
}

// The operator depends on a_P alone, which the correctors of one step share:
// launch_pressure_matrix assembles it once per step and builds the multigrid
// hierarchy (and the coarsest inverse); each corrector then assembles only its
// right-hand side from its HbyA.
void launch_pressure_matrix(const BatchPlan& B, int coarse_sweeps, cudaStream_t s) {
  MDBS_LAUNCH(K_ASSEMBLE, grid_of(B, B.cells), kBlock, s, k_assemble, B.sd, B.cells, (int)kAsmMatrix);
  MDBS_LAUNCH(K_DIAG, grid_of(B, B.cells), kBlock, s, k_diag<double>, B.cg, B.cells, 0);
  if (!B.flexible) {
    build_hierarchy<double>(B, coarse_sweeps == 0, s);
  } else {
    MDBS_LAUNCH(K_CONVERT, grid_of(B, B.cells), kBlock, s, k_level0_to_float, B.cg, B.cells);
    build_hierarchy<float>(B, coarse_sweeps == 0, s);
  }
}

void launch_pressure_rhs(const BatchPlan& B, cudaStream_t s) {
  MDBS_LAUNCH(K_ASSEMBLE, grid_of(B, B.cells), kBlock, s, k_assemble, B.sd, B.cells, (int)kAsmRhs);
}

// Traversal direction of the next kernel over each level; flips at every launch
// (level 0 is shared by the V-cycle and the CG vector kernels).
struct Dirs {
  int l[kMaxLevels] = {};
  int on;
  explicit Dirs(int snake) : on(snake) {}
  int next(int lev) {
    const int d = l[lev];
    l[lev] ^= on;
    return d;
  }
};

// pro: the half sweep applies the prolongation from level l + 1 to the neighbours
// it reads (the first post-smoothing half sweep; no separate prolongation launch)
template <typename R, bool PRO>
static void smooth_half_t(const BatchPlan& B, int l, int col, int zero, Dirs& D, cudaStream_t s) {
  // the half sweep that carries the prolongation is timed as the prolongation
  const int id = PRO ? (l == 0 ? K_PROLONG0 : K_PROLONGC) : (l == 0 ? K_SMOOTH0 : K_SMOOTHC);
  const Work& w = B.lhalf[l];
  const int rev = D.next(l);
  if (B.vec_sweeps && (B.vec_levels >> l & 1u)) {
    const Work& wv = B.lvec[l];
    MDBS_LAUNCH(id, grid_of(B, wv), kBlock, s, (k_smooth_vec<R, PRO>), B.cg, wv, l, col, zero, rev);
    return;
  }
  switch (w.rep) {
    case 8: MDBS_LAUNCH(id, grid_of(B, w), kBlock, s, (k_smooth<R, 8, PRO>), B.cg, w, l, col, zero, rev); break;
    case 4: MDBS_LAUNCH(id, grid_of(B, w), kBlock, s, (k_smooth<R, 4, PRO>), B.cg, w, l, col, zero, rev); break;
    case 2: MDBS_LAUNCH(id, grid_of(B, w), kBlock, s, (k_smooth<R, 2, PRO>), B.cg, w, l, col, zero, rev); break;
    default: MDBS_LAUNCH(id, grid_of(B, w), kBlock, s, (k_smooth<R, 1, PRO>), B.cg, w, l, col, zero, rev); break;
  }
}

template <typename R>
static void smooth_half(const BatchPlan& B, int l, int col, int zero, Dirs& D, cudaStream_t s) {
  smooth_half_t<R, false>(B, l, col, zero, D, s);
}

template <typename R>
static void smooth_pair(const BatchPlan& B, int l, int first_col, bool zero_first, Dirs& D, cudaStream_t s) {
  smooth_half<R>(B, l, first_col, zero_first ? 1 : 0, D, s);
  smooth_half<R>(B, l, 1 - first_col, 0, D, s);
}

// Fused sweeps run on the FP32 hierarchy when the schedule asks for them.
template <typename R>
static bool fused_sweeps(const BatchPlan& B) {
  return B.sweep_kz > 0 && std::is_same<R, float>::value;
}

// One pre- (first colour 0) or post-smoothing (first colour 1) sweep pair of level l.
// Fused: one launch from buffer src into the other one; split: two in-place half sweeps.
template <typename R>
static void sweep(const BatchPlan& B, int l, int first_col, bool zero, int src, Dirs& D, cudaStream_t s) {
  if (fused_sweeps<R>(B)) {
    const dim3 blk(kSweepBX, kSweepBY);
    MDBS_LAUNCH_SMEM(l == 0 ? K_SMOOTH0 : K_SMOOTHC, grid_of(B, B.lsweep[l]), blk, sweep_smem_bytes(), s,
                     k_smooth_fused, B.cg, B.lsweep[l], l, first_col, zero ? 1 : 0, src, B.sweep_kz, B.err_flag);
  } else {
    smooth_pair<R>(B, l, first_col, zero, D, s);
  }
}

// Symmetric V-cycle of every active domain: level 0 receives M r.  Levels that
// precede a domain's tail start run as batched launches; the rest of each
// domain's cycle runs in its own CTA of the tail kernel.  With fused sweeps a
// batched level's iterate alternates between x and x2: after s of its nu1 + nu2
// sweeps it is in buffer (nu1 + nu2 - s) % 2 (1: x2), so it ends in x.
template <typename R>
static void vcycle(const BatchPlan& B, int nu1, int nu2, int cs, Dirs& D, cudaStream_t s) {
  const int S = nu1 + nu2;
  auto cur = [&](int sw) { return fused_sweeps<R>(B) ? (S - sw) & 1 : 0; };
  // the levels between the finest and the tail in one cooperative launch (split sweeps)
  const bool coop = B.coarse_coop && B.max_first >= 2 && !fused_sweeps<R>(B) && B.coop_grid > 0;
  const int batched_end = coop ? 1 : B.max_first;
  // FP32 levels, split sweeps: the restriction into a batched coarse level also stores
  // that level's zero-guess colour-0 half sweep (x = b / diag), which is then not
  // launched (a domain whose tail starts at that level recomputes the same values
  // there).  Measured: 0.5 % off the mixed step; the FP64 restriction is FP64-pipe
  // bound and the step got 0.9 % slower, so FP64 levels keep the separate sweep.
  const bool fold = nu1 > 0 && !fused_sweeps<R>(B) && std::is_same<R, float>::value;
  for (int l = 0; l < batched_end; l++) {
    if (nu1 == 0)
      MDBS_LAUNCH(K_ZERO, grid_of(B, B.lfine[l]), kBlock, s, k_zero<R>, B.cg, B.lfine[l], l, D.next(l), cur(0));
    for (int it = 0; it < nu1; it++) {
      if (it == 0 && l > 0 && fold)
        smooth_half<R>(B, l, 1, 0, D, s);  // colour 0 came with the restriction
      else
        sweep<R>(B, l, 0, it == 0, cur(it), D, s);
    }
    MDBS_LAUNCH(l == 0 ? K_RESTRICT0 : K_RESTRICTC, grid_of(B, B.lcoarse[l]), kBlock, s, k_resid_restrict<R>, B.cg,
                B.lcoarse[l], l, D.next(l), cur(nu1), nu1 > 0 ? 1 : 0, (fold && l + 1 < batched_end) ? 1 : 0);
  }
  if (coop) {
    const size_t smem = tail_smem_bytes(B, sizeof(R), 1);
    CoopWork cw;
    for (int l = 0; l < kMaxLevels; l++) {
      cw.half[l] = B.lhalf[l];
      cw.coarse[l] = B.lcoarse[l];
      cw.fine[l] = B.lfine[l];
    }
    cw.first = 1;
    cw.last = B.max_first;
    cw.ndom = B.ndom;
    prof_begin(K_COOP, s);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(B.coop_grid);
    cfg.blockDim = dim3(kCoopThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;  // every CTA resident: the grid barriers are safe
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    const cudaError_t le =
        cudaLaunchKernelEx(&cfg, k_coarse_coop<R>, B.cg, cw, nu1, nu2, cs, smem > 0 ? 1 : 0, B.coop_ctr, B.err_flag);
    if (le != cudaSuccess) set_launch_error(le);
    prof_end(K_COOP, s);
  }
  const int ctas = B.tail_ctas;
  const size_t tail_bytes = (size_t)B.tail_words * sizeof(R);
  const int tail_smem = ctas == 1 && tail_bytes <= kTailSmemMax ? 1 : 0;
  if (!coop) {
    prof_begin(K_TAIL, s);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(B.ndom * ctas);
    cfg.blockDim = dim3(kTailThreads);
    cfg.dynamicSmemBytes = tail_smem ? tail_bytes : 0;
    cfg.stream = s;
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    at[1].id = cudaLaunchAttributeClusterDimension;
    at[1].val.clusterDim.x = ctas;
    at[1].val.clusterDim.y = 1;
    at[1].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 2;
    const cudaError_t le = cudaLaunchKernelEx(&cfg, k_tail_vcycle<R>, B.cg, nu1, nu2, cs, tail_smem, ctas);
    if (le != cudaSuccess) set_launch_error(le);
    prof_end(K_TAIL, s);
  }
  for (int l = batched_end - 1; l >= 0; l--) {
    if (!fused_sweeps<R>(B) && nu2 > 0) {
      // split sweeps: the first post-smoothing half sweep applies the prolongation
      smooth_half_t<R, true>(B, l, 1, 0, D, s);
      smooth_half<R>(B, l, 0, 0, D, s);
      for (int it = 1; it < nu2; it++) sweep<R>(B, l, 1, false, 0, D, s);
      continue;
    }
    MDBS_LAUNCH(l == 0 ? K_PROLONG0 : K_PROLONGC, grid_of(B, B.lfine[l]), kBlock, s, k_prolong<R>, B.cg, B.lfine[l],
                l, D.next(l), cur(nu1));
    for (int it = 0; it < nu2; it++) sweep<R>(B, l, 1, false, cur(nu1 + it), D, s);
  }
}

cudaError_t pressure_solve(const BatchPlan& B, double tol, int max_it, int nu1, int nu2, int cs, int corr,
                           bool capture, cudaStream_t s, cudaStream_t body_stream, double* host_flag,
                           long long* body_launches) {
  const int flexible = B.flexible;  // the hierarchy comes from launch_pressure_matrix
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
  MDBS_LAUNCH(K_RESID0, grid_of(B, B.rcells), kBlock, s, (k_resid0<kRepBig>), B.sd, B.cg, B.rcells, flexible);
  MDBS_LAUNCH(K_FINALIZE, B.ndom, 1024, s, k_finalize, B.cg, B.rcells, 0, 1, tol, max_it);
  MDBS_LAUNCH(K_FINALIZE, 1, 1024, s, k_any, B.cg, B.ndom, B.any_flag, handle, use);
  MDBS_LAUNCH(K_ZERO, grid_of(B, B.cells), kBlock, s, k_zero_if_b0, B.sd, B.cg, B.cells);
  // one CG iteration, preconditioner first; the last kernels decide whether to continue
  Dirs D(B.snake);
  auto body = [&](cudaStream_t bs) {
    if (!flexible) {
      vcycle<double>(B, nu1, nu2, cs, D, bs);
    } else {
      // the FP32 right-hand side was narrowed by the residual update; the result is
      // widened by the dot products
      vcycle<float>(B, nu1, nu2, cs, D, bs);
    }
    MDBS_LAUNCH(K_DOTS, grid_of(B, B.rcells), kBlock, bs, (k_dots_rz<kRepBig>), B.sd, B.cg, B.rcells, flexible, D.next(0));
    MDBS_LAUNCH(K_FINALIZE, B.ndom, 1024, bs, k_finalize, B.cg, B.rcells, 3, flexible, tol, max_it);
    MDBS_LAUNCH(K_UPDATE_D, grid_of(B, B.rcells), kBlock, bs, (k_update_d<kRepBig>), B.sd, B.cg, B.rcells, flexible, D.next(0));
    MDBS_LAUNCH(K_SPMV_DOT, grid_of(B, B.rcells), kBlock, bs, (k_spmv_dot<kRepBig>), B.sd, B.cg, B.rcells, D.next(0));
    MDBS_LAUNCH(K_FINALIZE, B.ndom, 1024, bs, k_finalize, B.cg, B.rcells, 1, 0, tol, max_it);
    MDBS_LAUNCH(K_UPDATE_XR, grid_of(B, B.rcells), kBlock, bs, (k_update_xr<kRepBig>), B.sd, B.cg, B.rcells, D.next(0),
                flexible);
    MDBS_LAUNCH(K_FINALIZE, B.ndom, 1024, bs, k_finalize, B.cg, B.rcells, 2, 0, tol, max_it);
    MDBS_LAUNCH(K_FINALIZE, 1, 1024, bs, k_any, B.cg, B.ndom, B.any_flag, handle, use);
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
    e = cudaStreamBeginCaptureToGraph(body_stream, body_graph, nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    const long long c0 = launch_count();
    body(body_stream);
    if (body_launches) *body_launches = launch_count() - c0;
    cudaGraph_t out = nullptr;
    e = cudaStreamEndCapture(body_stream, &out);
    if (e != cudaSuccess) return e;
  } else {
    for (;;) {
      cudaError_t e = cudaMemcpyAsync(host_flag, B.any_flag, sizeof(int), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) return e;
      if (*(volatile int*)host_flag == 0) break;
      body(s);
    }
  }
  MDBS_LAUNCH(K_FINALIZE, B.ndom, 32, s, k_record, B.sd, B.cg, corr, tol);
  const cudaError_t le = take_launch_error();
  return le != cudaSuccess ? le : cudaGetLastError();
}

}  // namespace mdbs
