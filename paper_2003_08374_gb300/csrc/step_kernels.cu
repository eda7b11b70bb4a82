// step_kernels.cu -- CUDA kernels of the micro-continuum DBS-VOF time step
// (saturation update, closures, interface geometry, momentum predictor,
// velocity correction) for sm_103a.  One thread per cell or per face; the
// arrays are x-fastest so consecutive threads touch consecutive addresses.
// Paper references: Carrillo, Bourg & Soulaine, arXiv 2003.08374.
#include <math.h>

#include "mdbs_internal.cuh"

namespace mdbs {

namespace {

// Flat face numbering: all x faces, then y faces, then z faces.
__device__ __forceinline__ bool decode_face(const Prm& P, long long t, int& d, int& i, int& j, int& k,
                                            long long& f) {
  if (t < P.nf[0]) {
    d = 0;
    f = t;
  } else if (t < P.nf[0] + P.nf[1]) {
    d = 1;
    f = t - P.nf[0];
  } else if (P.dim == 3 && t < P.nf[0] + P.nf[1] + P.nf[2]) {
    d = 2;
    f = t - P.nf[0] - P.nf[1];
  } else {
    return false;
  }
  // 32-bit decode: mdbs_create limits every array to fewer than 2^31 entries
  // (divisions by multiplication with the domain's invariant-divisor constants)
  const unsigned fx = P.n[0] + (d == 0), fy = P.n[1] + (d == 1);
  const unsigned uf = (unsigned)f;
  const unsigned r = fastdiv(uf, d == 0 ? P.dn0p : P.dn0);
  i = (int)(uf - r * fx);
  const unsigned kk = fastdiv(r, d == 1 ? P.dn1p : P.dn1);
  j = (int)(r - kk * fy);
  k = (int)kk;
  return true;
}

__device__ __forceinline__ long long total_faces(const Prm& P) {
  return P.nf[0] + P.nf[1] + (P.dim == 3 ? P.nf[2] : 0);
}

__device__ __forceinline__ void decode_cell(const Prm& P, long long c, int& i, int& j, int& k) {
  const unsigned uc = (unsigned)c;
  const unsigned r = fastdiv(uc, P.dn0);
  i = (int)(uc - r * (unsigned)P.n[0]);
  const unsigned kk = fastdiv(r, P.dn1);
  j = (int)(r - kk * (unsigned)P.n[1]);
  k = (int)kk;
}

// central difference of a cell field along e at (i,j,k), zero-gradient ghosts
__device__ __forceinline__ double cgrad(const double* __restrict__ a, const Prm& P, int e, int i, int j,
                                        int k) {
  int di = (e == 0), dj = (e == 1), dk = (e == 2);
  return (ghost_read(a, P.n, i + di, j + dj, k + dk) - ghost_read(a, P.n, i - di, j - dj, k - dk)) * P.half_inv_h;
}

// 0 = interior face, 1 = fixed (wall / inlet) face, 2 = outlet face
__device__ __forceinline__ int face_kind(const Prm& P, int d, int cd) {
  if (cd > 0 && cd < P.n[d]) return 0;
  int side = 2 * d + (cd == 0 ? 0 : 1);
  return P.bc[side] == kOutlet ? 2 : 1;
}

__device__ __forceinline__ double warp_reduce_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}

// Sign and order tests of doubles on the integer pipe (GB300 runs FP64 compares
// and min / max on its narrow FP64 pipe).  For finite values: ge0 is x >= 0 with
// -0 counted negative, ge0z is x >= 0, gt0 is x > 0, nz is x != 0; okey maps a double to an int64
// whose signed order is the IEEE order (-0 just below +0), so min / max of keys
// select the same value as fmin / fmax.
__device__ __forceinline__ bool ge0(double x) { return __double_as_longlong(x) >= 0; }
__device__ __forceinline__ bool gt0(double x) { return __double_as_longlong(x) > 0; }
__device__ __forceinline__ bool ge0z(double x) {  // x >= 0 exactly as IEEE (-0 included)
  const long long b = __double_as_longlong(x);
  return b >= 0 || b == (long long)0x8000000000000000ull;
}
__device__ __forceinline__ bool nz(double x) { return (__double_as_longlong(x) << 1) != 0; }
__device__ __forceinline__ long long okey(double x) {
  const long long b = __double_as_longlong(x);
  return b ^ ((b >> 63) & 0x7fffffffffffffffll);
}
__device__ __forceinline__ double from_okey(long long k) { return __longlong_as_double(k ^ ((k >> 63) & 0x7fffffffffffffffll)); }
__device__ __forceinline__ long long kmax2(long long a, long long b) { return a > b ? a : b; }
__device__ __forceinline__ long long kmin2(long long a, long long b) { return a < b ? a : b; }


// ------------------------------------------------------------------ saturation
// Van Leer limited face value (section 3.1): aU + (1/2) psi(r) (aD - aU) with
// psi(r) = (r+|r|)/(1+|r|), r = (aU-aUU)/(aD-aU), evaluated without the ratio
// as aU + ab/(a+b) when ab > 0 (a = aU - aUU, b = aD - aU).
// (FP64 division is the costliest operation of the face flux: it is branched
// around, not selected, where the limiter is zero.)
__device__ __forceinline__ double van_leer(double aU, double aD, double aUU) {
  const double ga = aU - aUU, gb = aD - aU;
  const double ab = ga * gb;
  double v = aU;
  if (gt0(ab)) v = aU + ab / (ga + gb);
  return v;
}

// liquid fractional flow M_l / M of a cell, stored by the closures (alpha in a
// solid-free cell, which has no mobilities)
__device__ __forceinline__ double frac_flow(const Fld& F, long long c) { return F.fw[c]; }

// Face fluxes of the saturation equation (Eq. 15): upwind (low-order) flux,
// Van Leer high-order flux (section 3.1) plus the relative-velocity flux --
// compression in solid-free faces (Eq. 22 oriented as Eq. 41), or in porous faces
// the relative flux phi a_l a_g v_r of Eq. 34 in total-velocity form: with
// v = v_l + v_g the liquid Darcy flux is f v + lambda [(rho_l - rho_g) g + grad pc]
// (f = M_l / M, lambda = M_l M_g / M), taken with the face flux Q, f Van Leer
// limited like alpha and lambda phase-upwinded along the gravity-capillary drive;
// the relative flux is that minus Q * avl.  AF = high - low order.  Mixed
// solid-free / porous faces carry no relative flux.
// returns the boundary inflow of face t (0 for interior faces)
__device__ __forceinline__ double b_alpha_flux(const Prm& P, const Fld& F, long long t) {
  double inflow = 0.0;
  const double inv_h = P.inv_h;
  {
    int d, i, j, k;
    long long f;
    if (!decode_face(P, t, d, i, j, k, f)) return 0.0;
    const double uf = F.u[d][f];
    const double Q = P.A * uf;
    const int cd = d == 0 ? i : (d == 1 ? j : k);
    const int di = (d == 0), dj = (d == 1), dk = (d == 2);
    if (cd > 0 && cd < P.n[d]) {
      const long long l = cell_index(P.n, i - di, j - dj, k - dk);
      const long long r = cell_index(P.n, i, j, k);
      const double al = F.alpha[l], ar = F.alpha[r];
      // upwind, downwind and second-upwind cells (the last clamped into the grid)
      const bool pos = ge0z(Q);
      const long long uc = pos ? l : r, dc = pos ? r : l;
      const int s2 = pos ? -2 : 1;
      const long long uu = cell_index(P.n, clampi(i + s2 * di, 0, P.n[0] - 1), clampi(j + s2 * dj, 0, P.n[1] - 1),
                                      clampi(k + s2 * dk, 0, P.n[2] - 1));
      const double aU = pos ? al : ar, aD = pos ? ar : al, aUU = F.alpha[uu];
      const double flo = Q * aU;
      const bool fl = F.is_free[l], fr = F.is_free[r];
      double hi;  // high-order liquid flux of the face
      if (!fl && !fr) {
        // Q avl + (relative flux) = Q f_vl + A lambda drive: the Van Leer value of
        // alpha cancels, so porous faces do not form it
        const double fvl = van_leer(frac_flow(F, uc), frac_flow(F, dc), frac_flow(F, uu));
        const double drive = P.drho_g[d] + (F.pc[r] - F.pc[l]) * inv_h;
        hi = Q * fvl;
        if (nz(drive)) {
          // liquid from the cell the drive pushes it out of, gas from the other
          const bool fwd = ge0(drive);
          const double mlw = fwd ? F.Ml[l] : F.Ml[r], mgw = fwd ? F.Mg[r] : F.Mg[l];
          const double msum = mlw + mgw;  // mobilities are >= 0
          if (gt0(msum)) hi += P.A * (mlw * mgw / msum) * drive;
        }
      } else {
        double rel = 0.0;
        if (fl && fr) {
          double gf[3] = {0.0, 0.0, 0.0};
          for (int e = 0; e < P.dim; e++)
            gf[e] = 0.5 * (cgrad(F.alpha, P, e, i - di, j - dj, k - dk) + cgrad(F.alpha, P, e, i, j, k));
          const double mag = sqrt(gf[0] * gf[0] + gf[1] * gf[1] + gf[2] * gf[2]);
          const double nfc = gf[d] / (mag + 1e-8 * inv_h);
          const double w = P.c_alpha * fabs(uf) * nfc * P.A;
          rel = ge0z(w) ? w * al * (1.0 - ar) : w * ar * (1.0 - al);
        }
        hi = Q * van_leer(aU, aD, aUU) + rel;
      }
      F.FLO[d][f] = flo;
      F.AF[d][f] = hi - flo;
    } else {
      const bool high = cd != 0;
      const int side = 2 * d + (high ? 1 : 0);
      const long long c = high ? cell_index(P.n, i - di, j - dj, k - dk) : cell_index(P.n, i, j, k);
      double flo = 0.0;
      if (P.bc[side] == kInlet) {
        const bool entering = high ? (Q < 0.0) : (Q > 0.0);
        flo = Q * (entering ? P.inlet_alpha : F.alpha[c]);
      } else if (P.bc[side] == kOutlet) {
        flo = Q * F.alpha[c];
      }
      F.FLO[d][f] = flo;
      F.AF[d][f] = 0.0;
      inflow += high ? -flo : flo;
    }
  }
  return inflow;
}

// one partial sum of the boundary inflow per block (deterministic)
// 4 CTAs per SM (64 registers): measured faster than the unbounded allocation
__global__ void __launch_bounds__(kBlock, 4) k_alpha_flux(const StepDom* __restrict__ D, Work w) {
  MDBS_DEPENDENT_ENTRY();
  for (int b = blockIdx.x; b < w.total; b += gridDim.x) {
    const int dm = work_domain(w, b);
    const StepDom& S = D[dm];
    const int lb = b - w.blk[dm];
    double v = 0.0;
    for (int r = 0; r < w.rep; r++) {
      const long long t = ((long long)lb * w.rep + r) * blockDim.x + threadIdx.x;
      if (t < total_faces(S.P)) v += b_alpha_flux(S.P, S.F, t);
    }
    const double sum = block_sum(v);
    if (threadIdx.x == 0) S.partials[lb] = sum;
  }
}

// low-order (upwind) update
__device__ __forceinline__ void b_alpha_lo(const Prm& P, const Fld& F, long long c, double dt) {
  int i, j, k;
  decode_cell(P, c, i, j, k);
  double div = 0.0;
  for (int d = 0; d < P.dim; d++) {
    long long flo = face_index(P.n, d, i, j, k);
    long long fhi = face_index(P.n, d, i + (d == 0), j + (d == 1), k + (d == 2));
    div += F.FLO[d][fhi] - F.FLO[d][flo];
  }
  F.aL[c] = F.alpha[c] - dt * F.iphiV[c] * div;
}

// Zalesak limiter coefficients R+ / R-.  Bounds: local extrema of the old and
// low-order solutions over the cell and its face neighbours (within [0, 1]) in
// solid-free cells; [0, 1] in porous cells, where the relative flux is the
// physical Darcy phase flux of Eq. 34.
__device__ __forceinline__ void b_alpha_limit(const Prm& P, const Fld& F, long long c, double inv_dt) {
  int i, j, k;
  decode_cell(P, c, i, j, k);
  const double a0 = F.alpha[c], aLc = F.aL[c];
  // extrema through order-preserving integer keys (the same values fmin / fmax select)
  const long long k0 = okey(a0), kL = okey(aLc);
  long long kmax = kmax2(k0, kL), kmin = kmin2(k0, kL);
  double Pp = 0.0, Pm = 0.0;
  for (int d = 0; d < P.dim; d++) {
    const int di = (d == 0), dj = (d == 1), dk = (d == 2);
    const int cd = d == 0 ? i : (d == 1 ? j : k);
    if (cd > 0) {
      long long b = cell_index(P.n, i - di, j - dj, k - dk);
      const long long ka = okey(F.alpha[b]), kb = okey(F.aL[b]);
      kmax = kmax2(kmax, kmax2(ka, kb));
      kmin = kmin2(kmin, kmin2(ka, kb));
    }
    if (cd + 1 < P.n[d]) {
      long long b = cell_index(P.n, i + di, j + dj, k + dk);
      const long long ka = okey(F.alpha[b]), kb = okey(F.aL[b]);
      kmax = kmax2(kmax, kmax2(ka, kb));
      kmin = kmin2(kmin, kmin2(ka, kb));
    }
    const double alo = F.AF[d][face_index(P.n, d, i, j, k)];
    const double ahi = F.AF[d][face_index(P.n, d, i + di, j + dj, k + dk)];
    // fmax(0, x) and fmax(0, -x) from the sign bit
    const double alo_p = ge0(alo) ? alo : 0.0, alo_m = ge0(alo) ? 0.0 : -alo;
    const double ahi_p = ge0(ahi) ? ahi : 0.0, ahi_m = ge0(ahi) ? 0.0 : -ahi;
    Pp += alo_p + ahi_m;
    Pm += alo_m + ahi_p;
  }
  double amax = from_okey(kmin2(kmax, okey(1.0)));
  double amin = from_okey(kmax2(kmin, okey(0.0)));
  if (!F.is_free[c]) {
    amax = 1.0;
    amin = 0.0;
  }
  const double fac = F.phi[c] * P.V * inv_dt;
  const double dq_p = amax - aLc, dq_m = aLc - amin;
  const double Qp = (ge0(dq_p) ? dq_p : 0.0) * fac;
  const double Qm = (ge0(dq_m) ? dq_m : 0.0) * fac;
  F.Rp[c] = gt0(Pp) ? fmin(1.0, Qp / Pp) : 1.0;  // Pp, Pm >= 0
  F.Rm[c] = gt0(Pm) ? fmin(1.0, Qm / Pm) : 1.0;
}

__device__ __forceinline__ double limited_af(const Prm& P, const Fld& F, int d, int i, int j, int k) {
  const int cd = d == 0 ? i : (d == 1 ? j : k);
  if (cd == 0 || cd == P.n[d]) return 0.0;
  const long long l = cell_index(P.n, i - (d == 0), j - (d == 1), k - (d == 2));
  const long long r = cell_index(P.n, i, j, k);
  const double a = F.AF[d][face_index(P.n, d, i, j, k)];
  // R+ and R- lie in [0, 1]: the smaller bit pattern is the smaller value
  const unsigned long long bl = __double_as_longlong(ge0z(a) ? F.Rm[l] : F.Rp[l]);
  const unsigned long long br = __double_as_longlong(ge0z(a) ? F.Rp[r] : F.Rm[r]);
  return __longlong_as_double(bl < br ? bl : br) * a;
}

__device__ __forceinline__ void b_alpha_update(const Prm& P, const Fld& F, long long c, double dt) {
  int i, j, k;
  decode_cell(P, c, i, j, k);
  double corr = 0.0;
  for (int d = 0; d < P.dim; d++) {
    const double lo = limited_af(P, F, d, i, j, k);
    const double hi = limited_af(P, F, d, i + (d == 0), j + (d == 1), k + (d == 2));
    corr += hi - lo;
  }
  F.alpha[c] = F.aL[c] - dt * F.iphiV[c] * corr;
}

// per domain (one block each): scal[slot] += dt * (deterministic sum of the domain's
// partials, one per block of the space w)
__global__ void k_finalize_inflow(const StepDom* __restrict__ D, Work w, int slot) {
  MDBS_DEPENDENT_ENTRY();
  const StepDom& S = D[blockIdx.x];
  const int nb = w.blk[blockIdx.x + 1] - w.blk[blockIdx.x];
  double v = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) v += S.partials[b];
  v = block_sum(v);
  if (threadIdx.x == 0) S.scal[slot] += S.scal[kSlotDt] * v;
}

// ------------------------------------------------------------------ closures
// Appendix A closures, Eqs. 42 and 45 densities / drag, Eq. 38 coefficient.
__device__ __forceinline__ void b_properties(const Prm& P, const Fld& F, long long c) {
  const double a = F.alpha[c];
  F.mu[c] = a * P.mu_l + (1.0 - a) * P.mu_g;
  if (F.is_free[c]) {
    F.Ml[c] = 0.0;
    F.Mg[c] = 0.0;
    F.fw[c] = a;
    F.drag[c] = 0.0;
    F.pc[c] = 0.0;
    F.cf[c] = 0.0;
    F.rho[c] = a * P.rho_l + (1.0 - a) * P.rho_g;
    return;
  }
  double ae = (a - P.a_l_irr) * P.inv_ae_den;
  ae = fmin(fmax(ae, 0.0), 1.0);
  double krl, krg;
  if (P.kr_model == 0) {
    if (P.kr_m_int > 0) {  // integer exponent: repeated products instead of FP64 pow
      krl = ae;
      krg = 1.0 - ae;
      const double bl = krl, bg = krg;
      for (int q = 1; q < P.kr_m_int; q++) {
        krl *= bl;
        krg *= bg;
      }
    } else {
      krl = pow(ae, P.kr_m);
      krg = pow(1.0 - ae, P.kr_m);
    }
  } else {
    const double s1m = pow(ae, 1.0 / P.kr_m);
    krg = sqrt(1.0 - ae) * pow(1.0 - s1m, 2.0 * P.kr_m);
    const double t = 1.0 - pow(1.0 - s1m, P.kr_m);
    krl = sqrt(ae) * t * t;
  }
  const double k0 = F.k0[c];
  const double Ml = k0 * krl * P.inv_mu_l, Mg = k0 * krg * P.inv_mu_g, M = Ml + Mg;
  double s = (a - P.a_pc_irr) * P.inv_s_den;
  s = fmin(fmax(s, P.pc_eps), 1.0 - P.pc_eps);
  double pc;
  if (P.pc_model == 0)
    pc = P.pc_beta == 0.5 ? P.pc0 * rsqrt(s) : P.pc0 * pow(s, -P.pc_beta);
  else
    pc = P.pc0 * pow(pow(s, -1.0 / P.pc_m) - 1.0, 1.0 - P.pc_m);
  F.Ml[c] = Ml;
  F.Mg[c] = Mg;
  const double inv_M = 1.0 / M;  // M > 0 in porous cells: k0 > 0 and k_rl + k_rg > 0
  // f = M_l / M, exactly 1 where the gas has no mobility (M_l (1/M) can be 1 - 1 ulp
  // there, and a saturated region would carry a rounding-size antidiffusive flux)
  F.fw[c] = nz(Mg) ? Ml * inv_M : 1.0;
  F.drag[c] = inv_M;
  // rho* of Eq. 45, or Appendix B's saturation-weighted rho (its buoyancy remainder
  // c_f (rho_l - rho_g) g joins the porous capillary force)
  F.rho[c] = P.porous_density ? a * P.rho_l + (1.0 - a) * P.rho_g : (P.rho_l * Ml + P.rho_g * Mg) * inv_M;
  F.pc[c] = pc;
  F.cf[c] = (Ml * (1.0 - a) - Mg * a) * inv_M;
}

// interface normal toward the liquid (Eq. 24 with the orientation of Eq. 41)
// and the contact-angle normal of Eq. 40 in free cells next to porous cells
// central difference along e as the solid-free cell c sees it: a porous neighbour
// is a zero-gradient ghost (c's own value), like a wall, so that the normal and
// curvature next to a porous surface come from the fluid side before the contact
// angle replaces the normal; porous cells take plain central differences
__device__ __forceinline__ double fluid_grad(const double* __restrict__ a, const Prm& P, const Fld& F, int e,
                                            int i, int j, int k, long long c) {
  const int di = (e == 0), dj = (e == 1), dk = (e == 2);
  const long long hi = cell_index(P.n, clampi(i + di, 0, P.n[0] - 1), clampi(j + dj, 0, P.n[1] - 1),
                                  clampi(k + dk, 0, P.n[2] - 1));
  const long long lo = cell_index(P.n, clampi(i - di, 0, P.n[0] - 1), clampi(j - dj, 0, P.n[1] - 1),
                                  clampi(k - dk, 0, P.n[2] - 1));
  double ah = a[hi], al = a[lo];
  if (F.is_free[c]) {
    if (!F.is_free[hi]) ah = a[c];
    if (!F.is_free[lo]) al = a[c];
  }
  return (ah - al) * P.half_inv_h;
}

__device__ __forceinline__ void b_normals(const Prm& P, const Fld& F, long long c) {
  int i, j, k;
  decode_cell(P, c, i, j, k);
  double g[3] = {0.0, 0.0, 0.0};
  for (int e = 0; e < P.dim; e++) g[e] = fluid_grad(F.alpha, P, F, e, i, j, k, c);
  const double mag = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
  const double inv_den = 1.0 / (mag + P.reg_m);
  double m[3] = {g[0] * inv_den, g[1] * inv_den, g[2] * inv_den};
  const double nw[3] = {F.nw[0][c], F.nw[1][c], F.nw[2][c]};
  if (nw[0] != 0.0 || nw[1] != 0.0 || nw[2] != 0.0) {
    const double mm = sqrt(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
    const double mn = m[0] * nw[0] + m[1] * nw[1] + m[2] * nw[2];
    double t[3], tn = 0.0;
    for (int e = 0; e < 3; e++) {
      t[e] = m[e] - mn * nw[e];
      tn += t[e] * t[e];
    }
    tn = sqrt(tn);
    // no wall tangent where the interface lies parallel to the surface (a tangential
    // part below 1e-9 |m| is rounding, not a direction)
    const bool has_t = tn > 1e-9 * mm;
    for (int e = 0; e < 3; e++) m[e] = mm * (P.cos_t * nw[e] + P.sin_t * (has_t ? t[e] / tn : 0.0));
  }
  F.m[0][c] = m[0];
  F.m[1][c] = m[1];
  F.m[2][c] = m[2];
}

// curvature kappa = -div(m) (Eq. 27 / 43)
__device__ __forceinline__ void b_curvature(const Prm& P, const Fld& F, long long c) {
  int i, j, k;
  decode_cell(P, c, i, j, k);
  double kap = 0.0;
  for (int e = 0; e < P.dim; e++) kap -= fluid_grad(F.m[e], P, F, e, i, j, k, c);
  F.kappa[c] = kap;
}

// ------------------------------------------------------------------ edge viscosities
// The viscosity of an edge is the mean of the four cells around it (ghost cells
// clamp to the boundary cell, as for the faces).  Pair q of axes (a, b) = (0,1),
// (0,2), (1,2); edge (x, y, z) of pair q lies between cells x - 1 and x along a
// and y - 1 and y along b (in the pair's own coordinates), so its array has one
// more entry than the grid along a and along b.  Formed once per step here, read
// by the four faces around each edge in the momentum assembly.
__device__ __forceinline__ long long edge_index(const Prm& P, int q, int x, int y, int z) {
  const int a = q == 2 ? 1 : 0, b = q == 0 ? 1 : 2;
  const long long ex = P.n[0] + (a == 0), ey = P.n[1] + (a == 1 || b == 1);
  return x + ex * (y + ey * (long long)z);
}

__device__ __forceinline__ void edge_mu_at(const Prm& P, const Fld& F, int q, int x, int y, int z) {
  const int a = q == 2 ? 1 : 0, b = q == 0 ? 1 : 2;
  int c00[3] = {x, y, z}, c10[3] = {x, y, z}, c01[3] = {x, y, z}, c11[3] = {x, y, z};
  c00[a] -= 1;
  c00[b] -= 1;
  c10[b] -= 1;
  c01[a] -= 1;
  const double s = ghost_read(F.mu, P.n, c00[0], c00[1], c00[2]) + ghost_read(F.mu, P.n, c10[0], c10[1], c10[2]) +
                   ghost_read(F.mu, P.n, c01[0], c01[1], c01[2]) + ghost_read(F.mu, P.n, c11[0], c11[1], c11[2]);
  F.muE[q][edge_index(P, q, x, y, z)] = 0.25 * s;
}

// cell (i, j, k) forms the edges at its own position, and on the high boundaries of
// the pair's axes also those one position beyond
__device__ __forceinline__ void b_edge_mu(const Prm& P, const Fld& F, long long c) {
  int i, j, k;
  decode_cell(P, c, i, j, k);
  const int q_end = P.dim == 3 ? 3 : 1;
  for (int q = 0; q < q_end; q++) {
    const int a = q == 2 ? 1 : 0, b = q == 0 ? 1 : 2;
    const int pos[3] = {i, j, k};
    const bool ha = pos[a] == P.n[a] - 1, hb = pos[b] == P.n[b] - 1;
    for (int da = 0; da <= (ha ? 1 : 0); da++)
      for (int db = 0; db <= (hb ? 1 : 0); db++) {
        int e[3] = {i, j, k};
        e[a] += da;
        e[b] += db;
        edge_mu_at(P, F, q, e[0], e[1], e[2]);
      }
  }
}

// ------------------------------------------------------------------ momentum
// Staggered momentum equation of a face (Eqs. 46-48): diagonal a_P, neighbour
// coefficients (implicit upwind convection of rho u u / phi^2 and viscous
// diffusion), and rhs0 = Euler source + explicit transpose viscous stress +
// body force (gravity rho g and capillary force F_c, Eqs. 38, 43, 45).  The
// Euler term is taken in advective form, rho^{k+1} (v^{k+1} - v^k) / dt, like
// the convection: the conservative form would need momentum fluxes consistent
// with the saturation fluxes.
// max(w, 0) and max(-w, 0) from the sign bit: integer selects instead of FP64
// compares (GB300 runs FP64 compares on its narrow FP64 pipe)
__device__ __forceinline__ void split_sign(double w, double& pos, double& neg) {
  const long long wb = __double_as_longlong(w);
  pos = wb < 0 ? 0.0 : w;
  neg = wb < 0 ? __longlong_as_double(wb ^ (long long)0x8000000000000000ull) : 0.0;
}

__device__ __forceinline__ void b_momentum_assemble(const Prm& P, const Fld& F, long long t, double inv_dt) {
  int d, i, j, k;
  long long f;
  if (!decode_face(P, t, d, i, j, k, f)) return;
  const long long nf = P.nf[d];
  const int di = (d == 0), dj = (d == 1), dk = (d == 2);
  const int cd = d == 0 ? i : (d == 1 ? j : k);
  const int kind = face_kind(P, d, cd);
  double* __restrict__ anb = F.anb[d] + f;
  if (kind == 1) {
    for (int s = 0; s < 6; s++) anb[s * nf] = 0.0;
    F.aP[d][f] = 1.0;
    F.rhs0[d][f] = 0.0;
    F.B[d][f] = 0.0;
    return;
  }
  const int li = i - di, lj = j - dj, lk = k - dk;  // low cell (may be a ghost at an outlet)
  const double h = P.h, V = P.V;
  const double rhof = 0.5 * (ghost_read(F.rho, P.n, li, lj, lk) + ghost_read(F.rho, P.n, i, j, k));
  const double Df = 0.5 * (ghost_read(F.drag, P.n, li, lj, lk) + ghost_read(F.drag, P.n, i, j, k));
  const double muL = ghost_read(F.mu, P.n, li, lj, lk), muR = ghost_read(F.mu, P.n, i, j, k);
  double Bf = rhof * P.g[d];
  if (kind == 0) {
    const long long l = cell_index(P.n, li, lj, lk), r = cell_index(P.n, i, j, k);
    const bool fl = F.is_free[l], fr = F.is_free[r];
    if (fl && fr) {
      Bf += P.sigma * 0.5 * (F.kappa[l] + F.kappa[r]) * (F.alpha[r] - F.alpha[l]) * P.inv_h;
    } else if (!fl && !fr) {
      const double cff = 0.5 * (F.cf[l] + F.cf[r]);
      Bf += (cff * (F.pc[r] - F.pc[l]) - 0.5 * (F.pc[l] + F.pc[r]) * (F.alpha[r] - F.alpha[l])) * P.inv_h;
      if (P.porous_density) Bf += cff * (P.rho_l - P.rho_g) * P.g[d];  // Appendix B's F_c
    }
  }
  F.B[d][f] = Bf;
  const double uf = F.u[d][f];
  const double inv_phi = F.iphif[d][f];  // 1 / phi_f (static)
  const double inv_h = P.inv_h;
  const double at = V * rhof * (inv_phi * inv_dt);
  const double S = at * uf;  // advective form rho^{k+1} (v^{k+1} - v^k) / dt
  const double cconv = V * rhof * inv_phi * inv_phi * inv_h;
  const double cconv4 = 0.25 * cconv;
  double ap = at + V * Df;
  double tt = 0.0;
  double vgrad = 0.0;  // v . grad(phi^-2) at the face
  const double* __restrict__ gph = F.gphi[d] + f;
  for (int e = 0; e < P.dim; e++) {
    const int ei = (e == 0), ej = (e == 1), ek = (e == 2);
    // e-velocities on the low / high e-faces of the (clamped) low and high cells
    double vLlo = 0.0, vLhi = 0.0, vRlo = 0.0, vRhi = 0.0;
    if (e != d) {
      const int ci = clampi(li, 0, P.n[0] - 1), cj = clampi(lj, 0, P.n[1] - 1), ck = clampi(lk, 0, P.n[2] - 1);
      const int ri = clampi(i, 0, P.n[0] - 1), rj = clampi(j, 0, P.n[1] - 1), rk = clampi(k, 0, P.n[2] - 1);
      vLlo = F.u[e][face_index(P.n, e, ci, cj, ck)];
      vLhi = F.u[e][face_index(P.n, e, ci + ei, cj + ej, ck + ek)];
      vRlo = F.u[e][face_index(P.n, e, ri, rj, rk)];
      vRhi = F.u[e][face_index(P.n, e, ri + ei, rj + ej, rk + ek)];
    }
    // transverse: the sum of the four face velocities (4 w); the 1/4 sits in the static
    // gradient and in cconv4 (scaling by a power of two is exact)
    const double w = (e == d) ? uf : vLlo + vLhi + vRlo + vRhi;
    vgrad += w * gph[e * nf];
    // upwind split of cconv w from its sign (cconv > 0): max(cconv w, 0), max(-cconv w, 0)
    double cpos, cneg;
    split_sign((e == d ? cconv : cconv4) * w, cpos, cneg);
    double muE[2] = {0.0, 0.0};  // edge viscosities of the two e-sides (e != d)
    for (int sg = -1; sg <= 1; sg += 2) {
      const int slot = 2 * e + (sg > 0);
      const int ce = (e == 0 ? i : (e == 1 ? j : k)) + sg;
      int status;  // 0 exists, 1 mirror (no-slip ghost), 2 copy (zero-gradient ghost)
      if (e == d)
        status = (ce >= 0 && ce <= P.n[d]) ? 0 : 2;
      else if (ce >= 0 && ce < P.n[e])
        status = 0;
      else
        status = P.bc[2 * e + (sg > 0)] == kOutlet ? 2 : 1;
      const double cup = sg < 0 ? cpos : cneg;
      double mus;
      if (e == d) {
        mus = sg < 0 ? muL : muR;
      } else {
        // the edge between this face and its e-neighbour on side sg: at the face's
        // position along d, between cells c_e - 1 and c_e (sg < 0) or c_e and c_e + 1
        int q3[3] = {i, j, k};
        q3[e] += (sg > 0);
        mus = F.muE[d + e - 1][edge_index(P, d + e - 1, q3[0], q3[1], q3[2])];
        muE[sg > 0] = mus;
      }
      const double a = cup + mus * h;  // mu A / h with A = h^2
      anb[slot * nf] = status == 0 ? a : 0.0;
      if (status == 0)
        ap += a;
      else if (status == 1)
        ap += 2.0 * a;
    }
    // explicit div(mu grad(u)^T), component d (velocity differences; 1/h^2 once below)
    if (e == d) {
      const double dR = (cd + 1 <= P.n[d]) ? F.u[d][face_index(P.n, d, i + di, j + dj, k + dk)] - uf : 0.0;
      const double dL = (cd - 1 >= 0) ? uf - F.u[d][face_index(P.n, d, li, lj, lk)] : 0.0;
      tt += muR * dR - muL * dL;
    } else {
      tt -= muE[0] * (vRlo - vLlo);
      tt += muE[1] * (vRhi - vLhi);
    }
  }
  for (int s = 2 * P.dim; s < 6; s++) anb[s * nf] = 0.0;
  // The rest of Eq. 21's convection: with div v = 0 and the density carried by the
  // flow, (1/phi) div(rho v v / phi) minus the advective part above is
  // (rho/2) v (v . grad(phi^-2)), non-zero only where the porosity varies along the
  // flow; implicit where it decelerates the flow, explicit where it accelerates it.
  const double Gp = 0.5 * rhof * vgrad;
  double Sx = S;
  if (__double_as_longlong(Gp) >= 0)  // Gp >= 0 (+0 and -0 add nothing either way)
    ap += V * Gp;
  else
    Sx -= V * Gp * uf;
  F.aP[d][f] = 1.0 / ap;  // stored as the reciprocal: every later use multiplies
  F.rhs0[d][f] = Sx + V * (tt * P.inv_h2 + Bf);
}

// H(u) = sum_nb a_nb u_nb + rhs0 of an unknown face.  A missing neighbour has
// a_nb = 0: its product is formed with the face's own value (a flat index clamped
// into the array), which adds exactly zero for finite velocities, so the sum needs
// no FP64 compare per neighbour.
__device__ __forceinline__ double face_H(const Prm& P, const Fld& F, const double* const* u, int d, long long f) {
  const long long nf = P.nf[d];
  const long long fx = P.n[0] + (d == 0), fxy = fx * (P.n[1] + (d == 1));
  const double* __restrict__ ud = u[d];
  double hs = 0.0;
  for (int e = 0; e < P.dim; e++) {
    const long long st = e == 0 ? 1 : (e == 1 ? fx : fxy);
    const double am = F.anb[d][(2 * e) * nf + f];
    const double ap = F.anb[d][(2 * e + 1) * nf + f];
    const long long fm = f - st >= 0 ? f - st : f, fp = f + st < nf ? f + st : f;
    hs += am * ud[fm];
    hs += ap * ud[fp];
  }
  return hs + F.rhs0[d][f];
}

// p_R - p_L across a face; the outlet ghost holds -p (p = 0 on the face)
__device__ __forceinline__ double face_dp(const Prm& P, const double* __restrict__ p, int d, int i, int j,
                                          int k) {
  const int cd = d == 0 ? i : (d == 1 ? j : k);
  const int di = (d == 0), dj = (d == 1), dk = (d == 2);
  const double pl = cd > 0 ? p[cell_index(P.n, i - di, j - dj, k - dk)] : -p[cell_index(P.n, i, j, k)];
  const double pr = cd < P.n[d] ? p[cell_index(P.n, i, j, k)] : -p[cell_index(P.n, i - di, j - dj, k - dk)];
  return pr - pl;
}

// one Jacobi sweep of the momentum predictor (Eq. 50): out = (H(in) - V grad p^k)/a_P
// (in / out: the three face arrays of the iterate and of the result)
__device__ __forceinline__ void b_jacobi(const Prm& P, const Fld& F, long long t, const double* const* in,
                                         double* const* out) {
  int d, i, j, k;
  long long f;
  if (!decode_face(P, t, d, i, j, k, f)) return;
  const int cd = d == 0 ? i : (d == 1 ? j : k);
  if (face_kind(P, d, cd) == 1) {
    out[d][f] = in[d][f];
    return;
  }
  const double hs = face_H(P, F, in, d, f);
  out[d][f] = (hs - P.A * face_dp(P, F.p, d, i, j, k)) * F.aP[d][f];  // V/h = A; aP = 1/a_P
}

// utmp -> u (after an odd number of Jacobi sweeps)
__global__ void k_copy_faces(const StepDom* __restrict__ D, Work w) {
  MDBS_DEPENDENT_ENTRY();
  for (int b = blockIdx.x; b < w.total; b += gridDim.x) {
    const int dm = work_domain(w, b);
    const StepDom& S = D[dm];
    const int lb = b - w.blk[dm];
    for (int r = 0; r < w.rep; r++) {
      const long long t = ((long long)lb * w.rep + r) * blockDim.x + threadIdx.x;
      int d, i, j, k;
      long long f;
      if (decode_face(S.P, t, d, i, j, k, f)) S.F.u[d][f] = S.F.utmp[d][f];
    }
  }
}

// HbyA = H(u)/a_P (Eq. 51 without the pressure gradient)
__device__ __forceinline__ void b_hbya(const Prm& P, const Fld& F, long long t) {
  int d, i, j, k;
  long long f;
  if (!decode_face(P, t, d, i, j, k, f)) return;
  const int cd = d == 0 ? i : (d == 1 ? j : k);
  if (face_kind(P, d, cd) == 1) {
    F.hbya[d][f] = 0.0;
    return;
  }
  F.hbya[d][f] = face_H(P, F, F.u, d, f) * F.aP[d][f];
}

// corrected velocity, Eq. 51
__device__ __forceinline__ void b_correct(const Prm& P, const Fld& F, long long t) {
  int d, i, j, k;
  long long f;
  if (!decode_face(P, t, d, i, j, k, f)) return;
  const int cd = d == 0 ? i : (d == 1 ? j : k);
  if (face_kind(P, d, cd) == 1) return;
  F.u[d][f] = F.hbya[d][f] - (P.A * F.aP[d][f]) * face_dp(P, F.p, d, i, j, k);
}

__device__ __forceinline__ void b_boundary_velocities(const Prm& P, const Fld& F, long long t) {
  int d, i, j, k;
  long long f;
  if (!decode_face(P, t, d, i, j, k, f)) return;
  const int cd = d == 0 ? i : (d == 1 ? j : k);
  if (face_kind(P, d, cd) != 1) return;
  const int side = 2 * d + (cd == 0 ? 0 : 1);
  double v = 0.0;
  if (P.bc[side] == kInlet) v = (side & 1) ? -P.inlet_u : P.inlet_u;
  F.u[d][f] = v;
}

// mass, alpha min / max and a non-finite sentinel: one partial per block in four
// channels of the domain's partials (stride pcap)
__global__ void k_field_stats(const StepDom* __restrict__ D, Work w) {
  MDBS_DEPENDENT_ENTRY();
  __shared__ double smx[32], smn[32];
  for (int b = blockIdx.x; b < w.total; b += gridDim.x) {
    const int dm = work_domain(w, b);
    const StepDom& S = D[dm];
    const int lb = b - w.blk[dm];
    double mass = 0.0, amin = INFINITY, amax = -INFINITY, bad = 0.0;
    for (int r = 0; r < w.rep; r++) {
      const long long c = ((long long)lb * w.rep + r) * blockDim.x + threadIdx.x;
      if (c < S.P.cells) {
        const double a = S.F.alpha[c];
        mass += S.F.phi[c] * a * S.P.V;
        amin = fmin(amin, a);
        amax = fmax(amax, a);
        if (!isfinite(a) || !isfinite(S.F.p[c])) bad += 1.0;
      }
    }
    const long long pc = S.pcap;
    mass = block_sum(mass);
    if (threadIdx.x == 0) S.partials[lb] = mass;
    bad = block_sum(bad);
    if (threadIdx.x == 0) S.partials[3 * pc + lb] = bad;
    double vmx = warp_reduce_max(amax), vmn = -warp_reduce_max(-amin);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) {
      smx[threadIdx.x >> 5] = vmx;
      smn[threadIdx.x >> 5] = vmn;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double a = -INFINITY, bb = INFINITY;
      for (int q = 0; q < (int)(blockDim.x >> 5); q++) {
        a = fmax(a, smx[q]);
        bb = fmin(bb, smn[q]);
      }
      S.partials[pc + lb] = bb;
      S.partials[2 * pc + lb] = a;
    }
  }
}

// per domain (one block each): fold the partials of the cells space into the scalars
__global__ void k_finalize_stats(const StepDom* __restrict__ D, Work w) {
  MDBS_DEPENDENT_ENTRY();
  // one block per domain; each thread folds a fixed stride of the partials and the
  // block combines them in a fixed tree (deterministic sums)
  const StepDom& S = D[blockIdx.x];
  const int nb = w.blk[blockIdx.x + 1] - w.blk[blockIdx.x];
  const long long pc = S.pcap;
  double mass = 0.0, amin = INFINITY, amax = -INFINITY, bad = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    mass += S.partials[b];
    amin = fmin(amin, S.partials[pc + b]);
    amax = fmax(amax, S.partials[2 * pc + b]);
    bad += S.partials[3 * pc + b];
  }
  mass = block_sum(mass);
  bad = block_sum(bad);
  amin = block_minmax<false>(amin);
  amax = block_minmax<true>(amax);
  if (threadIdx.x == 0) {
    S.scal[kSlotMass] = mass;
    S.scal[kSlotAmin] = amin;
    S.scal[kSlotAmax] = amax;
    S.scal[kSlotBad] = bad;
  }
}

// max over faces of |u_f| / phi_f (CFL time step, section 3.2), one partial per block
__global__ void k_cfl(const StepDom* __restrict__ D, Work w) {
  MDBS_DEPENDENT_ENTRY();
  __shared__ double sm[32];
  for (int b = blockIdx.x; b < w.total; b += gridDim.x) {
    const int dm = work_domain(w, b);
    const StepDom& S = D[dm];
    const int lb = b - w.blk[dm];
    double vmax = 0.0;
    for (int r = 0; r < w.rep; r++) {
      const long long t = ((long long)lb * w.rep + r) * blockDim.x + threadIdx.x;
      int d, i, j, k;
      long long f;
      if (decode_face(S.P, t, d, i, j, k, f)) {
        const double phif = 0.5 * (ghost_read(S.F.phi, S.P.n, i - (d == 0), j - (d == 1), k - (d == 2)) +
                                   ghost_read(S.F.phi, S.P.n, i, j, k));
        vmax = fmax(vmax, fabs(S.F.u[d][f]) / phif);
      }
    }
    vmax = warp_reduce_max(vmax);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = vmax;
    __syncthreads();
    if (threadIdx.x == 0) {
      double a = 0.0;
      for (int q = 0; q < (int)(blockDim.x >> 5); q++) a = fmax(a, sm[q]);
      S.partials[lb] = a;
    }
  }
}

// per domain: time += dt; with cfl > 0 the next dt = min(cfl h / max|u/phi|, 1.2 dt, dt_max)
__global__ void k_finalize_time(const StepDom* __restrict__ D, Work w) {
  MDBS_DEPENDENT_ENTRY();
  const StepDom& S = D[blockIdx.x];
  double* scal = S.scal;
  const double dt = scal[kSlotDt];
  if (!(S.P.cfl > 0.0)) {
    if (threadIdx.x == 0) scal[kSlotTime] += dt;
    return;
  }
  const int nb = w.blk[blockIdx.x + 1] - w.blk[blockIdx.x];
  double a = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) a = fmax(a, S.partials[b]);
  a = block_minmax<true>(a);
  if (threadIdx.x != 0) return;
  scal[kSlotTime] += dt;
  scal[kSlotUmax] = a;
  double dtn = a > 0.0 ? S.P.cfl * S.P.h / a : S.P.dt_max;
  dtn = fmin(dtn, 1.2 * dt);
  dtn = fmin(dtn, S.P.dt_max);
  scal[kSlotDt] = dtn;
}

// static geometry: solid-free flag (porosity exactly 1) and, in free cells with a
// porous face neighbour, the wall normal n_w = -grad(phi)/|grad(phi)| pointing
// into the porous side (used by the contact-angle normal of Eq. 40)
__device__ __forceinline__ void b_static_geometry(const Prm& P, const Fld& F, long long c) {
  const double* __restrict__ phi = F.phi;
  int i, j, k;
  decode_cell(P, c, i, j, k);
  const bool fr = phi[c] == 1.0;
  const_cast<uint8_t*>(F.is_free)[c] = fr ? 1 : 0;
  double n[3] = {0.0, 0.0, 0.0};
  if (fr) {
    bool touch = false;
    for (int d = 0; d < P.dim; d++) {
      const int di = (d == 0), dj = (d == 1), dk = (d == 2);
      const int cd = d == 0 ? i : (d == 1 ? j : k);
      if (cd > 0 && phi[cell_index(P.n, i - di, j - dj, k - dk)] != 1.0) touch = true;
      if (cd + 1 < P.n[d] && phi[cell_index(P.n, i + di, j + dj, k + dk)] != 1.0) touch = true;
    }
    if (touch) {
      double g[3] = {0.0, 0.0, 0.0};
      for (int e = 0; e < P.dim; e++) g[e] = cgrad(phi, P, e, i, j, k);
      const double mag = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
      if (mag > 0.0)
        for (int e = 0; e < 3; e++) n[e] = -g[e] / mag;
    }
  }
  for (int e = 0; e < 3; e++) const_cast<double*>(F.nw[e])[c] = n[e];
  const_cast<double*>(F.iphi2)[c] = 1.0 / (phi[c] * phi[c]);
  const_cast<double*>(F.iphiV)[c] = 1.0 / (phi[c] * P.V);
}

__global__ void k_static_geometry(const StepDom* __restrict__ D, Work w) {
  MDBS_DEPENDENT_ENTRY();
  for (int b = blockIdx.x; b < w.total; b += gridDim.x) {
    const int dm = work_domain(w, b);
    const StepDom& S = D[dm];
    const int lb = b - w.blk[dm];
    for (int r = 0; r < w.rep; r++) {
      const long long c = ((long long)lb * w.rep + r) * blockDim.x + threadIdx.x;
      if (c < S.P.cells) b_static_geometry(S.P, S.F, c);
    }
  }
}

// Static face data of the momentum equation (the porosity never changes): 1 / phi_f
// with phi_f the mean of the face's two cells, and grad(phi^-2) at the face --
// across it along its own axis, the mean of the two cells' central differences
// along the others, stored times 1/4 because the assembly multiplies it with the sum
// (not the mean) of the four transverse face velocities (zero components beyond the
// grid's dimension).
__device__ __forceinline__ void b_static_faces(const Prm& P, const Fld& F, long long t) {
  int d, i, j, k;
  long long f;
  if (!decode_face(P, t, d, i, j, k, f)) return;
  const long long nf = P.nf[d];
  const int li = i - (d == 0), lj = j - (d == 1), lk = k - (d == 2);
  const double phif = 0.5 * (ghost_read(F.phi, P.n, li, lj, lk) + ghost_read(F.phi, P.n, i, j, k));
  const_cast<double*>(F.iphif[d])[f] = 1.0 / phif;
  const double inv_h = P.inv_h;
  for (int e = 0; e < 3; e++) {
    const int ei = (e == 0), ej = (e == 1), ek = (e == 2);
    double g = 0.0;
    if (e == d) {
      g = (ghost_read(F.iphi2, P.n, i, j, k) - ghost_read(F.iphi2, P.n, li, lj, lk)) * inv_h;
    } else if (e < P.dim) {
      const double gL = ghost_read(F.iphi2, P.n, li + ei, lj + ej, lk + ek) -
                        ghost_read(F.iphi2, P.n, li - ei, lj - ej, lk - ek);
      const double gR = ghost_read(F.iphi2, P.n, i + ei, j + ej, k + ek) -
                        ghost_read(F.iphi2, P.n, i - ei, j - ej, k - ek);
      g = 0.25 * ((gL + gR) * (0.25 * inv_h));  // times 1/4: the momentum assembly sums, not averages, w
    }
    const_cast<double*>(F.gphi[d])[e * nf + f] = g;
  }
}

__global__ void k_static_faces(const StepDom* __restrict__ D, Work w) {
  MDBS_DEPENDENT_ENTRY();
  for (int b = blockIdx.x; b < w.total; b += gridDim.x) {
    const int dm = work_domain(w, b);
    const StepDom& S = D[dm];
    const int lb = b - w.blk[dm];
    for (int r = 0; r < w.rep; r++) {
      const long long t = ((long long)lb * w.rep + r) * blockDim.x + threadIdx.x;
      if (t < total_faces(S.P)) b_static_faces(S.P, S.F, t);
    }
  }
}

// ------------------------------------------------------------------ batched entry points
__global__ void k_alpha_lo(const StepDom* __restrict__ D, Work w) {
  MDBS_DEPENDENT_ENTRY();
  for (int b = blockIdx.x; b < w.total; b += gridDim.x) {
    const int dm = work_domain(w, b);
    const StepDom& S = D[dm];
    const int lb = b - w.blk[dm];
    for (int r = 0; r < w.rep; r++) {
      const long long c = ((long long)lb * w.rep + r) * blockDim.x + threadIdx.x;
      if (c < S.P.cells) b_alpha_lo(S.P, S.F, c, S.scal[kSlotDt]);
    }
  }
}

// 5 CTAs per SM (51 registers): measured faster than the unbounded allocation
__global__ void __launch_bounds__(kBlock, 5) k_alpha_limit(const StepDom* __restrict__ D, Work w) {
  MDBS_DEPENDENT_ENTRY();
  __shared__ double s_inv_dt;  // one FP64 division per block, not per cell
  for (int b = blockIdx.x; b < w.total; b += gridDim.x) {
    const int dm = work_domain(w, b);
    const StepDom& S = D[dm];
    const int lb = b - w.blk[dm];
    __syncthreads();  // the previous item's readers are done
    if (threadIdx.x == 0) s_inv_dt = 1.0 / S.scal[kSlotDt];
    __syncthreads();
    const double inv_dt = s_inv_dt;
    for (int r = 0; r < w.rep; r++) {
      const long long c = ((long long)lb * w.rep + r) * blockDim.x + threadIdx.x;
      if (c < S.P.cells) b_alpha_limit(S.P, S.F, c, inv_dt);
    }
  }
}

__global__ void k_alpha_update(const StepDom* __restrict__ D, Work w) {
  MDBS_DEPENDENT_ENTRY();
  for (int b = blockIdx.x; b < w.total; b += gridDim.x) {
    const int dm = work_domain(w, b);
    const StepDom& S = D[dm];
    const int lb = b - w.blk[dm];
    for (int r = 0; r < w.rep; r++) {
      const long long c = ((long long)lb * w.rep + r) * blockDim.x + threadIdx.x;
      if (c < S.P.cells) b_alpha_update(S.P, S.F, c, S.scal[kSlotDt]);
    }
  }
}

__global__ void k_properties(const StepDom* __restrict__ D, Work w) {
  MDBS_DEPENDENT_ENTRY();
  for (int b = blockIdx.x; b < w.total; b += gridDim.x) {
    const int dm = work_domain(w, b);
    const StepDom& S = D[dm];
    const int lb = b - w.blk[dm];
    for (int r = 0; r < w.rep; r++) {
      const long long c = ((long long)lb * w.rep + r) * blockDim.x + threadIdx.x;
      if (c < S.P.cells) b_properties(S.P, S.F, c);
    }
  }
}

__global__ void k_normals(const StepDom* __restrict__ D, Work w) {
  MDBS_DEPENDENT_ENTRY();
  for (int b = blockIdx.x; b < w.total; b += gridDim.x) {
    const int dm = work_domain(w, b);
    const StepDom& S = D[dm];
    const int lb = b - w.blk[dm];
    for (int r = 0; r < w.rep; r++) {
      const long long c = ((long long)lb * w.rep + r) * blockDim.x + threadIdx.x;
      if (c < S.P.cells) b_normals(S.P, S.F, c);
    }
  }
}

__global__ void k_edge_mu(const StepDom* __restrict__ D, Work w) {
  MDBS_DEPENDENT_ENTRY();
  for (int b = blockIdx.x; b < w.total; b += gridDim.x) {
    const int dm = work_domain(w, b);
    const StepDom& S = D[dm];
    const int lb = b - w.blk[dm];
    for (int r = 0; r < w.rep; r++) {
      const long long c = ((long long)lb * w.rep + r) * blockDim.x + threadIdx.x;
      if (c < S.P.cells) b_edge_mu(S.P, S.F, c);
    }
  }
}

__global__ void k_curvature(const StepDom* __restrict__ D, Work w) {
  MDBS_DEPENDENT_ENTRY();
  for (int b = blockIdx.x; b < w.total; b += gridDim.x) {
    const int dm = work_domain(w, b);
    const StepDom& S = D[dm];
    const int lb = b - w.blk[dm];
    for (int r = 0; r < w.rep; r++) {
      const long long c = ((long long)lb * w.rep + r) * blockDim.x + threadIdx.x;
      if (c < S.P.cells) b_curvature(S.P, S.F, c);
    }
  }
}

// 3 CTAs per SM (80 registers): FP64-pipe bound, the extra warps hide its load latency
__global__ void __launch_bounds__(kBlock, 3) k_momentum_assemble(const StepDom* __restrict__ D, Work w) {
  MDBS_DEPENDENT_ENTRY();
  __shared__ double s_inv_dt;  // one FP64 division per block, not per face
  for (int b = blockIdx.x; b < w.total; b += gridDim.x) {
    const int dm = work_domain(w, b);
    const StepDom& S = D[dm];
    const int lb = b - w.blk[dm];
    __syncthreads();  // the previous item's readers are done
    if (threadIdx.x == 0) s_inv_dt = 1.0 / S.scal[kSlotDt];
    __syncthreads();
    const double inv_dt = s_inv_dt;
    for (int r = 0; r < w.rep; r++) {
      const long long t = ((long long)lb * w.rep + r) * blockDim.x + threadIdx.x;
      if (t < total_faces(S.P)) b_momentum_assemble(S.P, S.F, t, inv_dt);
    }
  }
}

__global__ void k_jacobi(const StepDom* __restrict__ D, Work w, int parity) {
  MDBS_DEPENDENT_ENTRY();
  for (int b = blockIdx.x; b < w.total; b += gridDim.x) {
    const int dm = work_domain(w, b);
    const StepDom& S = D[dm];
    const int lb = b - w.blk[dm];
    // even sweeps u -> utmp, odd sweeps utmp -> u
    const double* const* in = parity ? S.F.utmp : S.F.u;
    double* const* out = parity ? S.F.u : S.F.utmp;
    for (int r = 0; r < w.rep; r++) {
      const long long t = ((long long)lb * w.rep + r) * blockDim.x + threadIdx.x;
      b_jacobi(S.P, S.F, t, in, out);
    }
  }
}

// 6 CTAs per SM (40 registers): measured faster than the unbounded allocation
__global__ void __launch_bounds__(kBlock, 6) k_hbya(const StepDom* __restrict__ D, Work w) {
  MDBS_DEPENDENT_ENTRY();
  for (int b = blockIdx.x; b < w.total; b += gridDim.x) {
    const int dm = work_domain(w, b);
    const StepDom& S = D[dm];
    const int lb = b - w.blk[dm];
    for (int r = 0; r < w.rep; r++) {
      const long long t = ((long long)lb * w.rep + r) * blockDim.x + threadIdx.x;
      if (t < total_faces(S.P)) b_hbya(S.P, S.F, t);
    }
  }
}

__global__ void k_correct(const StepDom* __restrict__ D, Work w) {
  MDBS_DEPENDENT_ENTRY();
  for (int b = blockIdx.x; b < w.total; b += gridDim.x) {
    const int dm = work_domain(w, b);
    const StepDom& S = D[dm];
    const int lb = b - w.blk[dm];
    for (int r = 0; r < w.rep; r++) {
      const long long t = ((long long)lb * w.rep + r) * blockDim.x + threadIdx.x;
      if (t < total_faces(S.P)) b_correct(S.P, S.F, t);
    }
  }
}

__global__ void k_boundary_velocities(const StepDom* __restrict__ D, Work w) {
  MDBS_DEPENDENT_ENTRY();
  for (int b = blockIdx.x; b < w.total; b += gridDim.x) {
    const int dm = work_domain(w, b);
    const StepDom& S = D[dm];
    const int lb = b - w.blk[dm];
    for (int r = 0; r < w.rep; r++) {
      const long long t = ((long long)lb * w.rep + r) * blockDim.x + threadIdx.x;
      if (t < total_faces(S.P)) b_boundary_velocities(S.P, S.F, t);
    }
  }
}

}  // namespace

// ------------------------------------------------------------------ launchers
#define BATCH_LAUNCH(ID, SPACE, KERNEL, ...) \
  MDBS_LAUNCH(ID, grid_of(B, B.SPACE), kBlock, s, KERNEL, B.sd, B.SPACE, ##__VA_ARGS__)

void launch_alpha_step(const BatchPlan& B, cudaStream_t s) {
  BATCH_LAUNCH(K_ALPHA_FLUX, rfaces, k_alpha_flux);
  MDBS_LAUNCH(K_FINALIZE, B.ndom, 1024, s, k_finalize_inflow, B.sd, B.rfaces, kSlotInflow);
  BATCH_LAUNCH(K_ALPHA_LO, cells, k_alpha_lo);
  BATCH_LAUNCH(K_ALPHA_LIMIT, cells, k_alpha_limit);
  BATCH_LAUNCH(K_ALPHA_UPDATE, cells, k_alpha_update);
}

void launch_closures(const BatchPlan& B, cudaStream_t s) { BATCH_LAUNCH(K_PROPERTIES, cells, k_properties); }

void launch_properties(const BatchPlan& B, cudaStream_t s) {
  BATCH_LAUNCH(K_PROPERTIES, cells, k_properties);
  BATCH_LAUNCH(K_EDGE_MU, cells, k_edge_mu);  // reads the viscosity the closures just formed
  BATCH_LAUNCH(K_NORMALS, cells, k_normals);
  BATCH_LAUNCH(K_CURVATURE, cells, k_curvature);
}

void launch_momentum_assemble(const BatchPlan& B, cudaStream_t s) {
  BATCH_LAUNCH(K_MOM_ASSEMBLE, faces, k_momentum_assemble);
}

void launch_jacobi_sweeps(const BatchPlan& B, int sweeps, cudaStream_t s) {
  for (int it = 0; it < sweeps; it++) BATCH_LAUNCH(K_JACOBI, faces, k_jacobi, it & 1);
  // an odd sweep count leaves the result in the scratch buffers
  if (sweeps & 1) BATCH_LAUNCH(K_JACOBI, faces, k_copy_faces);
}

void launch_hbya(const BatchPlan& B, cudaStream_t s) { BATCH_LAUNCH(K_HBYA, faces, k_hbya); }

void launch_correct(const BatchPlan& B, cudaStream_t s) { BATCH_LAUNCH(K_CORRECT, faces, k_correct); }

void launch_set_boundary_velocities(const BatchPlan& B, cudaStream_t s) {
  BATCH_LAUNCH(K_BOUNDARY, faces, k_boundary_velocities);
}

void launch_field_stats(const BatchPlan& B, cudaStream_t s) {
  BATCH_LAUNCH(K_STATS, rcells, k_field_stats);
  MDBS_LAUNCH(K_FINALIZE, B.ndom, 1024, s, k_finalize_stats, B.sd, B.rcells);
}

void launch_time_advance(const BatchPlan& B, cudaStream_t s) {
  if (B.any_cfl) BATCH_LAUNCH(K_CFL, rfaces, k_cfl);
  MDBS_LAUNCH(K_FINALIZE, B.ndom, 1024, s, k_finalize_time, B.sd, B.rfaces);
}

void launch_static_geometry(const BatchPlan& B, cudaStream_t s) {
  BATCH_LAUNCH(K_STATIC, cells, k_static_geometry);
  BATCH_LAUNCH(K_STATIC, faces, k_static_faces);  // reads phi^-2 of the cells
}

}  // namespace mdbs
