/*
 * oracle.c -- plain FP64 CPU oracle of one pressure-velocity time step of the
 * two-phase micro-continuum DBS-VOF model of Carrillo, Bourg & Soulaine
 * (arXiv 2003.08374).
 *
 * TEST INFRASTRUCTURE ONLY: used by tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py.  Never a runtime fallback.  It
 * shares no code with the CUDA library.
 *
 * Written for clarity, not speed: one loop per formula, serial reductions in a
 * fixed order, no blocking or fusion.  Each block cites the passage it follows.
 * The discrete choices the paper leaves open are the documented readings of
 * the project (staggered MAC grid, face averages, Zalesak limiter, GMG-PCG).
 *
 * Step order (paper section 3.2, "Solution algorithm"):
 *   1. explicit saturation update by flux-corrected transport (MULES), Eq. 15
 *   2. boundary values (fixed wall / inlet face velocities)
 *   3. properties k, rho, mu from alpha^{k+1}; capillary force, Eqs. 41-45
 *   4. momentum predictor with grad p^k, Eq. 50
 *   5. PISO correctors: pressure equation Eq. 53, corrected velocity Eq. 51
 *   6. next time step from the CFL number
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define MAXLEV 16
enum { EXISTS = 0, MIRROR = 1, COPY = 2 };
enum { F_INTERIOR = 0, F_FIXED = 1, F_OUTLET = 2 };

typedef struct {
  int n[3];
  long cells;
  int cz[3]; /* axis coarsened relative to the finer level */
  double *Tx, *Ty, *Tz, *Dd, *diag, *x, *b, *r;
} level_t;

struct orc_state {
  orc_params P;
  int n[3], dim;
  long cells, nf[3];
  double h, A, V, dt, time;
  double *phi, *k0;
  unsigned char* is_free;
  unsigned char* has_nw;
  double* nw[3];
  double *alpha, *p, *u[3];
  /* properties */
  double *Ml, *Mg, *pc, *cf, *rho, *mu, *drag, *m[3], *kappa;
  /* alpha step */
  double *FLO[3], *AF[3], *aL, *Rp, *Rm;
  /* momentum */
  double *aP[3], *anb[3], *rhs0[3], *unew[3], *hbya[3], *B[3];
  /* pressure */
  level_t lev[MAXLEV];
  int nlev;
  double *cg_r, *cg_z, *cg_d, *cg_q;
  orc_stats st;
};

/* ------------------------------------------------------------------ */
/* indexing                                                             */
/* ------------------------------------------------------------------ */
static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }
static long cid3(const int n[3], const int c[3]) { return c[0] + (long)n[0] * (c[1] + (long)n[1] * c[2]); }
static long cidv(const orc_state* s, const int c[3]) { return cid3(s->n, c); }
static long fidv(const orc_state* s, int d, const int c[3]) {
  long fx = s->n[0] + (d == 0), fy = s->n[1] + (d == 1);
  return c[0] + fx * (c[1] + fy * (long)c[2]);
}
/* cell value with zero-gradient ghosts: coordinates clamped into the grid */
static double cval(const orc_state* s, const double* a, const int c[3]) {
  int q[3];
  for (int e = 0; e < 3; e++) q[e] = clampi(c[e], 0, s->n[e] - 1);
  return a[cidv(s, q)];
}
/* Van Leer limited face value (section 3.1): the upwind value plus half the
 * limited difference toward the downwind cell, psi(r) = (r + |r|)/(1 + |r|)
 * with r the ratio of the upwind to the face difference; psi -> 2 as r -> +inf
 * (a face difference too small for the ratio to be finite). */
static double van_leer(double aU, double aD, double aUU) {
  double den = aD - aU;
  if (den == 0.0) return aU;
  double r = (aU - aUU) / den;
  double psi = isinf(r) ? (r > 0.0 ? 2.0 : 0.0) : (r + fabs(r)) / (1.0 + fabs(r));
  return aU + 0.5 * psi * den;
}
/* liquid fractional flow M_l / M of the cell at c (clamped into the grid like
 * cval); a cell without mobilities (solid-free) gives its saturation */
static double frac_flow(const orc_state* s, const int c[3]) {
  int q[3];
  for (int e = 0; e < 3; e++) q[e] = clampi(c[e], 0, s->n[e] - 1);
  long i = cidv(s, q);
  double M = s->Ml[i] + s->Mg[i];
  return M > 0.0 ? s->Ml[i] / M : s->alpha[i];
}
static void cpy3(int dst[3], const int src[3]) { dst[0] = src[0]; dst[1] = src[1]; dst[2] = src[2]; }
/* phi^-2 of the cell at c, zero-gradient ghosts */
static double inv_phi2(const orc_state* s, const int c[3]) {
  double ph = cval(s, s->phi, c);
  return 1.0 / (ph * ph);
}
static void coords_of(const int n[3], long idx, int c[3]) {
  c[0] = (int)(idx % n[0]);
  c[1] = (int)((idx / n[0]) % n[1]);
  c[2] = (int)(idx / ((long)n[0] * n[1]));
}
static void face_dims(const orc_state* s, int d, int fn[3]) {
  cpy3(fn, s->n);
  fn[d] += 1;
}
static int face_kind(const orc_state* s, int d, const int c[3]) {
  if (c[d] > 0 && c[d] < s->n[d]) return F_INTERIOR;
  int side = 2 * d + (c[d] == 0 ? 0 : 1);
  return s->P.bc[side] == ORC_OUTLET ? F_OUTLET : F_FIXED;
}
/* e-direction face velocity on the low (hi=0) or high (hi=1) e-face of the
 * cell at c; a ghost cell (outside the grid) is replaced by its interior
 * neighbour. */
static double ue_cell(const orc_state* s, int e, const int c[3], int hi) {
  int q[3];
  for (int a = 0; a < 3; a++) q[a] = clampi(c[a], 0, s->n[a] - 1);
  q[e] += hi;
  return s->u[e][fidv(s, e, q)];
}

/* ------------------------------------------------------------------ */
/* closures (Appendix A; Eqs. 37, 38, 42, 45)                           */
/* ------------------------------------------------------------------ */
static void rel_perm(const orc_params* P, double a, double* krl, double* krg) {
  /* effective saturation, Appendix A.1 */
  double ae = (a - P->a_l_irr) / (1.0 - P->a_g_irr - P->a_l_irr);
  if (ae < 0.0) ae = 0.0;
  if (ae > 1.0) ae = 1.0;
  double m = P->kr_m;
  if (P->kr_model == 0) { /* Brooks-Corey */
    *krl = pow(ae, m);
    *krg = pow(1.0 - ae, m);
  } else { /* Van Genuchten */
    double s1m = pow(ae, 1.0 / m);
    *krg = sqrt(1.0 - ae) * pow(1.0 - s1m, 2.0 * m);
    double t = 1.0 - pow(1.0 - s1m, m);
    *krl = sqrt(ae) * t * t;
  }
}

static double cap_pressure(const orc_params* P, double a) {
  /* effective saturation for p_c, Appendix A.2, clamped away from the
   * singular end points by pc_eps */
  double s = (a - P->a_pc_irr) / (P->a_pc_max - P->a_pc_irr);
  if (s < P->pc_eps) s = P->pc_eps;
  if (s > 1.0 - P->pc_eps) s = 1.0 - P->pc_eps;
  if (P->pc_model == 0) return P->pc0 * pow(s, -P->pc_beta);     /* Brooks-Corey */
  return P->pc0 * pow(pow(s, -1.0 / P->pc_m) - 1.0, 1.0 - P->pc_m); /* Van Genuchten */
}

void orc_closures(const orc_params* P, double a, double k0, double* out) {
  double krl, krg;
  rel_perm(P, a, &krl, &krg);
  double Ml = k0 * krl / P->mu_l; /* mobilities M_i = k0 k_ri / mu_i, Eq. 30 */
  double Mg = k0 * krg / P->mu_g;
  double M = Ml + Mg;
  out[0] = krl;
  out[1] = krg;
  out[2] = Ml;
  out[3] = Mg;
  out[4] = 1.0 / M;                                /* mu k^-1 = M^-1, Eq. 42 */
  out[5] = (P->rho_l * Ml + P->rho_g * Mg) / M;    /* rho*, Eq. 45 porous branch */
  out[6] = cap_pressure(P, a);                     /* p_c, Appendix A.2 */
  out[7] = (Ml * (1.0 - a) - Mg * a) / M;          /* M^-1 (M_l a_g - M_g a_l), Eq. 38 */
}

static void update_props(orc_state* s) {
  const orc_params* P = &s->P;
  for (long c = 0; c < s->cells; c++) {
    double a = s->alpha[c];
    s->mu[c] = a * P->mu_l + (1.0 - a) * P->mu_g; /* mu = a_l mu_l + a_g mu_g, Eq. 18 */
    if (s->is_free[c]) {
      /* solid-free cell: no drag (Eq. 42), alpha-weighted density (Eq. 45) */
      s->Ml[c] = 0.0;
      s->Mg[c] = 0.0;
      s->drag[c] = 0.0;
      s->pc[c] = 0.0;
      s->cf[c] = 0.0;
      s->rho[c] = a * P->rho_l + (1.0 - a) * P->rho_g;
    } else {
      double o[8];
      orc_closures(P, a, s->k0[c], o);
      s->Ml[c] = o[2];
      s->Mg[c] = o[3];
      s->drag[c] = o[4];
      /* rho* of Eq. 45, or Appendix B's saturation-weighted density */
      s->rho[c] = P->porous_density ? a * P->rho_l + (1.0 - a) * P->rho_g : o[5];
      s->pc[c] = o[6];
      s->cf[c] = o[7];
    }
  }
}

/* central-difference gradient at a cell, zero-gradient ghosts */
static void grad_cell(const orc_state* s, const double* a, const int c[3], double g[3]) {
  g[0] = g[1] = g[2] = 0.0;
  for (int e = 0; e < s->dim; e++) {
    int lo[3], hi[3];
    cpy3(lo, c);
    cpy3(hi, c);
    lo[e] -= 1;
    hi[e] += 1;
    g[e] = (cval(s, a, hi) - cval(s, a, lo)) / (2.0 * s->h);
  }
}

/* interface normals (Eq. 24, oriented toward the liquid), contact-angle
 * correction at the free/porous interface (Eq. 40 / 44) and curvature
 * kappa = -div(m) used in the CSF force (Eq. 27 / 43).  Solid-free cells take
 * their gradients from the fluid side only (free_side). */
/* value of a at the neighbour nb as a solid-free cell c sees it: a porous
 * neighbour counts as a zero-gradient ghost (c's own value), like a wall, so
 * that the normal and curvature next to the porous surface come from the fluid
 * side before the contact angle replaces the normal (section 2.3, Eq. 40) */
static double free_side(const orc_state* s, const double* a, const int c[3], const int nb[3]) {
  int q[3];
  for (int e = 0; e < 3; e++) q[e] = clampi(nb[e], 0, s->n[e] - 1);
  long i = cidv(s, q);
  if (s->is_free[cidv(s, c)] && !s->is_free[i]) return a[cidv(s, c)];
  return a[i];
}
static void normals_curvature(orc_state* s) {
  double dn = 1e-8 / s->h;
  double th = s->P.theta_deg * M_PI / 180.0;
  double ct = cos(th), st = sin(th);
  for (long c = 0; c < s->cells; c++) {
    int q[3];
    coords_of(s->n, c, q);
    double g[3] = {0.0, 0.0, 0.0};
    for (int e = 0; e < s->dim; e++) {
      int lo[3], hi[3];
      cpy3(lo, q);
      cpy3(hi, q);
      lo[e] -= 1;
      hi[e] += 1;
      g[e] = (free_side(s, s->alpha, q, hi) - free_side(s, s->alpha, q, lo)) / (2.0 * s->h);
    }
    double mag = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    for (int e = 0; e < 3; e++) s->m[e][c] = g[e] / (mag + dn);
  }
  for (long c = 0; c < s->cells; c++) {
    if (!s->has_nw[c]) continue;
    double mv[3] = {s->m[0][c], s->m[1][c], s->m[2][c]};
    double nw[3] = {s->nw[0][c], s->nw[1][c], s->nw[2][c]};
    double mm = sqrt(mv[0] * mv[0] + mv[1] * mv[1] + mv[2] * mv[2]);
    double mn = mv[0] * nw[0] + mv[1] * nw[1] + mv[2] * nw[2];
    double t[3], tn = 0.0;
    for (int e = 0; e < 3; e++) {
      t[e] = mv[e] - mn * nw[e];
      tn += t[e] * t[e];
    }
    tn = sqrt(tn);
    for (int e = 0; e < 3; e++) {
      /* the wall tangent is undefined when the interface lies parallel to the
       * surface: a tangential part below 1e-9 |m| is rounding, not a direction */
      double te = tn > 1e-9 * mm ? t[e] / tn : 0.0;
      s->m[e][c] = mm * (ct * nw[e] + st * te);
    }
  }
  for (long c = 0; c < s->cells; c++) {
    int q[3];
    coords_of(s->n, c, q);
    double k = 0.0;
    for (int e = 0; e < s->dim; e++) {
      int lo[3], hi[3];
      cpy3(lo, q);
      cpy3(hi, q);
      lo[e] -= 1;
      hi[e] += 1;
      k -= (free_side(s, s->m[e], q, hi) - free_side(s, s->m[e], q, lo)) / (2.0 * s->h);
    }
    s->kappa[c] = k;
  }
}

/* ------------------------------------------------------------------ */
/* 1. saturation equation, Eq. 15, by flux-corrected transport           */
/* ------------------------------------------------------------------ */
static void alpha_step(orc_state* s, double dt) {
  const orc_params* P = &s->P;
  double h = s->h, A = s->A, V = s->V;
  double dn = 1e-8 / h;
  double inflow = 0.0;
  for (int d = 0; d < s->dim; d++) {
    int fn[3];
    face_dims(s, d, fn);
    for (int k = 0; k < fn[2]; k++)
      for (int j = 0; j < fn[1]; j++)
        for (int i = 0; i < fn[0]; i++) {
          int c[3] = {i, j, k};
          long f = fidv(s, d, c);
          double Q = A * s->u[d][f]; /* volumetric face flux */
          int L[3], R[3];
          cpy3(L, c);
          cpy3(R, c);
          L[d] -= 1;
          int hasL = c[d] > 0, hasR = c[d] < s->n[d];
          if (hasL && hasR) {
            long l = cidv(s, L), r = cidv(s, R);
            double aU, aD, aUU;
            int UU[3];
            if (Q >= 0.0) {
              aU = s->alpha[l];
              aD = s->alpha[r];
              cpy3(UU, L);
              UU[d] -= 1;
            } else {
              aU = s->alpha[r];
              aD = s->alpha[l];
              cpy3(UU, R);
              UU[d] += 1;
            }
            aUU = cval(s, s->alpha, UU);
            double flo = Q * aU; /* upwind (low order) flux */
            double avl = van_leer(aU, aD, aUU);
            double Rf = 0.0;
            if (s->is_free[l] && s->is_free[r]) {
              /* compression relative velocity in solid-free faces, Eq. 22
               * with the sign of Eq. 41 (toward the liquid), face-local |v| */
              double gl[3], gr[3], gf[3], mag = 0.0;
              grad_cell(s, s->alpha, L, gl);
              grad_cell(s, s->alpha, R, gr);
              for (int e = 0; e < 3; e++) {
                gf[e] = 0.5 * (gl[e] + gr[e]);
                mag += gf[e] * gf[e];
              }
              mag = sqrt(mag);
              double nf = gf[d] / (mag + dn);
              double w = P->c_alpha * fabs(s->u[d][f]) * nf * A;
              if (w >= 0.0)
                Rf = w * s->alpha[l] * (1.0 - s->alpha[r]);
              else
                Rf = w * s->alpha[r] * (1.0 - s->alpha[l]);
            } else if (!s->is_free[l] && !s->is_free[r]) {
              /* porous relative flux phi a_l a_g v_r (Eq. 34).  With the
               * single-field velocity v = v_l + v_g (section 2.2), the liquid
               * Darcy flux a_l v + phi a_l a_g v_r of Eq. 34 equals
               * f v + lambda [(rho_l - rho_g) g + grad pc],
               * f = M_l / M, lambda = M_l M_g / M; Eq. 34 rewritten that way is
               * discretised with the face flux Q itself: f by the same Van Leer
               * limited upwind value as alpha (section 3.1), lambda by phase
               * upwinding along the gravity-capillary drive.  The relative flux is
               * that liquid flux minus the convective part Q * avl. */
              int Ucell[3], Dcell[3];
              cpy3(Ucell, Q >= 0.0 ? L : R);
              cpy3(Dcell, Q >= 0.0 ? R : L);
              double fU = frac_flow(s, Ucell), fD = frac_flow(s, Dcell), fUU = frac_flow(s, UU);
              double fvl = van_leer(fU, fD, fUU);
              double drive = (P->rho_l - P->rho_g) * P->g[d] + (s->pc[r] - s->pc[l]) / h;
              /* liquid from the cell the drive pushes it out of, gas from the other */
              double mlw = drive >= 0.0 ? s->Ml[l] : s->Ml[r];
              double mgw = drive >= 0.0 ? s->Mg[r] : s->Mg[l];
              double lam = (mlw + mgw) > 0.0 ? mlw * mgw / (mlw + mgw) : 0.0;
              Rf = Q * (fvl - avl) + A * lam * drive;
            }
            s->FLO[d][f] = flo;
            s->AF[d][f] = (Q * avl + Rf) - flo; /* anti-diffusive flux */
          } else {
            int side = 2 * d + (hasL ? 1 : 0);
            long cc = hasL ? cidv(s, L) : cidv(s, R);
            double flo = 0.0;
            if (P->bc[side] == ORC_INLET) {
              int in = (side & 1) ? (Q < 0.0) : (Q > 0.0);
              flo = Q * (in ? P->inlet_alpha : s->alpha[cc]);
            } else if (P->bc[side] == ORC_OUTLET) {
              flo = Q * s->alpha[cc];
            }
            s->FLO[d][f] = flo;
            s->AF[d][f] = 0.0;
            inflow += (side & 1) ? -flo : flo;
          }
        }
  }
  s->st.boundary_in += dt * inflow;

  /* low-order solution */
  for (long c = 0; c < s->cells; c++) {
    int q[3];
    coords_of(s->n, c, q);
    double div = 0.0;
    for (int d = 0; d < s->dim; d++) {
      int hi[3];
      cpy3(hi, q);
      hi[d] += 1;
      div += s->FLO[d][fidv(s, d, hi)] - s->FLO[d][fidv(s, d, q)];
    }
    s->aL[c] = s->alpha[c] - dt / (s->phi[c] * V) * div;
  }
  /* Zalesak limiter coefficients */
  for (long c = 0; c < s->cells; c++) {
    int q[3];
    coords_of(s->n, c, q);
    double amax = fmax(s->alpha[c], s->aL[c]);
    double amin = fmin(s->alpha[c], s->aL[c]);
    for (int d = 0; d < s->dim; d++)
      for (int sg = -1; sg <= 1; sg += 2) {
        int nb[3];
        cpy3(nb, q);
        nb[d] += sg;
        if (nb[d] < 0 || nb[d] >= s->n[d]) continue;
        long b = cidv(s, nb);
        amax = fmax(amax, fmax(s->alpha[b], s->aL[b]));
        amin = fmin(amin, fmin(s->alpha[b], s->aL[b]));
      }
    amax = fmin(1.0, amax);
    amin = fmax(0.0, amin);
    if (!s->is_free[c]) {
      /* porous cell: the relative flux is the physical Darcy phase flux
       * (Eq. 34), which may create new extrema; bound by [0, 1] only */
      amax = 1.0;
      amin = 0.0;
    }
    double fac = s->phi[c] * V / dt;
    double Qp = fmax(0.0, amax - s->aL[c]) * fac;
    double Qm = fmax(0.0, s->aL[c] - amin) * fac;
    double Pp = 0.0, Pm = 0.0;
    for (int d = 0; d < s->dim; d++) {
      int hi[3];
      cpy3(hi, q);
      hi[d] += 1;
      double alo = s->AF[d][fidv(s, d, q)], ahi = s->AF[d][fidv(s, d, hi)];
      Pp += fmax(0.0, alo) + fmax(0.0, -ahi);
      Pm += fmax(0.0, -alo) + fmax(0.0, ahi);
    }
    s->Rp[c] = Pp > 0.0 ? fmin(1.0, Qp / Pp) : 1.0;
    s->Rm[c] = Pm > 0.0 ? fmin(1.0, Qm / Pm) : 1.0;
  }
  /* limited update */
  for (long c = 0; c < s->cells; c++) {
    int q[3];
    coords_of(s->n, c, q);
    double corr = 0.0;
    for (int d = 0; d < s->dim; d++) {
      double la[2];
      for (int side = 0; side < 2; side++) {
        int fc[3];
        cpy3(fc, q);
        fc[d] += side;
        la[side] = 0.0;
        if (fc[d] == 0 || fc[d] == s->n[d]) continue; /* boundary: no correction */
        int L[3];
        cpy3(L, fc);
        L[d] -= 1;
        long l = cidv(s, L), r = cidv(s, fc);
        double a = s->AF[d][fidv(s, d, fc)];
        double lam = a >= 0.0 ? fmin(s->Rm[l], s->Rp[r]) : fmin(s->Rp[l], s->Rm[r]);
        la[side] = lam * a;
      }
      corr += la[1] - la[0];
    }
    s->alpha[c] = s->aL[c] - dt / (s->phi[c] * V) * corr;
  }
}

/* ------------------------------------------------------------------ */
/* 3-4. face forces and momentum predictor, Eqs. 46-50                  */
/* ------------------------------------------------------------------ */
static void momentum_assemble(orc_state* s, double dt) {
  const orc_params* P = &s->P;
  double h = s->h, A = s->A, V = s->V;
  for (int d = 0; d < s->dim; d++) {
    int fn[3];
    face_dims(s, d, fn);
    for (int k = 0; k < fn[2]; k++)
      for (int j = 0; j < fn[1]; j++)
        for (int i = 0; i < fn[0]; i++) {
          int c[3] = {i, j, k};
          long f = fidv(s, d, c);
          double* an = s->anb[d] + f * 6;
          for (int q = 0; q < 6; q++) an[q] = 0.0;
          int kind = face_kind(s, d, c);
          if (kind == F_FIXED) {
            s->aP[d][f] = 1.0;
            s->rhs0[d][f] = 0.0;
            s->B[d][f] = 0.0;
            continue;
          }
          int L[3], R[3];
          cpy3(L, c);
          cpy3(R, c);
          L[d] -= 1;
          double phif = 0.5 * (cval(s, s->phi, L) + cval(s, s->phi, R));
          double rhof = 0.5 * (cval(s, s->rho, L) + cval(s, s->rho, R));
          double Df = 0.5 * (cval(s, s->drag, L) + cval(s, s->drag, R));
          /* face body force: gravity rho g (Eq. 45 density) and capillary F_c */
          double G = rhof * P->g[d];
          double F = 0.0;
          if (kind == F_INTERIOR) {
            long l = cidv(s, L), r = cidv(s, R);
            if (s->is_free[l] && s->is_free[r]) {
              /* CSF, Eq. 27 / 43: F = sigma kappa grad(alpha) */
              F = P->sigma * 0.5 * (s->kappa[l] + s->kappa[r]) * (s->alpha[r] - s->alpha[l]) / h;
            } else if (!s->is_free[l] && !s->is_free[r]) {
              /* porous capillary force, Eq. 38 (dp_c/da grad a = grad p_c) */
              F = (0.5 * (s->cf[l] + s->cf[r]) * (s->pc[r] - s->pc[l]) -
                   0.5 * (s->pc[l] + s->pc[r]) * (s->alpha[r] - s->alpha[l])) /
                  h;
              /* Appendix B: with the saturation-weighted density, F_c also
               * carries M^-1 (M_l a_g - M_g a_l)(rho_l - rho_g) g */
              if (P->porous_density)
                F += 0.5 * (s->cf[l] + s->cf[r]) * (P->rho_l - P->rho_g) * P->g[d];
            }
          }
          s->B[d][f] = G + F;
          /* Euler implicit inertia with the 1/phi factors of Eq. 21, in
           * advective form rho^{k+1} (v^{k+1} - v^k) / dt: with the upwind
           * advective convection below it is the same equation as the
           * conservative form, which would need momentum fluxes consistent
           * with the saturation fluxes (a water/air interface leaving a face
           * otherwise hands water momentum to air) */
          double at = V * rhof / (phif * dt);
          double S = at * s->u[d][f];
          double cconv = V * rhof / (phif * phif * h);
          double ap = at + V * Df; /* Darcy drag K_fs, Eq. 46 */
          double TT = 0.0;        /* explicit div(mu grad(v)^T) */
          double vgrad = 0.0;     /* v . grad(phi^-2) at the face */
          for (int e = 0; e < s->dim; e++) {
            for (int sg = -1; sg <= 1; sg += 2) {
              int slot = 2 * e + (sg > 0);
              int nb[3];
              cpy3(nb, c);
              nb[e] += sg;
              int status;
              if (e == d) {
                status = (nb[d] >= 0 && nb[d] <= s->n[d]) ? EXISTS : COPY;
              } else if (nb[e] >= 0 && nb[e] < s->n[e]) {
                status = EXISTS;
              } else {
                int side = 2 * e + (sg > 0);
                status = P->bc[side] == ORC_OUTLET ? COPY : MIRROR;
              }
              double w;
              if (e == d)
                w = s->u[d][f];
              else
                w = 0.25 * (ue_cell(s, e, L, 0) + ue_cell(s, e, L, 1) + ue_cell(s, e, R, 0) +
                            ue_cell(s, e, R, 1));
              if (sg < 0) {
                /* e-derivative of phi^-2 at the face: across it (e == d), or the mean
                 * of the two cells' central differences (e != d) */
                double ge;
                if (e == d) {
                  ge = (inv_phi2(s, R) - inv_phi2(s, L)) / h;
                } else {
                  int Lm[3], Lp[3], Rm[3], Rp[3];
                  cpy3(Lm, L);
                  cpy3(Lp, L);
                  cpy3(Rm, R);
                  cpy3(Rp, R);
                  Lm[e] -= 1;
                  Lp[e] += 1;
                  Rm[e] -= 1;
                  Rp[e] += 1;
                  ge = ((inv_phi2(s, Lp) - inv_phi2(s, Lm)) + (inv_phi2(s, Rp) - inv_phi2(s, Rm))) / (4.0 * h);
                }
                vgrad += w * ge;
              }
              double cup = cconv * (sg < 0 ? fmax(w, 0.0) : fmax(-w, 0.0));
              double mus;
              if (e == d) {
                mus = sg < 0 ? cval(s, s->mu, L) : cval(s, s->mu, R);
              } else {
                int L2[3], R2[3];
                cpy3(L2, L);
                cpy3(R2, R);
                L2[e] += sg;
                R2[e] += sg;
                mus = 0.25 * (cval(s, s->mu, L) + cval(s, s->mu, R) + cval(s, s->mu, L2) +
                              cval(s, s->mu, R2));
              }
              double a = cup + mus * A / h;
              if (status == EXISTS) {
                an[slot] = a;
                ap += a;
              } else if (status == MIRROR) {
                ap += 2.0 * a;
              }
            }
            /* transpose part of the viscous stress, lagged (Eq. 21, S = mu(grad v + grad v^T)) */
            if (e == d) {
              int fp[3], fm[3];
              cpy3(fp, c);
              cpy3(fm, c);
              fp[d] += 1;
              fm[d] -= 1;
              double dR = fp[d] <= s->n[d] ? (s->u[d][fidv(s, d, fp)] - s->u[d][f]) / h : 0.0;
              double dL = fm[d] >= 0 ? (s->u[d][f] - s->u[d][fidv(s, d, fm)]) / h : 0.0;
              TT += (cval(s, s->mu, R) * dR - cval(s, s->mu, L) * dL) / h;
            } else {
              double tsum = 0.0;
              for (int sg = -1; sg <= 1; sg += 2) {
                int L2[3], R2[3];
                cpy3(L2, L);
                cpy3(R2, R);
                L2[e] += sg;
                R2[e] += sg;
                double muE = 0.25 * (cval(s, s->mu, L) + cval(s, s->mu, R) + cval(s, s->mu, L2) +
                                     cval(s, s->mu, R2));
                int hi = sg > 0;
                double der = (ue_cell(s, e, R, hi) - ue_cell(s, e, L, hi)) / h;
                tsum += (sg > 0 ? muE * der : -muE * der);
              }
              TT += tsum / h;
            }
          }
          /* The rest of Eq. 21's convection.  (1/phi) div(rho v v / phi) equals the
           * advective (rho/phi^2)(v.grad)v above plus (1/phi) v div(rho v / phi); with
           * div v = 0 and the density carried by the flow (its part cancels the
           * v d(rho)/dt left out of the Euler term), what remains is
           * (rho/phi) v (v.grad(1/phi)) = (rho/2) v (v.grad(phi^-2)), non-zero only where
           * the porosity varies along the flow.  Its coefficient Gp multiplies u_f:
           * implicit (on the diagonal) where it decelerates the flow, explicit where it
           * accelerates it. */
          double Gp = 0.5 * rhof * vgrad;
          if (Gp >= 0.0)
            ap += V * Gp;
          else
            S -= V * Gp * s->u[d][f];
          s->aP[d][f] = ap;
          s->rhs0[d][f] = S + V * (TT + s->B[d][f]);
        }
  }
}

/* H(u)_f = sum_nb a_nb u_nb + rhs0 for an unknown face (Eq. 48) */
static double face_H(const orc_state* s, int d, const int c[3]) {
  long f = fidv(s, d, c);
  const double* an = s->anb[d] + f * 6;
  double hs = 0.0;
  for (int e = 0; e < s->dim; e++)
    for (int sg = -1; sg <= 1; sg += 2) {
      int slot = 2 * e + (sg > 0);
      if (an[slot] == 0.0) continue;
      int nb[3];
      cpy3(nb, c);
      nb[e] += sg;
      hs += an[slot] * s->u[d][fidv(s, d, nb)];
    }
  return hs + s->rhs0[d][f];
}

/* p_R - p_L across a face; the outlet ghost holds -p so that p = 0 on the face */
static double face_dp(const orc_state* s, int d, const int c[3]) {
  int L[3];
  cpy3(L, c);
  L[d] -= 1;
  double pl = c[d] > 0 ? s->p[cidv(s, L)] : -s->p[cidv(s, c)];
  double pr = c[d] < s->n[d] ? s->p[cidv(s, c)] : -s->p[cidv(s, L)];
  return pr - pl;
}

static void momentum_predictor(orc_state* s) {
  double h = s->h, V = s->V;
  for (int it = 0; it < s->P.mom_sweeps; it++) {
    for (int d = 0; d < s->dim; d++) {
      int fn[3];
      face_dims(s, d, fn);
      for (int k = 0; k < fn[2]; k++)
        for (int j = 0; j < fn[1]; j++)
          for (int i = 0; i < fn[0]; i++) {
            int c[3] = {i, j, k};
            long f = fidv(s, d, c);
            if (face_kind(s, d, c) == F_FIXED) {
              s->unew[d][f] = s->u[d][f];
              continue;
            }
            double hs = face_H(s, d, c);
            s->unew[d][f] = (hs - V * face_dp(s, d, c) / h) / s->aP[d][f];
          }
    }
    for (int d = 0; d < s->dim; d++) {
      double* t = s->u[d];
      s->u[d] = s->unew[d];
      s->unew[d] = t;
    }
  }
}

/* ------------------------------------------------------------------ */
/* 5. pressure equation, Eq. 53: GMG-preconditioned CG                   */
/* ------------------------------------------------------------------ */
static void level_alloc(level_t* L) {
  L->cells = (long)L->n[0] * L->n[1] * L->n[2];
  L->Tx = calloc(L->cells, sizeof(double));
  L->Ty = calloc(L->cells, sizeof(double));
  L->Tz = calloc(L->cells, sizeof(double));
  L->Dd = calloc(L->cells, sizeof(double));
  L->diag = calloc(L->cells, sizeof(double));
  L->x = calloc(L->cells, sizeof(double));
  L->b = calloc(L->cells, sizeof(double));
  L->r = calloc(L->cells, sizeof(double));
}
static void level_free(level_t* L) {
  free(L->Tx);
  free(L->Ty);
  free(L->Tz);
  free(L->Dd);
  free(L->diag);
  free(L->x);
  free(L->b);
  free(L->r);
}

/* hierarchy: every axis longer than 4 cells is halved (rounding up) */
static int build_levels(level_t* lev, const int n[3]) {
  int nlev = 1;
  cpy3(lev[0].n, n);
  lev[0].cz[0] = lev[0].cz[1] = lev[0].cz[2] = 0;
  level_alloc(&lev[0]);
  while (nlev < MAXLEV) {
    level_t* F = &lev[nlev - 1];
    level_t* C = &lev[nlev];
    int changed = 0;
    for (int d = 0; d < 3; d++) {
      if (F->n[d] > 4) {
        C->n[d] = (F->n[d] + 1) / 2;
        C->cz[d] = 1;
        changed = 1;
      } else {
        C->n[d] = F->n[d];
        C->cz[d] = 0;
      }
    }
    if (!changed) break;
    level_alloc(C);
    nlev++;
  }
  return nlev;
}

static const double* lev_T(const level_t* L, int d) { return d == 0 ? L->Tx : (d == 1 ? L->Ty : L->Tz); }

static void level_diag(level_t* L) {
  for (long c = 0; c < L->cells; c++) {
    int q[3];
    coords_of(L->n, c, q);
    double dg = 0.0;
    for (int d = 0; d < 3; d++) {
      const double* T = lev_T(L, d);
      dg += T[c];
      if (q[d] > 0) {
        int m[3];
        cpy3(m, q);
        m[d] -= 1;
        dg += T[cid3(L->n, m)];
      }
    }
    L->diag[c] = dg + L->Dd[c];
  }
}

/* Coarse transmissibilities.  A coarse face link is the sum of the fine links
 * that cross the face (the Galerkin coarse operator of piecewise-constant
 * prolongation with its transpose as restriction), halved when the face's normal
 * axis is coarsened: in a uniform medium the fine links crossing a face sum to
 * k A_face / h, while the 2h link is k A_face / (2 h).  With every axis coarsened
 * the coarse operator is half the Galerkin operator, i.e. the coarse correction
 * is doubled. */
static void coarsen_coeffs(const level_t* F, level_t* C) {
  for (long ci = 0; ci < C->cells; ci++) {
    int Q[3];
    coords_of(C->n, ci, Q);
    for (int d = 0; d < 3; d++) {
      double* Tc = (double*)lev_T(C, d);
      if (Q[d] + 1 >= C->n[d]) {
        Tc[ci] = 0.0;
        continue;
      }
      const double* Tf = lev_T(F, d);
      int lo[3], hi[3];
      for (int a = 0; a < 3; a++) {
        if (a == d) continue;
        lo[a] = C->cz[a] ? 2 * Q[a] : Q[a];
        hi[a] = C->cz[a] ? (2 * Q[a] + 1 < F->n[a] ? 2 * Q[a] + 1 : 2 * Q[a]) : Q[a];
      }
      /* the fine link across the coarse face: from the last fine cell of coarse
       * cell Q to the first of coarse cell Q + 1 */
      lo[d] = hi[d] = C->cz[d] ? 2 * Q[d] + 1 : Q[d];
      double sum = 0.0;
      for (int z = lo[2]; z <= hi[2]; z++)
        for (int y = lo[1]; y <= hi[1]; y++)
          for (int x = lo[0]; x <= hi[0]; x++) {
            int fc[3] = {x, y, z};
            sum += Tf[cid3(F->n, fc)];
          }
      Tc[ci] = C->cz[d] ? 0.5 * sum : sum;
    }
  }
  /* Dirichlet (outlet) diagonal: half the sum over the covered fine cells */
  for (long ci = 0; ci < C->cells; ci++) C->Dd[ci] = 0.0;
  for (long fi = 0; fi < F->cells; fi++) {
    int q[3], Q[3];
    coords_of(F->n, fi, q);
    for (int a = 0; a < 3; a++) Q[a] = C->cz[a] ? q[a] / 2 : q[a];
    C->Dd[cid3(C->n, Q)] += 0.5 * F->Dd[fi];
  }
  level_diag(C);
}

static void apply_A_level(const level_t* L, const double* x, double* y) {
  for (long c = 0; c < L->cells; c++) {
    int q[3];
    coords_of(L->n, c, q);
    double v = L->diag[c] * x[c];
    for (int d = 0; d < 3; d++) {
      const double* T = lev_T(L, d);
      if (q[d] > 0) {
        int m[3];
        cpy3(m, q);
        m[d] -= 1;
        long cm = cid3(L->n, m);
        v -= T[cm] * x[cm];
      }
      if (q[d] + 1 < L->n[d]) {
        int p[3];
        cpy3(p, q);
        p[d] += 1;
        v -= T[c] * x[cid3(L->n, p)];
      }
    }
    y[c] = v;
  }
}

/* one red-black Gauss-Seidel half sweep over the cells of colour col */
static void smooth_color(level_t* L, int col) {
  for (long c = 0; c < L->cells; c++) {
    int q[3];
    coords_of(L->n, c, q);
    if (((q[0] + q[1] + q[2]) & 1) != col) continue;
    double v = L->b[c];
    for (int d = 0; d < 3; d++) {
      const double* T = lev_T(L, d);
      if (q[d] > 0) {
        int m[3];
        cpy3(m, q);
        m[d] -= 1;
        long cm = cid3(L->n, m);
        v += T[cm] * L->x[cm];
      }
      if (q[d] + 1 < L->n[d]) {
        int p[3];
        cpy3(p, q);
        p[d] += 1;
        v += T[c] * L->x[cid3(L->n, p)];
      }
    }
    L->x[c] = v / L->diag[c];
  }
}

/* Exact solve of the coarsest level (at most 4 x 4 x 4 cells): dense matrix of
 * the operator, Cholesky factorisation, forward and back substitution. */
static void coarsest_direct(level_t* L) {
  long n = L->cells;
  double* M = calloc(n * n, sizeof(double));
  for (long c = 0; c < n; c++) {
    int q[3];
    coords_of(L->n, c, q);
    M[c * n + c] = L->diag[c];
    for (int d = 0; d < 3; d++) {
      if (q[d] + 1 < L->n[d]) {
        int p[3];
        cpy3(p, q);
        p[d] += 1;
        long o = cid3(L->n, p);
        M[c * n + o] -= lev_T(L, d)[c];
        M[o * n + c] -= lev_T(L, d)[c];
      }
    }
  }
  /* Cholesky M = G G^T, G lower, stored in M */
  for (long j = 0; j < n; j++) {
    double dj = M[j * n + j];
    for (long k = 0; k < j; k++) dj -= M[j * n + k] * M[j * n + k];
    dj = sqrt(dj);
    M[j * n + j] = dj;
    for (long i = j + 1; i < n; i++) {
      double v = M[i * n + j];
      for (long k = 0; k < j; k++) v -= M[i * n + k] * M[j * n + k];
      M[i * n + j] = v / dj;
    }
  }
  for (long i = 0; i < n; i++) { /* G y = b */
    double v = L->b[i];
    for (long k = 0; k < i; k++) v -= M[i * n + k] * L->x[k];
    L->x[i] = v / M[i * n + i];
  }
  for (long i = n - 1; i >= 0; i--) { /* G^T x = y */
    double v = L->x[i];
    for (long k = i + 1; k < n; k++) v -= M[k * n + i] * L->x[k];
    L->x[i] = v / M[i * n + i];
  }
  free(M);
}

/* symmetric V-cycle from a zero initial guess: (red, black) x nu1 before the
 * coarse correction, (black, red) x nu2 after it; the coarsest level is solved
 * exactly (cs == 0) or by cs forward then cs backward sweep pairs. */
static void vcycle_rec(level_t* lev, int l, int nlev, int nu1, int nu2, int cs) {
  level_t* L = &lev[l];
  memset(L->x, 0, L->cells * sizeof(double));
  if (l == nlev - 1) {
    if (cs == 0) {
      coarsest_direct(L);
      return;
    }
    for (int i = 0; i < cs; i++) {
      smooth_color(L, 0);
      smooth_color(L, 1);
    }
    for (int i = 0; i < cs; i++) {
      smooth_color(L, 1);
      smooth_color(L, 0);
    }
    return;
  }
  for (int i = 0; i < nu1; i++) {
    smooth_color(L, 0);
    smooth_color(L, 1);
  }
  apply_A_level(L, L->x, L->r);
  for (long c = 0; c < L->cells; c++) L->r[c] = L->b[c] - L->r[c];
  level_t* C = &lev[l + 1];
  memset(C->b, 0, C->cells * sizeof(double));
  for (long c = 0; c < L->cells; c++) {
    int q[3], Q[3];
    coords_of(L->n, c, q);
    for (int a = 0; a < 3; a++) Q[a] = C->cz[a] ? q[a] / 2 : q[a];
    C->b[cid3(C->n, Q)] += L->r[c];
  }
  vcycle_rec(lev, l + 1, nlev, nu1, nu2, cs);
  for (long c = 0; c < L->cells; c++) {
    int q[3], Q[3];
    coords_of(L->n, c, q);
    for (int a = 0; a < 3; a++) Q[a] = C->cz[a] ? q[a] / 2 : q[a];
    L->x[c] += C->x[cid3(C->n, Q)];
  }
  for (int i = 0; i < nu2; i++) {
    smooth_color(L, 1);
    smooth_color(L, 0);
  }
}

static double dot(const double* a, const double* b, long n) {
  double s = 0.0;
  for (long i = 0; i < n; i++) s += a[i] * b[i];
  return s;
}

static void hierarchy_setup(level_t* lev, int nlev) {
  level_diag(&lev[0]);
  for (int l = 1; l < nlev; l++) coarsen_coeffs(&lev[l - 1], &lev[l]);
}

static void precond(level_t* lev, int nlev, int nu1, int nu2, int cs, const double* r, double* z) {
  memcpy(lev[0].b, r, lev[0].cells * sizeof(double));
  vcycle_rec(lev, 0, nlev, nu1, nu2, cs);
  memcpy(z, lev[0].x, lev[0].cells * sizeof(double));
}

/* preconditioned CG; x holds the initial guess (warm start) and the result */
static int pcg_solve(level_t* lev, int nlev, int nu1, int nu2, int cs, const double* b, double* x,
                     double tol, int max_it, double* r, double* z, double* dv, double* q,
                     double* resid_out) {
  long n = lev[0].cells;
  double bn = sqrt(dot(b, b, n));
  if (bn == 0.0) {
    memset(x, 0, n * sizeof(double));
    *resid_out = 0.0;
    return 0;
  }
  apply_A_level(&lev[0], x, r);
  for (long i = 0; i < n; i++) r[i] = b[i] - r[i];
  double rn = sqrt(dot(r, r, n));
  if (rn <= tol * bn) {
    *resid_out = rn / bn;
    return 0;
  }
  precond(lev, nlev, nu1, nu2, cs, r, z);
  memcpy(dv, z, n * sizeof(double));
  double rz = dot(r, z, n);
  int it = 0;
  while (it < max_it) {
    it++;
    apply_A_level(&lev[0], dv, q);
    double al = rz / dot(dv, q, n);
    for (long i = 0; i < n; i++) {
      x[i] += al * dv[i];
      r[i] -= al * q[i];
    }
    rn = sqrt(dot(r, r, n));
    if (rn <= tol * bn) break;
    precond(lev, nlev, nu1, nu2, cs, r, z);
    double rz2 = dot(r, z, n);
    double be = rz2 / rz;
    rz = rz2;
    for (long i = 0; i < n; i++) dv[i] = z[i] + be * dv[i];
  }
  *resid_out = rn / bn;
  return it;
}

static void pressure_assemble(orc_state* s) {
  double A = s->A;
  level_t* L0 = &s->lev[0];
  for (int d = 0; d < 3; d++) {
    double* T = (double*)lev_T(L0, d);
    memset(T, 0, s->cells * sizeof(double));
  }
  memset(L0->Dd, 0, s->cells * sizeof(double));
  for (long c = 0; c < s->cells; c++) {
    int q[3];
    coords_of(s->n, c, q);
    double div = 0.0;
    for (int d = 0; d < s->dim; d++) {
      int hi[3];
      cpy3(hi, q);
      hi[d] += 1;
      long flo = fidv(s, d, q), fhi = fidv(s, d, hi);
      double* T = (double*)lev_T(L0, d);
      if (q[d] + 1 < s->n[d]) T[c] = A * A / s->aP[d][fhi]; /* T_f = A^2 / a_P,f */
      if (q[d] == 0 && s->P.bc[2 * d] == ORC_OUTLET) L0->Dd[c] += 2.0 * A * A / s->aP[d][flo];
      if (q[d] + 1 == s->n[d] && s->P.bc[2 * d + 1] == ORC_OUTLET)
        L0->Dd[c] += 2.0 * A * A / s->aP[d][fhi];
      /* HbyA on unknown faces, the fixed value on wall / inlet faces */
      double ulo = face_kind(s, d, q) == F_FIXED ? s->u[d][flo] : s->hbya[d][flo];
      double uhi = face_kind(s, d, hi) == F_FIXED ? s->u[d][fhi] : s->hbya[d][fhi];
      div += A * uhi - A * ulo;
    }
    L0->b[c] = -div;
  }
}

static void piso_corrector(orc_state* s, int corr) {
  double A = s->A;
  /* HbyA = H(u)/a_P (Eq. 51 without the pressure gradient) */
  for (int d = 0; d < s->dim; d++) {
    int fn[3];
    face_dims(s, d, fn);
    for (int k = 0; k < fn[2]; k++)
      for (int j = 0; j < fn[1]; j++)
        for (int i = 0; i < fn[0]; i++) {
          int c[3] = {i, j, k};
          long f = fidv(s, d, c);
          s->hbya[d][f] = face_kind(s, d, c) == F_FIXED ? 0.0 : face_H(s, d, c) / s->aP[d][f];
        }
  }
  pressure_assemble(s);
  hierarchy_setup(s->lev, s->nlev);
  double res;
  /* the level-0 RHS array is reused by the V-cycle; solve from a copy */
  double* bb = malloc(s->cells * sizeof(double));
  memcpy(bb, s->lev[0].b, s->cells * sizeof(double));
  int it = pcg_solve(s->lev, s->nlev, s->P.mg_nu1, s->P.mg_nu2, s->P.mg_coarse_sweeps, bb, s->p,
                     s->P.p_tol, s->P.max_cg, s->cg_r, s->cg_z, s->cg_d, s->cg_q, &res);
  memcpy(s->lev[0].b, bb, s->cells * sizeof(double));
  free(bb);
  if (corr < 8) {
    s->st.cg_iters[corr] = it;
    s->st.cg_resid[corr] = res;
  }
  s->st.cg_iters_total += it;
  if (!(res <= s->P.p_tol)) s->st.not_converged++;
  /* corrected velocity, Eq. 51 */
  for (int d = 0; d < s->dim; d++) {
    int fn[3];
    face_dims(s, d, fn);
    for (int k = 0; k < fn[2]; k++)
      for (int j = 0; j < fn[1]; j++)
        for (int i = 0; i < fn[0]; i++) {
          int c[3] = {i, j, k};
          long f = fidv(s, d, c);
          if (face_kind(s, d, c) == F_FIXED) continue;
          s->u[d][f] = s->hbya[d][f] - (A / s->aP[d][f]) * face_dp(s, d, c);
        }
  }
}

/* ------------------------------------------------------------------ */
/* public API                                                           */
/* ------------------------------------------------------------------ */
static void set_boundary_velocities(orc_state* s) {
  for (int d = 0; d < s->dim; d++) {
    int fn[3];
    face_dims(s, d, fn);
    for (int k = 0; k < fn[2]; k++)
      for (int j = 0; j < fn[1]; j++)
        for (int i = 0; i < fn[0]; i++) {
          int c[3] = {i, j, k};
          if (face_kind(s, d, c) != F_FIXED) continue;
          int side = 2 * d + (c[d] == 0 ? 0 : 1);
          double v = 0.0;
          if (s->P.bc[side] == ORC_INLET) v = (side & 1) ? -s->P.inlet_u : s->P.inlet_u;
          s->u[d][fidv(s, d, c)] = v;
        }
  }
}

static void update_stats(orc_state* s) {
  double mass = 0.0, amin = INFINITY, amax = -INFINITY;
  for (long c = 0; c < s->cells; c++) {
    mass += s->phi[c] * s->alpha[c] * s->V;
    amin = fmin(amin, s->alpha[c]);
    amax = fmax(amax, s->alpha[c]);
  }
  s->st.mass = mass;
  s->st.alpha_min = amin;
  s->st.alpha_max = amax;
}

orc_state* orc_create(const orc_params* prm, const double* porosity, const double* permeability) {
  if (prm->nx < 1 || prm->ny < 1 || prm->nz < 1 || !(prm->h > 0)) return NULL;
  int has_outlet = 0;
  for (int sd = 0; sd < 6; sd++) has_outlet |= prm->bc[sd] == ORC_OUTLET;
  if (!has_outlet) return NULL;
  orc_state* s = calloc(1, sizeof(orc_state));
  s->P = *prm;
  s->n[0] = prm->nx;
  s->n[1] = prm->ny;
  s->n[2] = prm->nz;
  s->dim = prm->nz == 1 ? 2 : 3;
  s->cells = (long)prm->nx * prm->ny * prm->nz;
  s->h = prm->h;
  s->A = prm->h * prm->h;
  s->V = prm->h * prm->h * prm->h;
  s->dt = prm->dt;
  long nc = s->cells;
  for (int d = 0; d < 3; d++) {
    int fn[3];
    face_dims(s, d, fn);
    s->nf[d] = (long)fn[0] * fn[1] * fn[2];
  }
#define CA(n) calloc((n), sizeof(double))
  s->phi = CA(nc);
  s->k0 = CA(nc);
  s->alpha = CA(nc);
  s->p = CA(nc);
  s->is_free = calloc(nc, 1);
  s->has_nw = calloc(nc, 1);
  s->Ml = CA(nc);
  s->Mg = CA(nc);
  s->pc = CA(nc);
  s->cf = CA(nc);
  s->rho = CA(nc);
  s->mu = CA(nc);
  s->drag = CA(nc);
  s->kappa = CA(nc);
  s->aL = CA(nc);
  s->Rp = CA(nc);
  s->Rm = CA(nc);
  s->cg_r = CA(nc);
  s->cg_z = CA(nc);
  s->cg_d = CA(nc);
  s->cg_q = CA(nc);
  for (int d = 0; d < 3; d++) {
    long nf = s->nf[d];
    s->nw[d] = CA(nc);
    s->m[d] = CA(nc);
    s->u[d] = CA(nf);
    s->FLO[d] = CA(nf);
    s->AF[d] = CA(nf);
    s->aP[d] = CA(nf);
    s->anb[d] = CA(nf * 6);
    s->rhs0[d] = CA(nf);
    s->unew[d] = CA(nf);
    s->hbya[d] = CA(nf);
    s->B[d] = CA(nf);
  }
#undef CA
  for (long c = 0; c < nc; c++) {
    s->phi[c] = porosity[c];
    s->k0[c] = permeability[c];
    s->is_free[c] = porosity[c] == 1.0;
  }
  /* wall normal for the contact angle (Eq. 40): free cells with a porous face
   * neighbour, n_wall = -grad(phi)/|grad(phi)| pointing into the porous side */
  for (long c = 0; c < nc; c++) {
    if (!s->is_free[c]) continue;
    int q[3];
    coords_of(s->n, c, q);
    int touch = 0;
    for (int d = 0; d < s->dim; d++)
      for (int sg = -1; sg <= 1; sg += 2) {
        int nb[3];
        cpy3(nb, q);
        nb[d] += sg;
        if (nb[d] < 0 || nb[d] >= s->n[d]) continue;
        if (!s->is_free[cidv(s, nb)]) touch = 1;
      }
    if (!touch) continue;
    double g[3];
    grad_cell(s, s->phi, q, g);
    double mag = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    if (mag > 0.0) {
      s->has_nw[c] = 1;
      for (int e = 0; e < 3; e++) s->nw[e][c] = -g[e] / mag;
    }
  }
  s->nlev = build_levels(s->lev, s->n);
  set_boundary_velocities(s);
  return s;
}

int orc_set_fields(orc_state* s, const double* alpha, const double* ux, const double* uy,
                   const double* uz, const double* p) {
  const double* src[3] = {ux, uy, uz};
  for (long c = 0; c < s->cells; c++) {
    if (!(alpha[c] >= -1e-9 && alpha[c] <= 1.0 + 1e-9)) return -1; /* round-off of a previous step */
  }
  memcpy(s->alpha, alpha, s->cells * sizeof(double));
  memcpy(s->p, p, s->cells * sizeof(double));
  for (int d = 0; d < s->dim; d++) memcpy(s->u[d], src[d], s->nf[d] * sizeof(double));
  set_boundary_velocities(s);
  update_props(s);
  normals_curvature(s);
  memset(&s->st, 0, sizeof(s->st));
  s->st.dt = s->dt;
  update_stats(s);
  return 0;
}

int orc_step(orc_state* s, int nsteps) {
  for (int it = 0; it < nsteps; it++) {
    double dt = s->dt;
    /* 1. saturation */
    alpha_step(s, dt);
    /* 3. properties at alpha^{k+1} */
    update_props(s);
    normals_curvature(s);
    /* 4. momentum predictor */
    momentum_assemble(s, dt);
    momentum_predictor(s);
    /* 5. PISO */
    for (int c = 0; c < s->P.n_corr; c++) piso_corrector(s, c);
    /* 6. time step */
    s->time += dt;
    s->st.steps++;
    if (s->P.cfl > 0.0) {
      double umax = 0.0;
      for (int d = 0; d < s->dim; d++) {
        int fn[3];
        face_dims(s, d, fn);
        for (int k = 0; k < fn[2]; k++)
          for (int j = 0; j < fn[1]; j++)
            for (int i = 0; i < fn[0]; i++) {
              int c[3] = {i, j, k};
              int L[3];
              cpy3(L, c);
              L[d] -= 1;
              double phif = 0.5 * (cval(s, s->phi, L) + cval(s, s->phi, c));
              umax = fmax(umax, fabs(s->u[d][fidv(s, d, c)]) / phif);
            }
      }
      double dtn = umax > 0.0 ? s->P.cfl * s->h / umax : s->P.dt_max;
      dtn = fmin(dtn, 1.2 * dt);
      dtn = fmin(dtn, s->P.dt_max);
      s->dt = dtn;
    }
    s->st.time = s->time;
    s->st.dt = s->dt;
    update_stats(s);
    if (!isfinite(s->st.mass)) return -4;
    for (long c = 0; c < s->cells; c++)
      if (!isfinite(s->p[c])) return -4;
  }
  return 0;
}

int orc_get_fields(const orc_state* s, double* alpha, double* ux, double* uy, double* uz, double* p) {
  double* dst[3] = {ux, uy, uz};
  if (alpha) memcpy(alpha, s->alpha, s->cells * sizeof(double));
  if (p) memcpy(p, s->p, s->cells * sizeof(double));
  for (int d = 0; d < s->dim; d++)
    if (dst[d]) memcpy(dst[d], s->u[d], s->nf[d] * sizeof(double));
  return 0;
}

int orc_get_stats(const orc_state* s, orc_stats* out) {
  *out = s->st;
  return 0;
}

long orc_get_array(const orc_state* s, const char* name, double* out) {
  struct {
    const char* nm;
    const double* a;
    long n;
  } tab[] = {
      {"rho", s->rho, s->cells},        {"mu", s->mu, s->cells},
      {"drag", s->drag, s->cells},      {"pc", s->pc, s->cells},           {"cf", s->cf, s->cells},
      {"Ml", s->Ml, s->cells},          {"Mg", s->Mg, s->cells},           {"kappa", s->kappa, s->cells},
      {"mx", s->m[0], s->cells},        {"my", s->m[1], s->cells},         {"mz", s->m[2], s->cells},
      {"Tx", s->lev[0].Tx, s->cells},   {"Ty", s->lev[0].Ty, s->cells},    {"Tz", s->lev[0].Tz, s->cells},
      {"Dd", s->lev[0].Dd, s->cells},   {"b", s->lev[0].b, s->cells},      {"aL", s->aL, s->cells},
      {"Rp", s->Rp, s->cells},          {"Rm", s->Rm, s->cells},           {"aPx", s->aP[0], s->nf[0]},
      {"aPy", s->aP[1], s->nf[1]},      {"aPz", s->aP[2], s->nf[2]},       {"rhs0x", s->rhs0[0], s->nf[0]},
      {"rhs0y", s->rhs0[1], s->nf[1]},  {"rhs0z", s->rhs0[2], s->nf[2]},   {"Bx", s->B[0], s->nf[0]},
      {"By", s->B[1], s->nf[1]},        {"Bz", s->B[2], s->nf[2]},         {"hbyax", s->hbya[0], s->nf[0]},
      {"hbyay", s->hbya[1], s->nf[1]},  {"hbyaz", s->hbya[2], s->nf[2]},   {"FLOx", s->FLO[0], s->nf[0]},
      {"FLOy", s->FLO[1], s->nf[1]},    {"FLOz", s->FLO[2], s->nf[2]},     {"AFx", s->AF[0], s->nf[0]},
      {"AFy", s->AF[1], s->nf[1]},      {"AFz", s->AF[2], s->nf[2]},       {"nwx", s->nw[0], s->cells},
      {"nwy", s->nw[1], s->cells},      {"nwz", s->nw[2], s->cells},
  };
  for (size_t i = 0; i < sizeof(tab) / sizeof(tab[0]); i++) {
    if (strcmp(tab[i].nm, name) == 0) {
      if (out) memcpy(out, tab[i].a, tab[i].n * sizeof(double));
      return tab[i].n;
    }
  }
  if (strcmp(name, "anbx") == 0 || strcmp(name, "anby") == 0 || strcmp(name, "anbz") == 0) {
    int d = name[3] - 'x';
    if (out) memcpy(out, s->anb[d], s->nf[d] * 6 * sizeof(double));
    return s->nf[d] * 6;
  }
  return -1;
}

void orc_destroy(orc_state* s) {
  if (!s) return;
  free(s->phi);
  free(s->k0);
  free(s->alpha);
  free(s->p);
  free(s->is_free);
  free(s->has_nw);
  free(s->Ml);
  free(s->Mg);
  free(s->pc);
  free(s->cf);
  free(s->rho);
  free(s->mu);
  free(s->drag);
  free(s->kappa);
  free(s->aL);
  free(s->Rp);
  free(s->Rm);
  free(s->cg_r);
  free(s->cg_z);
  free(s->cg_d);
  free(s->cg_q);
  for (int d = 0; d < 3; d++) {
    free(s->nw[d]);
    free(s->m[d]);
    free(s->u[d]);
    free(s->FLO[d]);
    free(s->AF[d]);
    free(s->aP[d]);
    free(s->anb[d]);
    free(s->rhs0[d]);
    free(s->unew[d]);
    free(s->hbya[d]);
    free(s->B[d]);
  }
  for (int l = 0; l < s->nlev; l++) level_free(&s->lev[l]);
  free(s);
}

/* ---------------- standalone solver entry points (tests) ---------------- */
static int standalone_levels(level_t* lev, int nx, int ny, int nz, const double* Tx,
                             const double* Ty, const double* Tz, const double* Dd) {
  int n[3] = {nx, ny, nz};
  int nlev = build_levels(lev, n);
  long nc = lev[0].cells;
  memcpy(lev[0].Tx, Tx, nc * sizeof(double));
  memcpy(lev[0].Ty, Ty, nc * sizeof(double));
  memcpy(lev[0].Tz, Tz, nc * sizeof(double));
  memcpy(lev[0].Dd, Dd, nc * sizeof(double));
  hierarchy_setup(lev, nlev);
  return nlev;
}

void orc_apply_A(int nx, int ny, int nz, const double* Tx, const double* Ty, const double* Tz,
                 const double* Dd, const double* x, double* y) {
  level_t lev[MAXLEV];
  int nlev = standalone_levels(lev, nx, ny, nz, Tx, Ty, Tz, Dd);
  apply_A_level(&lev[0], x, y);
  for (int l = 0; l < nlev; l++) level_free(&lev[l]);
}

int orc_vcycle(int nx, int ny, int nz, const double* Tx, const double* Ty, const double* Tz,
               const double* Dd, int nu1, int nu2, int cs, const double* r, double* z) {
  level_t lev[MAXLEV];
  int nlev = standalone_levels(lev, nx, ny, nz, Tx, Ty, Tz, Dd);
  precond(lev, nlev, nu1, nu2, cs, r, z);
  for (int l = 0; l < nlev; l++) level_free(&lev[l]);
  return nlev;
}

int orc_pcg(int nx, int ny, int nz, const double* Tx, const double* Ty, const double* Tz,
            const double* Dd, int nu1, int nu2, int cs, const double* b, double* x, double tol,
            int max_it, double* resid_out) {
  level_t lev[MAXLEV];
  int nlev = standalone_levels(lev, nx, ny, nz, Tx, Ty, Tz, Dd);
  long nc = lev[0].cells;
  double* r = calloc(nc, sizeof(double));
  double* z = calloc(nc, sizeof(double));
  double* dv = calloc(nc, sizeof(double));
  double* q = calloc(nc, sizeof(double));
  int it = pcg_solve(lev, nlev, nu1, nu2, cs, b, x, tol, max_it, r, z, dv, q, resid_out);
  free(r);
  free(z);
  free(dv);
  free(q);
  for (int l = 0; l < nlev; l++) level_free(&lev[l]);
  return it;
}
