/*
 * oracle.h -- plain, slow FP64 CPU oracle of one pressure-velocity time step
 * of the two-phase micro-continuum Darcy-Brinkman-Stokes VOF model
 * (Carrillo, Bourg & Soulaine, arXiv 2003.08374).
 *
 * TEST INFRASTRUCTURE ONLY.  This library exists to check the CUDA path; it is
 * never a runtime fallback.  Only the tests, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load it.  It shares no code,
 * header, table or helper with the CUDA library.
 *
 * Grid: uniform spacing h, cell-centred alpha, p, porosity, permeability;
 * staggered (MAC) face velocities.  Arrays are x-fastest.
 *   cells  : nx*ny*nz,            c = i + nx*(j + ny*k)
 *   x faces: (nx+1)*ny*nz,        f = i + (nx+1)*(j + ny*k), i in [0,nx]
 *   y faces: nx*(ny+1)*nz,        f = i + nx*(j + (ny+1)*k)
 *   z faces: nx*ny*(nz+1)         (unused when nz == 1: two-dimensional run)
 */
#ifndef MDBS_ORACLE_H
#define MDBS_ORACLE_H
#ifdef __cplusplus
extern "C" {
#endif

/* side order: x-, x+, y-, y+, z-, z+ ; side types */
#define ORC_WALL 0
#define ORC_INLET 1
#define ORC_OUTLET 2

typedef struct {
  int nx, ny, nz;
  double h;
  /* fluids (l = wetting liquid, g = non-wetting gas); Table 1 */
  double rho_l, mu_l, rho_g, mu_g, sigma;
  double g[3];
  /* closures, Appendix A: model 0 Brooks-Corey, 1 Van Genuchten */
  int kr_model, pc_model;
  double kr_m, a_l_irr, a_g_irr;
  double pc0, pc_beta, pc_m, a_pc_irr, a_pc_max, pc_eps;
  int porous_density; /* 0: rho* of Eq. 45 in porous cells; 1: Appendix B */
  double theta_deg; /* contact angle at the free/porous interface, Eq. 40 */
  /* time stepping and solver */
  double dt, cfl, dt_max, c_alpha, p_tol;
  int n_corr, mom_sweeps, max_cg;
  int mg_nu1, mg_nu2, mg_coarse_sweeps; /* 0: exact solve of the coarsest level */
  int bc[6];
  double inlet_u, inlet_alpha;
} orc_params;

typedef struct orc_state orc_state;

typedef struct {
  long steps;
  double time, dt;
  int cg_iters[8];     /* per corrector of the last step */
  double cg_resid[8];  /* final relative residual per corrector */
  long cg_iters_total;
  int not_converged;   /* solves that hit max_cg */
  double mass;         /* sum phi*alpha*V */
  double boundary_in;  /* cumulative (time-integrated) boundary alpha volume inflow */
  double alpha_min, alpha_max;
} orc_stats;

orc_state* orc_create(const orc_params* prm, const double* porosity, const double* permeability);
int orc_set_fields(orc_state* s, const double* alpha, const double* ux, const double* uy,
                   const double* uz, const double* p);
int orc_step(orc_state* s, int n);
int orc_get_fields(const orc_state* s, double* alpha, double* ux, double* uy, double* uz, double* p);
int orc_get_stats(const orc_state* s, orc_stats* out);
/* copies an internal array by name ("rho", "mu", "pc", "kappa", "Tx", "b", ...);
 * returns the element count, or -1 for an unknown name */
long orc_get_array(const orc_state* s, const char* name, double* out);
void orc_destroy(orc_state* s);

/* Closures of Appendix A at one saturation: out = {krl, krg, Ml, Mg, drag, rho, pc, cf}
 * for a porous cell of permeability k0 (Eqs. 37, 38, 45). */
void orc_closures(const orc_params* prm, double alpha, double k0, double* out8);

/* Standalone pressure operator, V-cycle and PCG on a cell grid with per-cell
 * high-face coefficients Tx, Ty, Tz and Dirichlet diagonal Dd (see oracle.c). */
void orc_apply_A(int nx, int ny, int nz, const double* Tx, const double* Ty, const double* Tz,
                 const double* Dd, const double* x, double* y);
int orc_vcycle(int nx, int ny, int nz, const double* Tx, const double* Ty, const double* Tz,
               const double* Dd, int nu1, int nu2, int coarse_sweeps, const double* r, double* z);
int orc_pcg(int nx, int ny, int nz, const double* Tx, const double* Ty, const double* Tz,
            const double* Dd, int nu1, int nu2, int coarse_sweeps, const double* b, double* x,
            double tol, int max_it, double* resid_out);

#ifdef __cplusplus
}
#endif
#endif
