"""Seeded synthetic inputs for the micro-continuum DBS-VOF step.

This module holds no arithmetic of the method: only geometry, random fields
and initial states.  It serves both the CUDA path and the oracle, which read
identical arrays.  Recipes:

* ``fracture_2d``  -- a solid-free fracture, 8 cells wide, crossing a porous
  matrix (porosity 0.5, Kozeny-Carman k = 1e-12 m^2) on a 2-D grid, water
  displacing air, inlet on x-, outlet on x+.  Stand-in for the paper's
  fractured microporous matrix application (section 5.2).
* ``grf_3d``       -- a 3-D porous block whose ln k is a Gaussian random field
  (FFT-filtered white noise, Gaussian covariance, correlation length in cells,
  sigma_lnk), porosity tied monotonically to k, one planar solid-free fracture
  normal to y, water injected into oil, gravity on.
* ``wave_tank``    -- water/air tank with a porous barrier block on the floor
  and a solitary-wave free surface (stand-in for section 5.1).
* ``darcy_domain`` -- porous-only domain with a random porosity field mapped
  into [0.1, 0.9] and uniform initial saturation (batched / served domains).
* ``buckley_leverett`` -- the Darcy-scale 1-D column of sections 4.1.1-4.1.2
  (water injected into air or oil, optional gravity along the flow).
* ``capillary_column`` -- the gravity-capillarity column of section 4.1.3
  (step-wise initial saturation relaxing to capillary-gravity equilibrium).
* ``capillary_rise`` -- water rising between porous walls (section 4.2.2).

Every array is x-fastest: cell c = i + nx*(j + ny*k).  Face arrays hold
(nx+1)*ny*nz x-faces, nx*(ny+1)*nz y-faces and nx*ny*(nz+1) z-faces; a 2-D
case (nz == 1) has no z-faces.
"""
from __future__ import annotations

import dataclasses
import math
from dataclasses import dataclass, field

import numpy as np

WALL, INLET, OUTLET = 0, 1, 2
BROOKS_COREY, VAN_GENUCHTEN = 0, 1
RHO_MOBILITY, RHO_SATURATION = 0, 1  # porous-cell density: Eq. 45 rho*, or Appendix B
FP64, MIXED, MIXED_BF16 = 0, 1, 2


@dataclass
class Case:
    name: str
    nx: int
    ny: int
    nz: int
    h: float
    # fluids: l = wetting liquid, g = non-wetting phase (Table 1 values by default)
    rho_l: float = 1000.0
    mu_l: float = 1e-3
    rho_g: float = 1.0
    mu_g: float = 1.8e-5
    sigma: float = 0.07
    g: tuple = (0.0, 0.0, 0.0)
    # closures (Appendix A, Table 2)
    kr_model: int = BROOKS_COREY
    pc_model: int = BROOKS_COREY
    kr_m: float = 2.0
    a_l_irr: float = 0.0
    a_g_irr: float = 0.0
    pc0: float = 100.0
    pc_beta: float = 0.5
    pc_m: float = 0.5
    a_pc_irr: float = 0.0
    a_pc_max: float = 1.0
    pc_eps: float = 1e-3
    porous_density: int = RHO_MOBILITY
    theta_deg: float = 45.0
    # time stepping / solver options
    dt: float = 1e-6
    cfl: float = 0.0
    dt_max: float = 1e-6
    c_alpha: float = 1.0
    p_tol: float = 1e-8
    n_corr: int = 2
    mom_sweeps: int = 4
    max_cg: int = 200
    mg_nu1: int = 2
    mg_nu2: int = 2
    mg_coarse_sweeps: int = 0  # 0: exact solve of the coarsest level
    bc: tuple = (INLET, OUTLET, WALL, WALL, WALL, WALL)
    inlet_u: float = 1e-3
    inlet_alpha: float = 1.0
    precision: int = FP64
    steps: int = 100
    # fields
    porosity: np.ndarray = field(default=None, repr=False)
    permeability: np.ndarray = field(default=None, repr=False)
    alpha: np.ndarray = field(default=None, repr=False)
    ux: np.ndarray = field(default=None, repr=False)
    uy: np.ndarray = field(default=None, repr=False)
    uz: np.ndarray = field(default=None, repr=False)
    p: np.ndarray = field(default=None, repr=False)

    @property
    def cells(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def dim(self) -> int:
        return 2 if self.nz == 1 else 3

    def replace(self, **kw) -> "Case":
        return dataclasses.replace(self, **kw)


def kozeny_carman(phi, phi_ref=0.5, k_ref=1e-12):
    """Input recipe (not part of the paper's method): k(phi) anchored at (phi_ref, k_ref)."""
    phi = np.asarray(phi, dtype=np.float64)
    return k_ref * phi ** 3 / (1.0 - phi) ** 2 * (1.0 - phi_ref) ** 2 / phi_ref ** 3


def gaussian_random_field(shape, corr_len, rng):
    """Zero-mean unit-variance field: white noise filtered by a Gaussian kernel
    of standard deviation corr_len / sqrt(2) cells, in Fourier space."""
    noise = rng.standard_normal(shape)
    freqs = np.meshgrid(*[np.fft.fftfreq(n) for n in shape], indexing="ij")
    k2 = sum(f ** 2 for f in freqs)
    sig = corr_len / math.sqrt(2.0)
    filt = np.exp(-2.0 * (math.pi ** 2) * (sig ** 2) * k2)
    fld = np.real(np.fft.ifftn(np.fft.fftn(noise) * filt))
    fld -= fld.mean()
    sd = fld.std()
    return fld / sd if sd > 0 else fld


def _std_normal_cdf(x):
    from scipy.special import ndtr
    return ndtr(x)


def _zero_fields(c: Case):
    nx, ny, nz = c.nx, c.ny, c.nz
    c.ux = np.zeros((nx + 1) * ny * nz)
    c.uy = np.zeros(nx * (ny + 1) * nz)
    c.uz = np.zeros(nx * ny * (nz + 1)) if nz > 1 else np.zeros(0)
    c.p = np.zeros(nx * ny * nz)


def _plug_flow(c: Case, u):
    """Uniform x-velocity on every x-face: divergence free for any porosity."""
    c.ux[:] = u


def to_xfast(a_zyx):
    """(nz, ny, nx) array -> flat x-fastest vector."""
    return np.ascontiguousarray(a_zyx, dtype=np.float64).ravel()


def fracture_2d(nx=64, ny=64, frac_lo=None, frac_w=8, inlet_cols=4, steps=100, **kw) -> Case:
    """2-D fracture across a porous matrix; water (1000, 1e-3) displaces air (1, 1.8e-5)."""
    c = Case(name="fracture_2d_%dx%d" % (nx, ny), nx=nx, ny=ny, nz=1, h=1e-5, steps=steps)
    c = c.replace(**kw)
    if frac_lo is None:
        frac_lo = ny // 2 - frac_w // 2
    phi = np.full((1, ny, nx), 0.5)
    phi[:, frac_lo:frac_lo + frac_w, :] = 1.0
    k = np.where(phi < 1.0, kozeny_carman(np.minimum(phi, 0.5)), 0.0)
    alpha = np.zeros((1, ny, nx))
    alpha[:, :, :inlet_cols] = 1.0
    c.porosity, c.permeability, c.alpha = to_xfast(phi), to_xfast(k), to_xfast(alpha)
    _zero_fields(c)
    _plug_flow(c, c.inlet_u)
    return c


def grf_3d(n=128, seed=2, corr_len=8.0, sigma_lnk=1.0, k_mean=1e-13, frac_w=6, inlet_cols=4,
           steps=1000, shape=None, **kw) -> Case:
    """3-D porous block with log-normal permeability, one fracture, water into oil, gravity -z."""
    nx, ny, nz = shape if shape is not None else (n, n, n)
    c = Case(name="grf_3d_%dx%dx%d" % (nx, ny, nz), nx=nx, ny=ny, nz=nz, h=1e-5,
             rho_l=1000.0, mu_l=1e-3, rho_g=800.0, mu_g=1e-2, g=(0.0, 0.0, -9.81), steps=steps)
    c = c.replace(**kw)
    rng = np.random.default_rng(seed)
    z = gaussian_random_field((nz, ny, nx), corr_len, rng)
    mu_lnk = math.log(k_mean) - 0.5 * sigma_lnk ** 2
    lnk = mu_lnk + sigma_lnk * z
    phi = 0.2 + 0.4 * _std_normal_cdf(z)
    k = np.exp(lnk)
    lo = ny // 2 - frac_w // 2
    phi[:, lo:lo + frac_w, :] = 1.0
    k[:, lo:lo + frac_w, :] = 0.0
    alpha = np.zeros((nz, ny, nx))
    alpha[:, :, :inlet_cols] = 1.0
    c.porosity, c.permeability, c.alpha = to_xfast(phi), to_xfast(k), to_xfast(alpha)
    _zero_fields(c)
    _plug_flow(c, c.inlet_u)
    return c


def wave_tank(nx=512, ny=128, nz=256, h=5e-3, depth=80, amp_frac=0.2, x0=128,
              barrier=(320, 384, 96), steps=2000, **kw) -> Case:
    """Water/air tank, porous barrier on the floor, solitary-wave free surface, walls + open top."""
    c = Case(name="wave_tank_%dx%dx%d" % (nx, ny, nz), nx=nx, ny=ny, nz=nz, h=h,
             rho_l=1000.0, mu_l=1e-3, rho_g=1.0, mu_g=1.8e-5, g=(0.0, 0.0, -9.81),
             kr_model=VAN_GENUCHTEN, pc_model=VAN_GENUCHTEN, kr_m=0.8, pc_m=0.8, pc0=1000.0,
             theta_deg=90.0, cfl=0.5, dt=1e-4, dt_max=2e-3,
             bc=(WALL, WALL, WALL, WALL, WALL, OUTLET), inlet_u=0.0, precision=MIXED_BF16,
             steps=steps)
    c = c.replace(**kw)
    xb0, xb1, hb = barrier
    phi = np.ones((nz, ny, nx))
    phi[:hb, :, xb0:xb1] = 0.5
    k = np.where(phi < 1.0, 1e-9, 0.0)
    A = amp_frac * depth
    xc = np.arange(nx) + 0.5
    eta = A / np.cosh(math.sqrt(3.0 * A / (4.0 * depth ** 3)) * (xc - x0)) ** 2
    surf = depth + eta  # in cells
    zlo = np.arange(nz)[:, None]
    frac = np.clip(surf[None, :] - zlo, 0.0, 1.0)  # (nz, nx)
    alpha = np.broadcast_to(frac[:, None, :], (nz, ny, nx))
    c.porosity, c.permeability, c.alpha = to_xfast(phi), to_xfast(k), to_xfast(alpha)
    _zero_fields(c)
    return c


def darcy_domain(shape, seed, corr_len=4.0, sat=None, inlet_u=1e-4, **kw) -> Case:
    """Porous-only domain: porosity GRF mapped linearly into [0.1, 0.9], Kozeny-Carman k,
    uniform initial saturation (drawn from U(0.1, 0.9) unless given)."""
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    c = Case(name="darcy_%dx%dx%d_s%d" % (nx, ny, nz, seed), nx=nx, ny=ny, nz=nz, h=1e-5,
             inlet_u=inlet_u)
    c = c.replace(**kw)
    z = gaussian_random_field((nz, ny, nx), corr_len, rng)
    lo, hi = z.min(), z.max()
    phi = 0.1 + 0.8 * (z - lo) / (hi - lo) if hi > lo else np.full(z.shape, 0.5)
    k = kozeny_carman(phi)
    s0 = float(rng.uniform(0.1, 0.9)) if sat is None else float(sat)
    c.porosity, c.permeability = to_xfast(phi), to_xfast(k)
    c.alpha = np.full(nx * ny * nz, s0)
    _zero_fields(c)
    _plug_flow(c, c.inlet_u)
    return c


DISPLACED = {"air": (1.0, 1.76e-5), "oil": (800.0, 0.1)}  # Table 1: (density, viscosity)


def buckley_leverett(nx=2000, length=4.0, displaced="air", kr_model=BROOKS_COREY, kr_m=None,
                     gravity=False, phi=0.5, k0=1e-11, u=1e-5, cfl=None, **kw) -> Case:
    """Darcy-scale 1-D column of section 4.1.1 (4 m, 2000 cells, porosity 0.5, k0 = 1e-11 m^2):
    water (1000, 1e-3) injected at u = 1e-5 m/s through x- into a column saturated with air or
    oil (Table 1), outlet at p = 0 on x+, no capillary pressure.  Relative permeability by
    Brooks-Corey (m = 3) or Van Genuchten (m = 0.5), Table 2.  ``gravity`` adds g = 9.81 m/s^2
    along the injection direction (section 4.1.2).  The time step follows the CFL number on
    the face velocity; the default keeps the saturation Courant number below about 0.3 for
    these fluids (the fractional-flow wave speeds reach about 3 u / phi)."""
    rho_g, mu_g = DISPLACED[displaced]
    if kr_m is None:
        kr_m = 3.0 if kr_model == BROOKS_COREY else 0.5
    if cfl is None:
        cfl = 0.02 if gravity else 0.05
    h = length / nx
    name = "buckley_leverett_%s_%s%s_%d" % (displaced, "bc" if kr_model == BROOKS_COREY else "vg",
                                            "_gravity" if gravity else "", nx)
    c = Case(name=name, nx=nx, ny=1, nz=1, h=h, rho_l=1000.0, mu_l=1e-3, rho_g=rho_g, mu_g=mu_g,
             sigma=0.0, pc0=0.0, kr_model=kr_model, kr_m=kr_m, g=(9.81 if gravity else 0.0, 0.0, 0.0),
             cfl=cfl, dt=cfl * h / u, dt_max=1e9, inlet_u=u, inlet_alpha=1.0, p_tol=1e-12, max_cg=300)
    c = c.replace(**kw)
    c.porosity = np.full(nx, float(phi))
    c.permeability = np.full(nx, float(k0))
    c.alpha = np.zeros(nx)
    _zero_fields(c)
    _plug_flow(c, u)
    return c


def capillary_column(ny=1500, length=1.0, model=BROOKS_COREY, phi=0.5, k0=1e-11, dt=None, **kw) -> Case:
    """Gravity-capillarity column of section 4.1.3 (1 m, 1500 cells, porosity 0.5,
    k0 = 1e-11 m^2): water (1000, 1e-3) and air (1, 1.76e-5), lower half at
    saturation 0.5, upper half dry, gravity -9.81 m/s^2 along y; closed bottom and
    an open top (p = 0, zero-gradient velocity), so the column relaxes to the
    capillary-gravity equilibrium dp_c/dy = (rho_g - rho_l) g_y.  Brooks-Corey
    (kr m = 3, p_c0 = 100 Pa, beta = 0.5) or Van Genuchten (m = 0.5) closures
    (Table 2).  Fixed time step, by default 300 s (40 / ny)^2, about half the
    explicit capillary-diffusion limit h^2 / (2 D_max) (D = lambda |dp_c/dalpha| / phi
    peaks at 4.8e-7 m^2/s near alpha = 0.69 for Brooks-Corey): 0.21 s at the paper's
    1500 cells.  Above the limit the flux-corrected update stays bounded but the
    profile oscillates."""
    h = length / ny
    if dt is None:
        dt = 300.0 * (40.0 / ny) ** 2
    c = Case(name="capillary_column_%s_%d" % ("bc" if model == BROOKS_COREY else "vg", ny), nx=1, ny=ny, nz=1,
             h=h, rho_l=1000.0, mu_l=1e-3, rho_g=1.0, mu_g=1.76e-5, sigma=0.0, g=(0.0, -9.81, 0.0),
             kr_model=model, pc_model=model, kr_m=3.0 if model == BROOKS_COREY else 0.5, pc0=100.0,
             pc_beta=0.5, pc_m=0.5, bc=(WALL, WALL, WALL, OUTLET, WALL, WALL), inlet_u=0.0,
             dt=dt, dt_max=dt, cfl=0.0, p_tol=1e-12, max_cg=500)
    c = c.replace(**kw)
    c.porosity = np.full(ny, float(phi))
    c.permeability = np.full(ny, float(k0))
    a = np.zeros(ny)
    a[: ny // 2] = 0.5
    c.alpha = a
    _zero_fields(c)
    return c


def capillary_rise(cells_across=16, walls=2, width=1e-3, height=12.5e-3, meniscus=8e-3, theta=45.0,
                   mu_l=1e-2, **kw) -> Case:
    """Capillary rise of section 4.2.2: a 2-D tube 1 mm wide between porous walls of
    negligible permeability (k0 = 1e-20 m^2, porosity 0.5, ``walls`` cells thick), water
    below ``meniscus`` and air above, contact angle 45 degrees, gravity -9.81 m/s^2 along y.
    The bottom is a pressure boundary at the level of an infinite reservoir (p = 0, water
    enters with the saturation of the cell above it) and the top is open (p = 0), so the
    meniscus rises toward h = 2 sigma cos(theta) / (rho g width) = 10.1 mm.  The liquid
    viscosity defaults to 1e-2 Pa s (ten times water's) to damp the approach; the time
    step is 0.3 of the capillary-wave limit sqrt(rho_mean h^3 / (2 pi sigma))."""
    h = width / cells_across
    nx = cells_across + 2 * walls
    ny = int(round(height / h))
    dt = 0.3 * math.sqrt(500.0 * h ** 3 / (2.0 * math.pi * 0.07))
    c = Case(name="capillary_rise_%dx%d" % (nx, ny), nx=nx, ny=ny, nz=1, h=h, rho_l=1000.0, mu_l=mu_l,
             rho_g=1.0, mu_g=0.018 * mu_l, sigma=0.07, theta_deg=theta, g=(0.0, -9.81, 0.0), pc0=0.0,
             dt=dt, dt_max=dt, cfl=0.0, bc=(WALL, WALL, OUTLET, OUTLET, WALL, WALL), inlet_u=0.0,
             p_tol=1e-10, max_cg=500)
    c = c.replace(**kw)
    phi = np.ones((ny, nx))
    phi[:, :walls] = 0.5
    phi[:, nx - walls:] = 0.5
    a = np.zeros((ny, nx))
    a[: int(round(meniscus / h)), :] = 1.0
    c.porosity = to_xfast(phi[None])
    c.permeability = to_xfast(np.where(phi < 1.0, 1e-20, 0.0)[None])
    c.alpha = to_xfast(a[None])
    _zero_fields(c)
    return c


def batched_domains(count=512, seed=4, frac3d=0.75, lo3=32, hi3=96, lo2=64, hi2=256, **kw):
    """Uneven independent domains: sides log-uniform in [lo3, hi3] (3-D) or [lo2, hi2] (2-D)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        if rng.uniform() < frac3d:
            s = int(round(math.exp(rng.uniform(math.log(lo3), math.log(hi3)))))
            shape = (s, s, s)
        else:
            s = int(round(math.exp(rng.uniform(math.log(lo2), math.log(hi2)))))
            shape = (s, s, 1)
        out.append(darcy_domain(shape, seed=int(rng.integers(1 << 31)), **kw))
    return out


def poisson_requests(rate=20.0, duration=60.0, seed=5, lo=32, hi=192, ca_lo=1e-5, ca_hi=1e-2,
                     sigma=0.07, mu_w=1e-3):
    """Arrival trace of fractured-porous requests: (t_arrival, side, capillary number, inlet_u, seed)."""
    rng = np.random.default_rng(seed)
    t, reqs = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t > duration:
            break
        side = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        ca = math.exp(rng.uniform(math.log(ca_lo), math.log(ca_hi)))
        reqs.append({"t": t, "side": side, "ca": ca, "inlet_u": ca * sigma / mu_w,
                     "seed": int(rng.integers(1 << 31))})
    return reqs
