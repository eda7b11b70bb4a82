"""Appendix B's formulation of the porous momentum balance: the saturation-weighted
density rho in porous cells, with the capillary force extended by
M^-1 (M_l a_g - M_g a_l)(rho_l - rho_g) g.  The appendix shows it equivalent to
the main text's mobility-weighted rho* (Eq. 45) with the plain capillary force
(Eq. 38): rho* - rho = c_f (rho_l - rho_g) cell by cell, so the buoyancy plus
capillary face forces agree, and only the inertia density differs -- negligible
wherever the Darcy drag dominates."""
import math

import numpy as np
import pytest

from oracle.api import OracleSim
from paper_2003_08374_gb300 import workloads as W


@pytest.fixture(scope="module", autouse=True)
def built():
    from oracle.build import build_oracle
    build_oracle()


def _porous_box(porous_density):
    """A porous-only 3-D box, gravity along z (normal to the outlet x+), capillarity on."""
    c = W.darcy_domain((12, 10, 8), seed=3, sat=0.4, p_tol=1e-13, max_cg=400, g=(0.0, 0.0, -9.81),
                       porous_density=porous_density, dt=1e-6)
    rng = np.random.default_rng(7)
    c.alpha = np.clip(0.4 + 0.3 * rng.standard_normal(c.cells), 0.02, 0.98)
    return c


def test_face_forces_agree_between_formulations():
    """One step from the same state: alpha^{k+1} is the same, and on every face the
    buoyancy + capillary force of Appendix B equals the main text's to rounding."""
    a, b = OracleSim(_porous_box(W.RHO_MOBILITY)), OracleSim(_porous_box(W.RHO_SATURATION))
    a.step(1)
    b.step(1)
    assert np.array_equal(a.fields()["alpha"], b.fields()["alpha"])
    ra, rb = a.array("rho"), b.array("rho")
    assert np.max(np.abs(ra - rb)) > 1.0  # the densities do differ
    for name in ("Bx", "By", "Bz"):
        fa, fb = a.array(name), b.array(name)
        scale = np.max(np.abs(fa))
        assert scale > 0 and np.max(np.abs(fa - fb)) <= 1e-12 * scale, name


@pytest.mark.parametrize("model,m", [(W.BROOKS_COREY, 3.0), (W.VAN_GENUCHTEN, 0.5)])
def test_darcy_column_same_under_both_formulations(model, m):
    """The gravity-dominated column of section 4.1.2 (dt ~ 4 s, drag ~ mu / k0 = 1e8 Pa s/m^2):
    inertia is ~1e-6 of the drag, so both formulations give the same saturations and fluxes
    to that order, and the same plateau."""
    out = []
    for form in (W.RHO_MOBILITY, W.RHO_SATURATION):
        c = W.buckley_leverett(nx=60, length=0.3, displaced="air", kr_model=model, kr_m=m, gravity=True,
                               porous_density=form)
        s = OracleSim(c)
        s.step(400)
        out.append((s.fields(), s.stats()))
    (fa, sa), (fb, sb) = out
    assert abs(sa["time"] - sb["time"]) <= 1e-9 * sa["time"]
    assert np.max(np.abs(fa["alpha"] - fb["alpha"])) <= 1e-6
    assert np.max(np.abs(fa["ux"] - fb["ux"])) <= 1e-6 * np.max(np.abs(fa["ux"]))
    # the pressure carries the buoyancy: equal only if the face forces are
    assert np.max(np.abs(fa["p"] - fb["p"])) <= 1e-6 * np.max(np.abs(fa["p"]))
    assert abs(sa["mass"] - sb["mass"]) <= 1e-9 * sa["mass"]


def test_gravity_capillary_equilibrium_under_appendix_b():
    """The capillary-gravity equilibrium of section 4.1.3 (dp_c/dy = (rho_g - rho_l) g) is
    also at rest with Appendix B's density and capillary force."""
    ny, L = 64, 0.02
    h = L / ny
    k0, rho_l, rho_g, g = 1e-11, 1000.0, 1.0, 9.81
    y = (np.arange(ny) + 0.5) * h
    pc = 100.0 / math.sqrt(0.9) + (rho_l - rho_g) * g * y
    alpha = (pc / 100.0) ** (-2.0)
    c = W.Case(name="col", nx=1, ny=ny, nz=1, h=h, rho_l=rho_l, rho_g=rho_g, mu_l=1e-3, mu_g=1.8e-5,
               g=(0.0, -g, 0.0), kr_m=3.0, pc0=100.0, pc_beta=0.5, pc_eps=1e-6,
               bc=(W.WALL, W.WALL, W.WALL, W.OUTLET, W.WALL, W.WALL), inlet_u=0.0, dt=1e-3, p_tol=1e-13,
               max_cg=500, porous_density=W.RHO_SATURATION)
    c.porosity = np.full(ny, 0.5)
    c.permeability = np.full(ny, k0)
    c.alpha = alpha
    W._zero_fields(c)
    s = OracleSim(c)
    s.step(1)
    a1 = s.fields()["alpha"]
    s.step(3)
    Ug = k0 * (rho_l - rho_g) * g / 1e-3
    f = s.fields()
    assert np.abs(f["uy"]).max() < 1e-9 * Ug
    assert np.abs(f["alpha"] - a1).max() < 1e-6
