"""Pins of the oracle's closures (Appendix A; Eqs. 37, 38, 42, 45, 54) against
values the paper prints and closed forms derived by hand."""
import math
import os

import numpy as np
import pytest

from oracle import api
from paper_2003_08374_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _case(**kw):
    c = W.Case(name="closure", nx=1, ny=1, nz=1, h=1.0)
    return c.replace(**kw)


def _bisect(f, lo, hi, it=200):
    flo = f(lo)
    for _ in range(it):
        mid = 0.5 * (lo + hi)
        fm = f(mid)
        if (fm > 0) == (flo > 0):
            lo, flo = mid, fm
        else:
            hi = mid
    return 0.5 * (lo + hi)


def test_gravity_front_saturation_matches_paper():
    """Section 4.1.2, Eq. 54: k0 k_rl(alpha_f) rho_l g / mu_l = v_inj.  The paper
    prints alpha_f = 0.467 (Brooks-Corey m=3) and 0.753 (Van Genuchten m=0.5)."""
    rows = [l.split() for l in open(os.path.join(GOLD, "gravity_front.txt"))
            if l.strip() and not l.startswith("#")]
    v, k0, rho, mu, g = 1e-5, 1e-11, 1000.0, 1e-3, 9.81
    for name, m, expect in rows:
        model = W.BROOKS_COREY if name == "brooks_corey" else W.VAN_GENUCHTEN
        c = _case(kr_model=model, kr_m=float(m), mu_l=mu, rho_l=rho)
        af = _bisect(lambda a: k0 * api.closures(c, a, k0)[0] * rho * g / mu - v, 1e-9, 1 - 1e-9)
        # one unit of the last printed digit (the paper truncates: 0.7536 is printed 0.753)
        assert abs(af - float(expect)) < 1e-3, (name, af, expect)


def test_brooks_corey_closed_forms():
    c = _case(kr_model=W.BROOKS_COREY, kr_m=2.0, pc_model=W.BROOKS_COREY, pc0=100.0, pc_beta=0.5)
    krl, krg, *_ = api.closures(c, 0.5, 1e-12)
    assert krl == pytest.approx(0.25, rel=1e-15) and krg == pytest.approx(0.25, rel=1e-15)
    krl, krg, *_ = api.closures(c, 0.2, 1e-12)
    assert krl == pytest.approx(0.04, rel=1e-14) and krg == pytest.approx(0.64, rel=1e-14)
    # p_c = p0 * s^-beta: s = 0.25 -> 2 p0 ; s = 0.04 -> 5 p0
    assert api.closures(c, 0.25, 1e-12)[6] == pytest.approx(200.0, rel=1e-14)
    assert api.closures(c, 0.04, 1e-12)[6] == pytest.approx(500.0, rel=1e-14)
    # irreducible saturations rescale the effective saturation (Appendix A.1)
    c2 = c.replace(a_l_irr=0.2, a_g_irr=0.2)
    krl, krg, *_ = api.closures(c2, 0.5, 1e-12)
    assert krl == pytest.approx(0.25, rel=1e-14)
    krl, krg, *_ = api.closures(c2, 0.1, 1e-12)   # below irreducible -> clamped to 0
    assert krl == 0.0 and krg == 1.0


def test_van_genuchten_closed_forms():
    c = _case(kr_model=W.VAN_GENUCHTEN, kr_m=0.5, pc_model=W.VAN_GENUCHTEN, pc_m=0.5, pc0=100.0)
    # m = 1/2: s^(1/m) = s^2.  s = 0.6: krg = sqrt(0.4) (1 - 0.36)^1 = 0.64 sqrt(0.4)
    krl, krg, *_ = api.closures(c, 0.6, 1e-12)
    assert krg == pytest.approx(0.64 * math.sqrt(0.4), rel=1e-14)
    # krl = sqrt(0.6) (1 - (1 - 0.36)^0.5)^2 = sqrt(0.6) (1 - 0.8)^2 = 0.04 sqrt(0.6)
    assert krl == pytest.approx(0.04 * math.sqrt(0.6), rel=1e-12)
    # p_c = p0 (s^-2 - 1)^(1/2): s = 0.5 -> p0 sqrt(3)
    assert api.closures(c, 0.5, 1e-12)[6] == pytest.approx(100.0 * math.sqrt(3.0), rel=1e-14)
    # end points: fully saturated phases move alone
    krl, krg, *_ = api.closures(c, 1.0, 1e-12)
    assert krl == pytest.approx(1.0) and krg == 0.0


@pytest.mark.parametrize("model", [W.BROOKS_COREY, W.VAN_GENUCHTEN])
def test_single_phase_limits_reduce_to_darcy(model):
    """Eq. 42 with one phase present: mu k^-1 = mu_i / k0 (Darcy's law), rho* = rho_i (Eq. 45)."""
    c = _case(kr_model=model, kr_m=2.0 if model == W.BROOKS_COREY else 0.5)
    k0 = 3e-13
    o = api.closures(c, 1.0, k0)
    assert o[4] == pytest.approx(c.mu_l / k0, rel=1e-14) and o[5] == pytest.approx(c.rho_l, rel=1e-14)
    o = api.closures(c, 0.0, k0)
    assert o[4] == pytest.approx(c.mu_g / k0, rel=1e-14) and o[5] == pytest.approx(c.rho_g, rel=1e-14)


def test_harmonic_mobility_and_fractional_flow():
    """Eq. 42 (the form printed in the summary; Eq. 37 prints the ratio inverted):
    M^-1 = 1/(k0 (k_rl/mu_l + k_rg/mu_g)).  With equal kr the liquid fractional flow is
    M_l/M = mu_g/(mu_l + mu_g), the textbook Buckley-Leverett f_w."""
    c = _case(kr_model=W.BROOKS_COREY, kr_m=2.0, mu_l=1e-3, mu_g=1.8e-5)
    k0 = 1e-12
    krl, krg, Ml, Mg, drag, rho, pc, cf = api.closures(c, 0.5, k0)
    assert drag == pytest.approx(1.0 / (k0 * 0.25 * (1 / 1e-3 + 1 / 1.8e-5)), rel=1e-14)
    assert Ml / (Ml + Mg) == pytest.approx(1.8e-5 / (1e-3 + 1.8e-5), rel=1e-14)


@pytest.mark.parametrize("alpha", [0.05, 0.3, 0.5, 0.77, 0.95])
@pytest.mark.parametrize("model", [W.BROOKS_COREY, W.VAN_GENUCHTEN])
def test_appendix_b_equivalence(alpha, model):
    """Appendix B: the main-text form (rho* in buoyancy, Eq. 38 capillary force) equals the
    alternative form (alpha-weighted rho, F_c with M^-1(M_l a_g - M_g a_l)(rho_l - rho_g) g).
    Equivalently rho* - (a rho_l + (1-a) rho_g) = cf (rho_l - rho_g), cf = M^-1(M_l a_g - M_g a_l)."""
    c = _case(kr_model=model, kr_m=3.0 if model == W.BROOKS_COREY else 0.5,
              rho_l=1000.0, rho_g=800.0, mu_l=1e-3, mu_g=1e-2)
    o = api.closures(c, alpha, 2e-13)
    rho_star, cf = o[5], o[7]
    rho_a = alpha * c.rho_l + (1 - alpha) * c.rho_g
    assert rho_star - rho_a == pytest.approx(cf * (c.rho_l - c.rho_g), rel=1e-10, abs=1e-12)
