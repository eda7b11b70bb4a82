"""Pins of the oracle's momentum predictor (Eq. 21 with the discretisation of
section 3.1, Eqs. 46-50) against what the mathematics fixes:

* the porous/free similarity of Eq. 21: in a uniform porous medium of porosity
  phi and negligible drag, v = phi w where w solves the solid-free equations
  with viscosity phi mu (same density, same pressure) -- this holds term by
  term for the 1/phi Euler factor, the 1/phi^2 convection factor, the viscous
  stress and the CFL speed |v|/phi of section 3.2;
* the spin-up of a porous column under gravity, whose time constant
  rho k / (phi mu) is set by the 1/phi on the time derivative;
* rigid-body rotation, which the full stress S = mu (grad v + grad v^T) leaves
  stress-free for any viscosity field (the transpose part cancels the
  viscosity-gradient part of div(mu grad v));
* the development length of laminar plane-channel flow from a uniform inlet
  (Durst, Ray, Uensal & Bayoumi, J. Fluids Eng. 127 (2005) 1154, the
  correlation L/H = [0.631^1.6 + (0.0442 Re)^1.6]^(1/1.6)), which the
  convective term sets;
* the time step from the CFL number on the interstitial velocity u/phi.
"""
import math

import numpy as np
import pytest

from oracle.api import OracleSim
from paper_2003_08374_gb300 import workloads as W


def make_case(nx, ny, nz, h, phi, k, alpha, **kw):
    c = W.Case(name="pin", nx=nx, ny=ny, nz=nz, h=h, **kw)
    c.porosity = np.ascontiguousarray(np.broadcast_to(phi, (nx * ny * nz,)), dtype=float)
    c.permeability = np.ascontiguousarray(np.broadcast_to(k, (nx * ny * nz,)), dtype=float)
    c.alpha = np.ascontiguousarray(np.broadcast_to(alpha, (nx * ny * nz,)), dtype=float)
    W._zero_fields(c)
    return c


@pytest.mark.parametrize("cfl", [0.0, 0.5])
def test_porous_channel_is_a_scaled_free_channel(cfl):
    """Eq. 21 in a uniform medium (phi = 0.5, k0 so large that mu/k0 is 1e-30 of the inertia):
    substituting v = phi w turns (rho/phi) dv/dt + (rho/phi^2)(v.grad)v = -grad p + div(mu grad v)
    into the solid-free equation for w with viscosity phi mu.  A developing channel flow
    started impulsively (inlet U into the porous channel, U/phi into the free one, Re about
    160) must therefore give u_porous = phi u_free and the same pressure at every step -- with
    cfl > 0 also the same adaptive time step, since section 3.2's CFL speed is |u|/phi.
    phi = 0.5 makes every scaling exact in binary, so only the pressure tolerance remains."""
    nx, ny, phi, U, mu = 32, 8, 0.5, 0.5, 0.1
    common = dict(rho_l=1.0, rho_g=1.0, sigma=0.0, pc0=0.0, c_alpha=0.0, dt=0.1, cfl=cfl, dt_max=10.0,
                  p_tol=1e-13, max_cg=500)
    por = OracleSim(make_case(nx, ny, 1, 1.0, phi, 1e20, 1.0, mu_l=mu, mu_g=mu, inlet_u=U, **common))
    fre = OracleSim(make_case(nx, ny, 1, 1.0, 1.0, 0.0, 1.0, mu_l=phi * mu, mu_g=phi * mu, inlet_u=U / phi,
                              **common))
    for _ in range(4):
        por.step(10)
        fre.step(10)
        fp, ff = por.fields(), fre.fields()
        for name in ("ux", "uy"):
            ref = phi * ff[name]
            assert np.abs(fp[name] - ref).max() <= 1e-11 * np.abs(ref).max(), name
        assert np.abs(fp["p"] - ff["p"]).max() <= 1e-11 * np.abs(ff["p"]).max()
        assert por.stats()["dt"] == pytest.approx(fre.stats()["dt"], rel=1e-12)
    # the flow is developing: cross-stream velocities are a sizeable part of the inlet velocity
    assert np.abs(ff["uy"]).max() > 0.02 * U / phi
    if cfl > 0.0:
        assert fre.stats()["dt"] != pytest.approx(0.1 * 1.2 ** 40, rel=1e-3)  # the CFL bound is active


def _spin_up_error(dt_over_tau, t_end_over_tau=3.0):
    ny, h = 8, 1e-2
    k, rho, mu, g, phi = 1e-12, 1000.0, 1e-3, 9.81, 0.5
    tau = rho * k / (phi * mu)
    dt = dt_over_tau * tau
    c = make_case(1, ny, 1, h, phi, k, 1.0, rho_l=rho, rho_g=rho, mu_l=mu, mu_g=mu, sigma=0.0, pc0=0.0,
                  g=(0.0, -g, 0.0), bc=(W.WALL, W.WALL, W.OUTLET, W.OUTLET, W.WALL, W.WALL), inlet_u=0.0,
                  dt=dt, dt_max=dt, p_tol=1e-13, max_cg=200)
    s = OracleSim(c)
    u_inf = k * rho * g / mu
    err = 0.0
    for n in range(int(round(t_end_over_tau / dt_over_tau))):
        s.step(1)
        uy = -s.fields()["uy"]
        t = (n + 1) * dt
        exact = u_inf * (1.0 - math.exp(-t / tau))
        err = max(err, float(np.abs(uy[1:-1] - exact).max()) / u_inf)
    return err


def test_porous_column_spins_up_with_time_constant_rho_k_over_phi_mu():
    """A water-filled vertical porous column open at both ends (p = 0 top and bottom), at rest
    when gravity acts: Eq. 21 reduces to (rho/phi) du/dt = rho g - (mu/k) u, so
    u(t) = (k rho g / mu)(1 - exp(-t phi mu / (rho k))).  The implicit Euler step of section 3.1
    is first-order accurate: its error is at most about 0.18 dt/tau over the transient, and
    halves with the time step.  (The side walls' shear, 4 mu/h^2, is 4e-8 of mu/k here.)"""
    e1 = _spin_up_error(0.02)
    e2 = _spin_up_error(0.01)
    assert e1 <= 0.2 * 0.02 and e2 <= 0.2 * 0.01, (e1, e2)
    assert 1.8 <= e1 / e2 <= 2.2, (e1, e2)


def _face_coords(n, d):
    """Cell-centred coordinates (x, y, z) of the d-faces of an n^3 grid of unit cells,
    shaped (nz', ny', nx') with the face axis one longer."""
    shape = [n, n, n]
    shape[2 - d] += 1
    z, y, x = np.meshgrid(*[np.arange(s, dtype=float) for s in shape], indexing="ij")
    pos = [x + 0.5, y + 0.5, z + 0.5]
    pos[d] = [x, y, z][d].copy()
    return [p - n / 2.0 for p in pos]


def test_rigid_rotation_is_stress_free_for_any_viscosity():
    """S = mu (grad v + grad v^T) of Eq. 21 vanishes for a rigid-body rotation v = Omega x r,
    whatever the viscosity field, while div(mu grad v) alone does not where mu varies.  With
    density so small that inertia and convection drop out, the assembled momentum equation of
    every interior face, a_P u_f - sum a_nb u_nb - rhs0, is then the viscous force, and it must
    vanish to rounding in all three directions for a smoothly varying two-phase viscosity
    (the discrete stencils are exact for linear fields)."""
    n, h = 10, 1e-3
    Om = np.array([0.7, -1.1, 1.9])
    z, y, x = np.meshgrid(*[np.arange(n) + 0.5] * 3, indexing="ij")
    a = 0.5 + 0.45 * np.sin(2 * np.pi * x / n + 0.3) * np.cos(2 * np.pi * y / n) * np.cos(np.pi * z / n)
    c = make_case(n, n, n, h, 1.0, 0.0, a.ravel(), rho_l=1e-20, rho_g=1e-20, mu_l=1e-3, mu_g=4e-2,
                  sigma=0.0, bc=(W.WALL, W.WALL, W.WALL, W.WALL, W.WALL, W.OUTLET), inlet_u=0.0,
                  dt=1e-12, dt_max=1e-12, p_tol=1e-10, c_alpha=0.0)
    vel = []
    for d in range(3):
        r = [p * h for p in _face_coords(n, d)]
        vel.append(np.cross(Om, np.stack(r, axis=-1))[..., d])
    c.ux, c.uy, c.uz = (v.ravel().copy() for v in vel)
    s = OracleSim(c)
    s.step(1)
    interior = (slice(2, n - 2),) * 3
    for d, name in enumerate("xyz"):
        aP = s.array("aP" + name).reshape(vel[d].shape)
        anb = s.array("anb" + name).reshape(vel[d].shape + (6,))
        rhs0 = s.array("rhs0" + name).reshape(vel[d].shape)
        u = vel[d]
        hs = np.zeros_like(u)
        visc = np.zeros_like(u)
        for e in range(3):
            ax = 2 - e
            lo = np.roll(u, 1, axis=ax)
            hi = np.roll(u, -1, axis=ax)
            hs += anb[..., 2 * e] * lo + anb[..., 2 * e + 1] * hi
            visc += np.abs(anb[..., 2 * e] * (u - lo)) + np.abs(anb[..., 2 * e + 1] * (u - hi))
        resid = (aP * u - hs - rhs0)[interior]
        scale = visc[interior].max()
        assert scale > 0.0
        assert np.abs(resid).max() <= 1e-12 * scale, (name, np.abs(resid).max() / scale)
        # the transpose part is active: the explicit source is a sizeable share of the stress
        assert np.abs(rhs0[interior]).max() > 0.05 * scale, name


def _development_length(H, Re, length):
    nx, ny, U = length * H, H, 1.0
    nu = U * H / Re
    c = make_case(nx, ny, 1, 1.0, 1.0, 0.0, 1.0, rho_l=1.0, rho_g=1.0, mu_l=nu, mu_g=nu, sigma=0.0,
                  c_alpha=0.0, inlet_u=U, dt=0.5, dt_max=0.5, p_tol=1e-11, max_cg=500)
    W._plug_flow(c, U)
    s = OracleSim(c)
    prev = None
    for _ in range(20):
        s.step(200)
        ux = s.fields()["ux"].reshape(ny, nx + 1)
        if prev is not None and np.abs(ux - prev).max() < 1e-7:
            break
        prev = ux
    else:
        raise AssertionError("channel flow did not reach a steady state")
    ucl = 0.5 * (ux[ny // 2 - 1] + ux[ny // 2])
    u_dev = ucl[-H // 2:].mean()
    i = int(np.argmax(ucl >= 0.99 * u_dev))
    x99 = (i - 1) + (0.99 * u_dev - ucl[i - 1]) / (ucl[i] - ucl[i - 1])
    return x99 / H, u_dev


@pytest.mark.parametrize("Re,length", [(50.0, 6), (100.0, 8)])
def test_channel_development_length_matches_durst_correlation(Re, length):
    """Developing laminar flow between plates from a uniform inlet: the centreline velocity
    reaches 99 % of its developed value at L/H = [0.631^1.6 + (0.0442 Re)^1.6]^(1/1.6)
    (Durst et al. 2005; Re = U H / nu, H the channel height).  The convective term of Eq. 21
    sets this length (without it, L/H would stay near the creeping-flow 0.63); at 16 cells
    across, the first-order upwind convection lands within 6 %."""
    L, u_dev = _development_length(16, Re, length)
    expect = (0.631 ** 1.6 + (0.0442 * Re) ** 1.6) ** (1 / 1.6)
    assert L == pytest.approx(expect, rel=0.06), (L, expect)
    assert u_dev == pytest.approx(1.5, rel=0.02)  # developed Poiseuille centreline, 1.5 U


def test_cfl_time_step_uses_the_interstitial_velocity():
    """Section 3.2's CFL number is taken on the velocity inside the pores, |u|/phi: plug flow U
    through a uniform column of porosity 0.25 gives dt = CFL h phi / U."""
    nx, h, U, phi, cfl = 16, 1e-3, 1e-3, 0.25, 0.5
    c = make_case(nx, 1, 1, h, phi, 1e-12, 1.0, inlet_u=U, cfl=cfl, dt=1.0, dt_max=10.0, p_tol=1e-12,
                  max_cg=200)
    W._plug_flow(c, U)
    s = OracleSim(c)
    s.step(1)
    assert s.stats()["dt"] == pytest.approx(cfl * h * phi / U, rel=1e-9)


def test_porosity_jump_gives_the_interstitial_bernoulli_pressure():
    """Steady single-phase flow U through a column whose porosity changes along the flow (a
    solid-free inlet section, ramps and a jump; drag and viscosity negligible): Eq. 21's
    (1/phi) div(rho v v / phi) with v = U constant integrates to p + (rho/2)(U/phi)^2 = const,
    Bernoulli's relation for the velocity inside the pores.  The advective form alone gives no
    pressure change at all here; the discrete porosity-gradient term telescopes, so the jump
    holds to the pressure tolerance for any porosity profile."""
    phi = np.array([1.0] * 8 + list(np.linspace(1.0, 0.4, 10)) + [0.4] * 6 + [0.7] * 8 +
                   list(np.linspace(0.7, 0.25, 6)) + [0.25] * 6)
    nx, U, rho = phi.size, 0.8, 1.0
    c = make_case(nx, 1, 1, 1.0, 1.0, 1.0, 1.0, rho_l=rho, rho_g=rho, mu_l=1e-12, mu_g=1e-12, sigma=0.0,
                  pc0=0.0, c_alpha=0.0, inlet_u=U, dt=0.5, dt_max=0.5, p_tol=1e-13, max_cg=200)
    c.porosity = phi.copy()
    c.permeability = np.where(phi < 1.0, 1e30, 0.0)
    W._plug_flow(c, U)
    s = OracleSim(c)
    s.step(2)
    p = s.fields()["p"]
    expect = -0.5 * rho * U * U * (phi ** -2 - phi[0] ** -2)
    assert np.abs((p - p[0]) - expect).max() <= 1e-9 * np.abs(expect).max()


def _convection_error(n):
    """Largest deviation, over faces two cells or more from the walls, of the assembled
    momentum equation's convective force from (1/phi) div(rho v v_d / phi) of the smooth
    field v = curl(psi), psi = sin^2(pi x) sin^2(pi y) / pi^2, with
    phi = 0.55 + 0.3 sin(2 pi x + 0.4) cos(pi y) on the unit square (rho = 1, viscosity and
    drag negligible); relative to the largest force.  Per direction x, y."""
    h = 1.0 / n

    def psi(x, y):
        return np.sin(np.pi * x) ** 2 * np.sin(np.pi * y) ** 2 / np.pi ** 2

    def phif(x, y):
        return 0.55 + 0.3 * np.sin(2 * np.pi * x + 0.4) * np.cos(np.pi * y)

    xc = (np.arange(n) + 0.5) * h
    xn = np.arange(n + 1) * h
    Xc, Yc = np.meshgrid(xc, xc)
    Xn, Yn = np.meshgrid(xn, xn)
    P = psi(Xn, Yn)
    ux = (P[1:, :] - P[:-1, :]) / h  # face fluxes from the stream function: divergence free
    uy = -(P[:, 1:] - P[:, :-1]) / h
    c = make_case(n, n, 1, h, phif(Xc, Yc).ravel(), 1.0, 1.0, rho_l=1.0, rho_g=1.0, mu_l=1e-30, mu_g=1e-30,
                  sigma=0.0, pc0=0.0, c_alpha=0.0, inlet_u=0.0, dt=1e-9, dt_max=1e-9, p_tol=1e-12, max_cg=200,
                  bc=(W.WALL, W.WALL, W.WALL, W.OUTLET, W.WALL, W.WALL))
    c.ux, c.uy = ux.ravel().copy(), uy.ravel().copy()
    s = OracleSim(c)
    s.step(1)
    eps, E = 1e-5, 1e-4

    def vel(x, y):
        return ((psi(x, y + eps) - psi(x, y - eps)) / (2 * eps), -(psi(x + eps, y) - psi(x - eps, y)) / (2 * eps))

    out = []
    for d, name, u in ((0, "x", ux), (1, "y", uy)):
        aP = s.array("aP" + name).reshape(u.shape)
        anb = s.array("anb" + name).reshape(u.shape + (6,))
        rhs0 = s.array("rhs0" + name).reshape(u.shape)
        hs = (anb[..., 0] * np.roll(u, 1, 1) + anb[..., 1] * np.roll(u, -1, 1) + anb[..., 2] * np.roll(u, 1, 0) +
              anb[..., 3] * np.roll(u, -1, 0))
        force = (aP * u - hs - rhs0) / h ** 3
        X, Y = np.meshgrid(xn, xc) if d == 0 else np.meshgrid(xc, xn)

        def flux(x, y, j):
            v = vel(x, y)
            return v[j] * v[d] / phif(x, y)

        cont = ((flux(X + E, Y, 0) - flux(X - E, Y, 0)) + (flux(X, Y + E, 1) - flux(X, Y - E, 1))) / (2 * E)
        cont /= phif(X, Y)
        sl = (slice(2, -2), slice(2, -2))
        out.append(np.abs(force[sl] - cont[sl]).max() / np.abs(cont[sl]).max())
    return out


def test_discrete_convection_converges_to_the_conservative_form():
    """The assembled convection (upwind advective part plus the porosity-gradient part) is a
    first-order approximation of Eq. 21's (1/phi) div(rho v v / phi) for a smooth
    divergence-free flow through smoothly varying porosity: the error halves with the cell
    size.  Leaving out the porosity-gradient part (or mis-scaling a factor of phi) leaves an
    error that does not shrink."""
    e16 = _convection_error(16)
    e32 = _convection_error(32)
    for a, b in zip(e16, e32):
        assert b <= 0.15, (e16, e32)
        assert a / b >= 1.7, (e16, e32)
