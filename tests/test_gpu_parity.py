"""Parity of the CUDA path (through the C-ABI) with the FP64 oracle on identical
seeded inputs.  FP64: relative L2 <= 1e-9 on alpha, p and every velocity
component; mixed precision: <= 1e-6."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL64 = 1e-9
TOLMIX = 1e-6
# Both sides solve the pressure equation to a relative residual of 1e-15, which
# the GMG-PCG reaches: velocities are differences of HbyA and the pressure
# gradient, so a looser stopping tolerance (1e-12) alone leaves ~1e-8 relative
# differences in u between any two correct solvers.


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2003_08374_gb300.build import build_library
    from oracle.build import build_oracle
    build_library()
    build_oracle()


def rel(a, b):
    nb = np.linalg.norm(b)
    if nb == 0.0:
        return float(np.linalg.norm(a))
    return float(np.linalg.norm(a - b) / nb)


def run_both(case, steps):
    from oracle.api import OracleSim
    from paper_2003_08374_gb300 import mdbs
    g = mdbs.Simulation(case)
    o = OracleSim(case)
    g.step(steps)
    o.step(steps)
    return g, o


def check_fields(g, o, tol):
    """Relative L2 of alpha, p and the velocity vector field u = (ux, uy, uz); each velocity
    component's error is also reported relative to |u| (a component that vanishes by
    symmetry carries only round-off, so its own relative error is meaningless)."""
    fg, fo = g.fields(), o.fields()
    ug = np.concatenate([fg["ux"], fg["uy"], fg["uz"]])
    uo = np.concatenate([fo["ux"], fo["uy"], fo["uz"]])
    errs = {"alpha": rel(fg["alpha"], fo["alpha"]), "p": rel(fg["p"], fo["p"]), "u": rel(ug, uo)}
    un = np.linalg.norm(uo)
    for n in ("ux", "uy", "uz"):
        if fo[n].size and un > 0:
            errs[n + "/|u|"] = float(np.linalg.norm(fg[n] - fo[n]) / un)
    bad = {n: e for n, e in errs.items() if not e <= tol}
    assert not bad, errs
    return errs


def test_stage_arrays_after_one_step():
    """Every intermediate array of one step (fluxes, limiter, closures, momentum
    coefficients, pressure system) against the oracle's."""
    from paper_2003_08374_gb300 import workloads as W
    case = W.fracture_2d(nx=24, ny=16, p_tol=1e-15, max_cg=500)
    g, o = run_both(case, 1)
    for name in ["FLOx", "FLOy", "AFx", "AFy", "aL", "Rp", "Rm", "rho", "mu", "drag", "pc", "cf",
                 "Ml", "Mg", "mx", "my", "kappa", "aPx", "aPy", "rhs0x", "rhs0y", "Bx", "By", "Tx", "Ty",
                 "Dd", "b", "hbyax", "hbyay", "nwx", "nwy"]:
        a, b = g.array(name), o.array(name)
        assert a.shape == b.shape, name
        assert rel(a, b) <= 1e-11, (name, rel(a, b))
    check_fields(g, o, 1e-10)


def test_fracture_2d_64_100_steps():
    """The 2-D 64x64 fracture workload (dx 10 um, dt 1e-6 s, 100 steps), FP64."""
    from paper_2003_08374_gb300 import workloads as W
    case = W.fracture_2d(nx=64, ny=64, p_tol=1e-15, max_cg=500)
    g, o = run_both(case, 100)
    check_fields(g, o, TOL64)
    sg, so = g.stats(), o.stats()
    assert abs(sg["mass"] - so["mass"]) <= 1e-12 * so["mass"]


@pytest.mark.parametrize("shape", [(20, 18, 16), (13, 9, 11), (33, 8, 5)])
def test_grf_3d_ragged(shape):
    """3-D log-normal porous block with a fracture, gravity, water into oil; ragged sizes that
    leave odd cells at every multigrid level."""
    from paper_2003_08374_gb300 import workloads as W
    case = W.grf_3d(shape=shape, seed=7, corr_len=3.0, frac_w=2, p_tol=1e-15, max_cg=500)
    g, o = run_both(case, 10)
    check_fields(g, o, TOL64)


def test_wave_tank_small_cfl():
    """Small wave tank: Van Genuchten closures, porous barrier, open top, adaptive CFL time step."""
    from paper_2003_08374_gb300 import workloads as W
    case = W.wave_tank(nx=32, ny=6, nz=20, h=5e-3, depth=10, x0=8, barrier=(20, 26, 8), p_tol=1e-15,
                       max_cg=500, precision=W.FP64, dt=1e-4)
    g, o = run_both(case, 10)
    check_fields(g, o, TOL64)
    assert g.stats()["dt"] == pytest.approx(o.stats()["dt"], rel=1e-9)


def test_appendix_b_density_matches_oracle():
    """Appendix B's saturation-weighted porous density with the extended capillary force,
    on the ragged fractured block (porous, free and mixed faces, gravity) and on the
    wave tank's porous barrier."""
    from paper_2003_08374_gb300 import workloads as W
    # (20, 18, 16) as in the ragged test: the (21, 18, 11) block amplifies one-ulp differences
    # to 1e-8 in u within 7 steps in the oracle itself (the test of the fracture corner case
    # bounds the CUDA path by that spread)
    case = W.grf_3d(shape=(20, 18, 16), seed=7, corr_len=3.0, frac_w=2, p_tol=1e-15, max_cg=500,
                    porous_density=W.RHO_SATURATION)
    g, o = run_both(case, 10)
    check_fields(g, o, TOL64)
    case = W.wave_tank(nx=32, ny=6, nz=20, h=5e-3, depth=10, x0=8, barrier=(20, 26, 8), p_tol=1e-15,
                       max_cg=500, precision=W.FP64, dt=1e-4, porous_density=W.RHO_SATURATION)
    # 10 steps, as for the main-text wave tank: the free surface amplifies rounding
    # differences about twofold per step once the adaptive step has grown (u: 1e-13
    # relative after 10 steps, 2e-10 after 20)
    g, o = run_both(case, 10)
    check_fields(g, o, TOL64)


def test_darcy_domain_and_2d_shapes():
    from paper_2003_08374_gb300 import workloads as W
    for shape in [(17, 23, 1), (9, 7, 6)]:
        case = W.darcy_domain(shape, seed=3, p_tol=1e-15, max_cg=500)
        g, o = run_both(case, 5)
        check_fields(g, o, TOL64)


@pytest.mark.parametrize("shape", [(1, 1, 1), (3, 2, 1), (1, 5, 1), (2, 2, 2), (5, 1, 3)])
def test_degenerate_grids(shape):
    """Single cell, single row / column, 2x2x2: no multigrid coarsening, boundary-only faces."""
    from paper_2003_08374_gb300 import workloads as W
    case = W.darcy_domain(shape, seed=1, p_tol=1e-15, max_cg=200, sat=0.4)
    g, o = run_both(case, 3)
    check_fields(g, o, TOL64)


@pytest.mark.parametrize("precision", [1, 2])
def test_mixed_precision_matches_fp64_oracle(precision):
    """FP32 V-cycle (coarse coefficients in BF16 for precision 2) inside FP64 flexible CG,
    solved to 1e-14: within 1e-6 of the FP64 oracle."""
    from paper_2003_08374_gb300 import workloads as W
    case = W.grf_3d(shape=(24, 20, 16), seed=5, corr_len=4.0, frac_w=4, p_tol=1e-14, max_cg=500,
                    precision=precision)
    g, o = run_both(case, 10)
    check_fields(g, o, TOLMIX)


def _developed_block(steps=20):
    """The fractured 3-D block of the mixed-precision tests, advanced by the oracle (at 1e-15)
    from its initial state: the state a benchmark step starts from (warm pressure)."""
    from oracle.api import OracleSim
    from paper_2003_08374_gb300 import workloads as W
    case = W.grf_3d(shape=(24, 20, 16), seed=5, corr_len=4.0, frac_w=4, p_tol=1e-15, max_cg=500)
    o = OracleSim(case)
    o.step(steps)
    return case, o


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_step_at_bench_tolerance_against_fp64_oracle(precision):
    """One step at the benchmark's pressure residual 1e-8 -- FP64, the FP32 V-cycle, and BF16
    coarse coefficients -- from a developed state, against the FP64 oracle's step solved to
    1e-15: within 1e-6 relative L2 on alpha, p and u.  The errors are printed (pytest -s)."""
    from paper_2003_08374_gb300 import mdbs
    case, o = _developed_block()
    f = o.fields()
    g = mdbs.Simulation(case.replace(p_tol=1e-8, precision=precision))
    g.set_fields(f["alpha"], f["ux"], f["uy"], f["uz"], f["p"])
    g.step(1)
    o.step(1)
    errs = check_fields(g, o, TOLMIX)
    print("one step, precision %d at p_tol 1e-8 vs oracle at 1e-15: %s" % (
        precision, {k: "%.2e" % v for k, v in errs.items()}))


@pytest.mark.parametrize("which", ["grf", "fracture_2d", "wave_tank"])
def test_cg_iterations_match_the_oracles_preconditioner(which):
    """The GPU's V-cycle is the oracle's preconditioner (same hierarchy, coarse operator,
    red-black order, exact coarsest solve), so at the bench tolerance 1e-8 each corrector's
    CG takes the oracle's number of iterations (one more or fewer where rounding moves the
    residual across the threshold) over several steps; a preconditioner that differed in
    quality would change the counts by several."""
    from oracle.api import OracleSim
    from paper_2003_08374_gb300 import mdbs
    from paper_2003_08374_gb300 import workloads as W
    case = {"grf": W.grf_3d(shape=(24, 20, 16), seed=3, corr_len=3.0, frac_w=2, p_tol=1e-8, max_cg=300),
            "fracture_2d": W.fracture_2d(nx=64, ny=64, p_tol=1e-8, max_cg=300),
            "wave_tank": W.wave_tank(nx=32, ny=6, nz=20, h=5e-3, depth=10, x0=8, barrier=(20, 26, 8),
                                     p_tol=1e-8, max_cg=300)}[which]
    g = mdbs.Simulation(case)
    o = OracleSim(case)
    seen = []
    for _ in range(4):
        g.step(1)
        o.step(1)
        ig, io = g.stats()["cg_iters"], o.stats()["cg_iters"]
        seen.append((ig, io))
        assert all(abs(a - b) <= 1 for a, b in zip(ig, io)), seen
    assert sum(sum(io) for _, io in seen) > 0
    print(which, "iterations (GPU, oracle) per step:", seen)


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_run_at_bench_tolerance_drifts_only_as_the_tolerance_allows(precision):
    """Over 100 steps at a pressure residual of 1e-8 the solution drifts from the one solved to
    1e-15 (the oracle against itself: alpha 2.4e-6, p 5.1e-6, u 2.0e-3 relative L2 on this
    block), because every corrected flux keeps a divergence of the size of the residual.  The
    CUDA path in every precision drifts no further than three times the oracle's own drift at
    that tolerance: the precision of the preconditioner adds no error of its own."""
    from oracle.api import OracleSim
    from paper_2003_08374_gb300 import mdbs
    from paper_2003_08374_gb300 import workloads as W
    case = W.grf_3d(shape=(24, 20, 16), seed=5, corr_len=4.0, frac_w=4, p_tol=1e-15, max_cg=500)
    o15, o8 = OracleSim(case), OracleSim(case.replace(p_tol=1e-8))
    g = mdbs.Simulation(case.replace(p_tol=1e-8, precision=precision))
    for x in (o15, o8, g):
        x.step(100)
    f15, f8, fg = o15.fields(), o8.fields(), g.fields()
    report = {}
    for n in ("alpha", "p", "u"):
        if n == "u":
            a, b, c = (np.concatenate([f["ux"], f["uy"], f["uz"]]) for f in (fg, f8, f15))
        else:
            a, b, c = fg[n], f8[n], f15[n]
        drift, err = rel(b, c), rel(a, c)
        report[n] = "gpu %.2e / oracle %.2e" % (err, drift)
        assert err <= 3.0 * drift + 1e-9, (n, err, drift)
    print("100 steps, precision %d at p_tol 1e-8 vs oracle at 1e-15: %s" % (precision, report))


def test_grf_3d_100_steps():
    """A 3-D fractured block (gravity, water into oil, porous and free cells, ragged multigrid
    levels) over 100 steps, FP64, within 1e-9 of the oracle.  Surface tension is off here:
    with it, the case amplifies rounding itself (the next test)."""
    from paper_2003_08374_gb300 import workloads as W
    case = W.grf_3d(shape=(20, 18, 16), seed=7, corr_len=3.0, frac_w=2, p_tol=1e-15, max_cg=500, sigma=0.0)
    g, o = run_both(case, 100)
    check_fields(g, o, TOL64)


def _within_rounding_sensitivity(case, checkpoints, factor=3.0):
    """The CUDA path against the oracle, bounded by the oracle's own spread: the oracle
    started from velocities perturbed by one rounding unit.  Returns the largest error."""
    from oracle.api import OracleSim
    from paper_2003_08374_gb300 import mdbs
    pert = case.replace()
    pert.ux = case.ux * (1.0 + 2.2e-16)
    o, o2, g = OracleSim(case), OracleSim(pert), mdbs.Simulation(case)
    done, worst = 0, 0.0
    for step in checkpoints:
        for x in (o, o2, g):
            x.step(step - done)
        done = step
        fo, fo2, fg = o.fields(), o2.fields(), g.fields()
        for n in ("alpha", "p", "ux", "uy", "uz"):
            spread = rel(fo2[n], fo[n])
            err = rel(fg[n], fo[n])
            worst = max(worst, err)
            assert err <= factor * spread + 1e-12, (step, n, err, spread)
    return worst


def test_fracture_corner_case_within_the_oracles_own_rounding_sensitivity():
    """With surface tension the step amplifies rounding: the interface normal
    m = grad(a) / (|grad(a)| + 1e-8/h) changes by 5e7 times a one-ulp change of alpha in
    nearly uniform cells, and the curvature of the next interface cell, and its CSF force,
    follow.  The oracle started from velocities perturbed by one rounding unit departs from
    itself by about 1e-9 after two steps and 8e-9 after seven on the (21, 18, 11) block with
    a 2-cell fracture, and by 1.4e-9 after 100 steps on the (20, 18, 16) block.  The CUDA
    path must stay as close to the oracle as that: within three times the oracle's own
    spread at every checkpoint."""
    from paper_2003_08374_gb300 import workloads as W
    worst = _within_rounding_sensitivity(
        W.grf_3d(shape=(21, 18, 11), seed=7, corr_len=3.0, frac_w=2, p_tol=1e-15, max_cg=500), range(1, 8))
    assert worst > 1e-10  # the case is as sensitive as stated: this is not a trivially equal run
    _within_rounding_sensitivity(
        W.grf_3d(shape=(20, 18, 16), seed=7, corr_len=3.0, frac_w=2, p_tol=1e-15, max_cg=500), (25, 50, 75, 100))


def test_deterministic_rerun():
    """Fixed reduction order: the same inputs give bit-identical fields."""
    from paper_2003_08374_gb300 import mdbs
    from paper_2003_08374_gb300 import workloads as W
    case = W.grf_3d(shape=(16, 16, 16), seed=2, corr_len=4.0, frac_w=2, p_tol=1e-10)
    a = mdbs.Simulation(case)
    a.step(5)
    b = mdbs.Simulation(case)
    b.step(5)
    fa, fb = a.fields(), b.fields()
    for n in fa:
        assert np.array_equal(fa[n], fb[n]), n


def test_set_fields_rejects_bad_alpha_and_invalid_create():
    from paper_2003_08374_gb300 import mdbs
    from paper_2003_08374_gb300 import workloads as W
    case = W.fracture_2d(nx=8, ny=8)
    s = mdbs.Simulation(case)
    bad = case.alpha.copy()
    bad[3] = 1.5
    with pytest.raises(mdbs.MdbsError) as e:
        s.set_fields(bad, case.ux, case.uy, case.uz, case.p)
    assert e.value.code == mdbs.ERR_ARG
    # the check runs on the device: a NaN in the last cell of a field larger than the
    # check's grid is caught, and a rejected call leaves the state as it was
    big = W.grf_3d(shape=(160, 130, 64), seed=3, corr_len=3.0, frac_w=2)
    g = mdbs.Simulation(big)
    g.step(1)
    before = g.fields()
    bad = before["alpha"].copy()
    bad[-1] = np.nan
    with pytest.raises(mdbs.MdbsError) as e:
        g.set_fields(bad, before["ux"], before["uy"], before["uz"], before["p"])
    assert e.value.code == mdbs.ERR_ARG
    after = g.fields()
    assert all(np.array_equal(before[k], after[k]) for k in before)
    g.step(1)
    g.close()
    c2 = case.replace(bc=(W.WALL,) * 6)
    with pytest.raises(mdbs.MdbsError):
        mdbs.Simulation(c2)
    c3 = case.replace(porosity=np.zeros(64))
    with pytest.raises(mdbs.MdbsError):
        mdbs.Simulation(c3)
