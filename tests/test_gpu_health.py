"""Health and state handling at the C-ABI (section 3.2's step taken as a unit):

* a non-finite pressure set from the host is reported as MDBS_ERR_DIVERGED;
* a pressure solve that stops at max_cg above p_tol gives MDBS_ERR_NOT_CONVERGED
  after the requested steps were taken;
* checkpoint and restart: 2n steps straight equal n steps, a get_fields /
  set_fields round trip, and n more steps, bit for bit;
* new saturation input must lie in [0, 1] to 1e-9, while a state the simulation
  produced itself (alpha outside [0, 1] by the transport error of the pressure
  tolerance) survives a round trip."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2003_08374_gb300.build import build_library
    build_library()


def test_non_finite_pressure_is_reported_as_diverged():
    from paper_2003_08374_gb300 import mdbs
    from paper_2003_08374_gb300 import workloads as W
    case = W.fracture_2d(nx=16, ny=12)
    s = mdbs.Simulation(case)
    p = case.p.copy()
    p[7] = np.nan
    with pytest.raises(mdbs.MdbsError) as e:
        s.set_fields(case.alpha, case.ux, case.uy, case.uz, p)
    assert e.value.code == mdbs.ERR_DIVERGED
    with pytest.raises(mdbs.MdbsError) as e:
        s.step(1)
    assert e.value.code == mdbs.ERR_DIVERGED
    # a finite state makes the simulation usable again
    s.set_fields(case.alpha, case.ux, case.uy, case.uz, case.p)
    s.step(2)
    assert s.stats()["steps"] == 2


def test_max_cg_reached_is_reported_as_not_converged():
    from paper_2003_08374_gb300 import mdbs
    from paper_2003_08374_gb300 import workloads as W
    case = W.grf_3d(shape=(16, 16, 16), seed=2, corr_len=4.0, frac_w=2, p_tol=1e-12, max_cg=2)
    s = mdbs.Simulation(case)
    with pytest.raises(mdbs.MdbsError) as e:
        s.step(3)
    assert e.value.code == mdbs.ERR_NOT_CONVERGED
    st = s.stats()
    assert st["steps"] == 3 and st["not_converged"] == 3 * case.n_corr
    assert all(it == 2 for it in st["cg_iters"]) and max(st["cg_resid"]) > 1e-12
    # the same case with room to converge reports nothing
    ok = mdbs.Simulation(case.replace(max_cg=200))
    ok.step(3)
    assert ok.stats()["not_converged"] == 0


def test_batch_reports_the_member_that_did_not_converge():
    from paper_2003_08374_gb300 import mdbs
    from paper_2003_08374_gb300 import workloads as W
    a = mdbs.Simulation(W.darcy_domain((12, 10, 8), seed=1, p_tol=1e-12, max_cg=3))
    b = mdbs.Simulation(W.darcy_domain((9, 9, 1), seed=2, p_tol=1e-12, max_cg=3))
    bt = mdbs.Batch([a, b])
    with pytest.raises(mdbs.MdbsError) as e:
        bt.step(1)
    assert e.value.code == mdbs.ERR_NOT_CONVERGED
    bt.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_checkpoint_restart_is_bitwise(precision):
    from paper_2003_08374_gb300 import mdbs
    from paper_2003_08374_gb300 import workloads as W
    case = W.grf_3d(shape=(18, 14, 12), seed=3, corr_len=3.0, frac_w=2, p_tol=1e-10, precision=precision)
    straight = mdbs.Simulation(case)
    straight.step(8)
    a = mdbs.Simulation(case)
    a.step(4)
    f = a.fields()
    a.close()
    b = mdbs.Simulation(case)
    b.set_fields(f["alpha"], f["ux"], f["uy"], f["uz"], f["p"])
    b.step(4)
    fs, fb = straight.fields(), b.fields()
    for n in fs:
        assert np.array_equal(fs[n], fb[n]), n


def test_alpha_range_new_input_and_round_trip():
    from paper_2003_08374_gb300 import mdbs
    from paper_2003_08374_gb300 import workloads as W
    case = W.fracture_2d(nx=12, ny=10)
    s = mdbs.Simulation(case)
    a = case.alpha.copy()
    a[4] = 1.0 + 1e-8
    with pytest.raises(mdbs.MdbsError) as e:
        s.set_fields(a, case.ux, case.uy, case.uz, case.p)
    assert e.value.code == mdbs.ERR_ARG
    a[4] = 1.0 + 5e-10  # round-off of an earlier computation
    s.set_fields(a, case.ux, case.uy, case.uz, case.p)
    # a loosely solved run drifts outside [0, 1]; its own state must survive a round trip
    run = mdbs.Simulation(W.grf_3d(shape=(16, 14, 12), seed=4, corr_len=3.0, frac_w=2, p_tol=1e-6, max_cg=50,
                                   precision=1))
    run.step(30)
    st = run.stats()
    f = run.fields()
    run.set_fields(f["alpha"], f["ux"], f["uy"], f["uz"], f["p"])
    assert run.stats()["alpha_min"] == st["alpha_min"] and run.stats()["alpha_max"] == st["alpha_max"]
