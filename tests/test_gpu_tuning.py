"""Execution schedules of the multigrid kernels (mdbs_tuning) and the autotuner.
A schedule changes only which launches update which cells and in which order the
CTAs walk them, never a value: fields must be bitwise identical under every
schedule, and autotuning must leave the simulation exactly where it was."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

def _sch(rows, tail, snake, kz, ctas, coop, vec=0):
    return {"smooth_rows": rows, "tail_cells": tail, "snake": snake, "sweep_kz": kz, "tail_ctas": ctas,
            "coarse_coop": coop, "vec_sweeps": vec}


SCHEDULES = [
    _sch(1, 4096, 0, 0, 1, 0, 0),  # default
    _sch(1, 4096, 0, 0, 1, 0, 1),  # vector half sweeps where aligned
    _sch(1, 4096, 0, 0, 1, 1),     # levels 1-2 and the tail in one cooperative launch
    _sch(1, 0, 1, 0, 1, 1, 1),     # vector sweeps where aligned, cooperative down to the coarsest level
    _sch(1, 4096, 1, 8, 1, 0, 1),  # fused sweeps (FP32) with vector sweeps elsewhere
    _sch(8, 4096, 1, 8, 1, 0),     # fused sweeps
    _sch(2, 0, 1, 0, 2, 0),        # coarsest only in the tail, 2 CTAs
    _sch(2, 0, 1, 0, 1, 1),        # cooperative down to the coarsest level
    _sch(4, 512, 0, 4, 4, 0),      # 37 planes: ragged chunks
    _sch(8, 0, 1, 32, 1, 0),       # fused down to 4x3x3
    _sch(8, 32768, 1, 16, 1, 0),   # all but level 0, one CTA
    _sch(1, 262144, 0, 0, 8, 0),   # all but level 0, cluster
    _sch(1, 262144, 0, 0, 1, 1),   # all but level 0: nothing for the cooperative launch (no effect)
]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2003_08374_gb300.build import build_library
    build_library()


def _case(precision):
    from paper_2003_08374_gb300 import workloads as W
    # ragged sizes: levels 61x47x37 -> 31x24x19 -> 16x12x10 -> 8x6x5 -> 4x3x3
    return W.grf_3d(shape=(61, 47, 37), seed=5, corr_len=4.0, frac_w=3, p_tol=1e-10, max_cg=300,
                    precision=precision)


def _run(case, schedule, steps=3):
    from paper_2003_08374_gb300 import mdbs
    s = mdbs.Simulation(case)
    if schedule is not None:
        s.set_tuning(schedule)
        assert s.tuning() == schedule
    s.step(steps)
    out = s.fields(), s.stats()
    s.close()
    return out


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_fields_bitwise_identical_under_every_schedule(precision):
    case = _case(precision)
    ref_f, ref_s = _run(case, None)
    assert ref_s["cg_iters_total"] > 0
    for sch in SCHEDULES:
        f, st = _run(case, sch)
        for k in ref_f:
            assert np.array_equal(ref_f[k], f[k]), (sch, k)
        assert st["cg_iters"] == ref_s["cg_iters"], sch


def test_invalid_schedules_are_rejected():
    from paper_2003_08374_gb300 import mdbs
    s = mdbs.Simulation(_case(0))
    for bad in ({"smooth_rows": 3, "tail_cells": 4096, "snake": 1, "sweep_kz": 8},
                {"smooth_rows": 8, "tail_cells": 300000, "snake": 1, "sweep_kz": 8},
                {"smooth_rows": 8, "tail_cells": -1, "snake": 1, "sweep_kz": 8},
                {"smooth_rows": 8, "tail_cells": 4096, "snake": 2, "sweep_kz": 8},
                {"smooth_rows": 8, "tail_cells": 4096, "snake": 1, "sweep_kz": 6},
                {"smooth_rows": 8, "tail_cells": 4096, "snake": 1, "sweep_kz": 8, "tail_ctas": 3},
                {"smooth_rows": 8, "tail_cells": 4096, "snake": 1, "sweep_kz": 8, "tail_ctas": 16},
                _sch(1, 4096, 0, 0, 1, 2)):
        with pytest.raises(mdbs.MdbsError) as e:
            s.set_tuning(bad)
        assert e.value.code == mdbs.ERR_ARG
    # still usable with the schedule it had
    assert s.tuning() == SCHEDULES[0]
    s.step(1)
    s.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_autotune_leaves_the_simulation_where_it_was(precision):
    from paper_2003_08374_gb300 import mdbs
    case = _case(precision)
    a = mdbs.Simulation(case)
    a.step(1)
    before = a.stats()
    chosen, trials = a.autotune(trial_steps=1)
    assert a.stats() == before
    # initial, snake, sweep_kz (mixed only), smooth_rows (split sweeps only), tail_cells
    assert len(trials) >= 1 + 1 + 3 + 3 and all(t > 0 for t in trials)
    assert chosen == a.tuning()
    assert chosen["smooth_rows"] in (1, 2, 4, 8) and chosen["snake"] in (0, 1)
    a.step(2)
    b = mdbs.Simulation(case)
    b.step(3)
    fa, fb = a.fields(), b.fields()
    for k in fa:
        assert np.array_equal(fa[k], fb[k]), k
    sa, sb = a.stats(), b.stats()
    for k in ("steps", "time", "cg_iters", "cg_iters_total", "mass"):
        assert sa[k] == sb[k], k
    a.close()
    b.close()


def test_batch_schedule_and_autotune_keep_members_identical():
    from paper_2003_08374_gb300 import mdbs
    from paper_2003_08374_gb300 import workloads as W
    cases = [W.darcy_domain((33, 17, 9), seed=21, p_tol=1e-10, max_cg=300),
             W.darcy_domain((40, 24, 1), seed=22, p_tol=1e-10, max_cg=300),
             _case(0)]
    alone = []
    for c in cases:
        s = mdbs.Simulation(c)
        s.step(3)
        alone.append(s.fields())
        s.close()
    sims = [mdbs.Simulation(c) for c in cases]
    b = mdbs.Batch(sims)
    b.set_tuning(_sch(1, 0, 0, 0, 1, 1))
    b.step(1)
    chosen, trials = b.autotune(trial_steps=1)
    assert chosen == b.tuning() and len(trials) >= 5
    b.step(2)
    for s, fa in zip(sims, alone):
        fb = s.fields()
        for k in fa:
            assert np.array_equal(fa[k], fb[k]), k
        assert s.stats()["steps"] == 3
    b.close()


@pytest.mark.parametrize("precision", [1, 2])
def test_fused_sweeps_with_tma_staging_are_bitwise_equal(precision):
    """Levels whose x extent is a multiple of 8 stage their planes with TMA box copies of
    the even and the odd cells (120 = 2 x 56 + 8: a ragged last tile; the 60- and
    30-cell levels use per-element copies); the fields must equal the split sweeps'."""
    from paper_2003_08374_gb300 import workloads as W
    case = W.grf_3d(shape=(120, 52, 20), seed=9, corr_len=4.0, frac_w=3, p_tol=1e-10, max_cg=300,
                    precision=precision)
    ref_f, ref_s = _run(case, _sch(1, 4096, 0, 0, 1, 0))
    for kz in (4, 8, 32):
        f, st = _run(case, _sch(1, 0, 0, kz, 1, 0))
        for k in ref_f:
            assert np.array_equal(ref_f[k], f[k]), (kz, k)
        assert st["cg_iters"] == ref_s["cg_iters"]


def test_bounded_wait_gives_up_and_the_device_stays_usable():
    """The fused sweeps' mbarrier waits have a time limit: a wait that nothing completes
    returns after about a second with an error status, and work runs afterwards."""
    from paper_2003_08374_gb300 import mdbs
    waited = mdbs.check_bounded_wait()
    assert 0.9 <= waited <= 5.0
    s = mdbs.Simulation(_case(1))
    s.step(1)
    assert s.stats()["steps"] == 1
    s.close()


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_vector_half_sweeps_are_bitwise_equal(precision):
    """Vector half sweeps (2 FP64 / 4 FP32 consecutive cells of a colour run per thread,
    16-byte loads) on every level whose n_x allows them: 40 x 23 x 19 (levels with n_x 40,
    20, 10, 5: the vector path where n_x is a multiple of 4 or 8, the scalar one
    elsewhere, ragged y and z) and 72 x 30 x 17, with and without the single-CTA tail;
    the fields must equal the scalar sweeps'."""
    from paper_2003_08374_gb300 import workloads as W
    for shape in ((40, 23, 19), (72, 30, 17)):
        case = W.grf_3d(shape=shape, seed=4, corr_len=4.0, frac_w=3, p_tol=1e-10, max_cg=300, precision=precision)
        ref_f, ref_s = _run(case, _sch(1, 0, 0, 0, 1, 0, 0))
        for sch in (_sch(1, 0, 0, 0, 1, 0, 1), _sch(1, 4096, 1, 0, 1, 0, 1), _sch(1, 0, 0, 0, 1, 1, 1)):
            f, st = _run(case, sch)
            for k in ref_f:
                assert np.array_equal(ref_f[k], f[k]), (shape, sch, k)
            assert st["cg_iters"] == ref_s["cg_iters"]


@pytest.mark.parametrize("precision", [0, 1])
def test_graph_step_equals_eager_step(precision):
    """The captured step runs the pressure operator's assembly, hierarchy and coarsest
    inverse on a side branch beside the momentum Jacobi sweeps; eager steps (profiling)
    run the same kernels in line.  A missing dependency between the branches would show
    as a difference: fields and CG iteration counts must be bitwise equal."""
    from paper_2003_08374_gb300 import mdbs
    from paper_2003_08374_gb300 import workloads as W
    case = W.grf_3d(shape=(40, 36, 32), seed=5, corr_len=3.0, frac_w=2, p_tol=1e-10, max_cg=300,
                    precision=precision)
    g = mdbs.Simulation(case)
    e = mdbs.Simulation(case)
    e.profile(True)
    for _ in range(3):
        g.step(2)
        e.step(2)
        assert g.stats()["cg_iters"] == e.stats()["cg_iters"]
    fg, fe = g.fields(), e.fields()
    for k in fg:
        assert np.array_equal(fg[k], fe[k]), k
    assert e.profile_read()["coarsen"][1] > 0  # the eager steps did run the in-line build
    g.close()
    e.close()
