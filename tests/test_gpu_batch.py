"""Batched execution: many uneven domains advanced with one launch per step phase.
Each member's fields must be identical (bitwise) alone and in the batch, and the
batch must respect each member's own convergence."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2003_08374_gb300.build import build_library
    build_library()


def _cases(precision):
    from paper_2003_08374_gb300 import workloads as W
    shapes = [(17, 23, 1), (9, 7, 6), (32, 32, 32), (40, 24, 1), (13, 9, 11), (5, 4, 3), (64, 8, 1)]
    cases = [W.darcy_domain(sh, seed=10 + i, p_tol=1e-10, max_cg=300, precision=precision)
             for i, sh in enumerate(shapes)]
    cases.append(W.grf_3d(shape=(20, 18, 16), seed=3, corr_len=3.0, frac_w=2, p_tol=1e-10, max_cg=300,
                          precision=precision))
    return cases


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_members_identical_alone_and_batched(precision):
    from paper_2003_08374_gb300 import mdbs
    cases = _cases(precision)
    alone = []
    for c in cases:
        s = mdbs.Simulation(c)
        s.step(4)
        alone.append((s.fields(), s.stats()))
        s.close()
    sims = [mdbs.Simulation(c) for c in cases]
    b = mdbs.Batch(sims)
    for _ in range(2):
        b.step(2)
    for s, (fa, sa) in zip(sims, alone):
        fb, sb = s.fields(), s.stats()
        for k in fa:
            assert np.array_equal(fa[k], fb[k]), k
        assert sb["cg_iters"] == sa["cg_iters"] and sb["steps"] == 4
    b.close()
    # released members step alone again
    sims[0].step(1)


def test_batch_rejects_mixed_solver_options_and_double_membership():
    from paper_2003_08374_gb300 import mdbs
    from paper_2003_08374_gb300 import workloads as W
    a = mdbs.Simulation(W.darcy_domain((8, 8, 1), seed=1))
    c = mdbs.Simulation(W.darcy_domain((8, 8, 1), seed=2, n_corr=3))
    with pytest.raises(mdbs.MdbsError):
        mdbs.Batch([a, c])
    b = mdbs.Batch([a])
    with pytest.raises(mdbs.MdbsError):
        mdbs.Batch([a])
    with pytest.raises(mdbs.MdbsError):
        a.step(1)
    b.close()
    a.step(1)
