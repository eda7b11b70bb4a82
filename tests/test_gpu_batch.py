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


def test_members_join_and_leave_between_steps():
    """mdbs_batch_add / mdbs_batch_remove (continuous batching): a member's results do not
    depend on when others join or leave, and a removed member steps alone again."""
    from paper_2003_08374_gb300 import mdbs
    cases = _cases(0)[:4]
    ref = []
    for c in cases:
        s = mdbs.Simulation(c)
        s.step(6)
        ref.append(s.fields())
        s.close()
    sims = [mdbs.Simulation(c) for c in cases]
    b = mdbs.Batch(sims[:2])
    b.step(2)                      # members 0, 1 at 2 steps
    sims[2].step(2)                # member 2 alone to 2 steps, then joins
    b.add(sims[2])
    b.step(2)                      # 0, 1, 2 at 4 steps
    b.remove(sims[0])
    sims[0].step(2)                # 0 alone to 6
    b.add(sims[3])                 # 3 joins at 0 steps
    b.step(2)                      # 1, 2 at 6; 3 at 2
    b.remove(sims[3])
    sims[3].step(4)                # 3 alone to 6
    for s, fa in zip(sims, ref):
        assert s.stats()["steps"] == 6
        fb = s.fields()
        for k in fa:
            assert np.array_equal(fa[k], fb[k]), k
    with pytest.raises(mdbs.MdbsError):
        b.add(sims[1])             # already a member
    with pytest.raises(mdbs.MdbsError):
        b.remove(sims[0])          # not a member
    b.remove(sims[1])
    with pytest.raises(mdbs.MdbsError):
        b.remove(sims[2])          # the last member stays
    b.close()


def test_allocator_hook_serves_the_arenas():
    """mdbs_set_allocator with PyTorch's caching allocator: the arenas come from torch
    (its allocated bytes grow by mdbs_bytes_required and fall back at destroy), and the
    results equal those of cudaMalloc'ed arenas."""
    torch = pytest.importorskip("torch")
    from paper_2003_08374_gb300 import mdbs
    from paper_2003_08374_gb300 import workloads as W
    case = W.grf_3d(shape=(20, 18, 16), seed=3, corr_len=3.0, frac_w=2, p_tol=1e-10, max_cg=300)
    s = mdbs.Simulation(case)
    s.step(3)
    ref = s.fields()
    s.close()
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    mdbs.use_torch_allocator()
    try:
        t = mdbs.Simulation(case)
        held = torch.cuda.memory_allocated() - base
        assert held >= mdbs.bytes_required(case)
        t.step(3)
        f = t.fields()
        for k in ref:
            assert np.array_equal(ref[k], f[k]), k
        t.close()
        torch.cuda.synchronize()
        assert torch.cuda.memory_allocated() == base
    finally:
        mdbs.set_allocator()
