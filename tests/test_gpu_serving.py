"""Continuous batching: requests admitted as they arrive and as memory frees up run
in a changing batch; each request's result must equal its result alone."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2003_08374_gb300.build import build_library
    build_library()


class VirtualClock:
    """Deterministic clock: every reading advances 5 ms."""

    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 0.005
        return self.t


def _trace(precision=0):
    from paper_2003_08374_gb300.serve import Request, fractured_request_case
    specs = [(0.00, 16, 1e-4, 7), (0.00, 20, 1e-3, 3), (0.02, 12, 3e-3, 9), (0.05, 24, 1e-5, 6),
             (0.05, 16, 5e-4, 4), (0.30, 18, 2e-3, 5)]
    reqs = []
    for rid, (t, side, ca, steps) in enumerate(specs):
        case = fractured_request_case(side, ca, seed=100 + rid, precision=precision, p_tol=1e-10, max_cg=300)
        reqs.append(Request(rid=rid, arrival=t, case=case, steps=steps))
    return reqs


@pytest.mark.parametrize("precision", [0, 1])
def test_results_same_alone_and_in_the_mix(precision):
    from paper_2003_08374_gb300 import mdbs
    from paper_2003_08374_gb300.serve import Server
    reqs = _trace(precision)
    srv = Server(max_active=4, round_steps=2)
    summary = srv.run(reqs, clock=VirtualClock())
    assert summary["completed"] == len(reqs) and summary["batch_rebuilds"] >= 3
    assert summary["p99_latency_s"] >= summary["p50_latency_s"] > 0
    for r in reqs:
        s = mdbs.Simulation(r.case)
        s.step(r.steps)
        alone = s.fields()
        for k in alone:
            assert np.array_equal(alone[k], r.result[k]), (r.rid, k)
        assert r.stats["steps"] == r.steps


def test_admission_waits_for_memory():
    from paper_2003_08374_gb300 import mdbs
    from paper_2003_08374_gb300.serve import Server
    reqs = _trace()
    need = max(mdbs.bytes_required(r.case) for r in reqs)
    # pretend the device only has room for two of the largest requests beside the reserve
    srv = Server(max_active=16, round_steps=3, reserve_bytes=0, free_bytes_fn=lambda: int(2.5 * need))
    summary = srv.run(reqs, clock=VirtualClock())
    assert summary["completed"] == len(reqs)
    assert srv.peak_active <= 2
