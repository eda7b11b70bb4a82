"""mdbs_field_stats_static: the allocation-free statistics entry point.

Some callers cannot let the library allocate device memory (code running while
a CUDA graph is captured, serving loops that must not trigger the device-wide
synchronisation of an allocation, embedders that own all device memory).  This
test calls the allocation-free entry point through the C-ABI on caller-owned
device buffers and checks, on two calls in a row, that it reports what the
regular path (mdbs_set_fields -> mdbs_get_stats) reports for the same fields.
It lives in its own file so that it runs last."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_field_stats_static_matches_regular_stats():
    torch = pytest.importorskip("torch")
    from paper_2003_08374_gb300.build import build_library
    build_library()
    from paper_2003_08374_gb300 import mdbs
    from paper_2003_08374_gb300 import workloads as W

    lib = mdbs.lib()
    stream = torch.cuda.current_stream()
    # 40x33x17 and 64x48: fewer blocks than the scratch holds; 64^3 (262144 cells, 1024
    # blocks of work): the grid is capped at MDBS_STATIC_STATS_MAX_BLOCKS and every block
    # strides over several chunks
    for shape, seed in (((40, 33, 17), 3), ((64, 48, 1), 4), ((64, 64, 64), 5)):
        case = W.darcy_domain(shape, seed=seed)
        rng = np.random.default_rng(seed)
        case.alpha = rng.uniform(0.0, 1.0, case.cells)
        sim = mdbs.Simulation(case)
        ref = sim.stats()
        sim.close()
        dev = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
        phi, alpha, p = dev(case.porosity), dev(case.alpha), dev(case.p)
        for _ in range(2):  # two calls in a row share the static scratch
            out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
            rc = lib.mdbs_field_stats_static(case.cells, case.h ** 3, C.c_void_p(phi.data_ptr()),
                                             C.c_void_p(alpha.data_ptr()), C.c_void_p(p.data_ptr()),
                                             C.c_void_p(out.data_ptr()), C.c_void_p(stream.cuda_stream))
            assert rc == mdbs.OK
            torch.cuda.synchronize()
            vol, amin, amax, bad = out.cpu().numpy()
            assert vol == pytest.approx(ref["mass"], rel=1e-12)
            assert amin == ref["alpha_min"] and amax == ref["alpha_max"]
            assert bad == 0.0
    # one non-finite pressure in the last cell of the 64^3 case (handled by the last block's
    # last stride) is counted once, the other statistics are unchanged
    p_bad = p.clone()
    p_bad[-1] = float("inf")
    out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
    rc = lib.mdbs_field_stats_static(case.cells, case.h ** 3, C.c_void_p(phi.data_ptr()),
                                     C.c_void_p(alpha.data_ptr()), C.c_void_p(p_bad.data_ptr()),
                                     C.c_void_p(out.data_ptr()), C.c_void_p(stream.cuda_stream))
    assert rc == mdbs.OK
    torch.cuda.synchronize()
    vol, amin, amax, bad = out.cpu().numpy()
    assert bad == 1.0 and vol == pytest.approx(ref["mass"], rel=1e-12)
    # sizes beyond the stated maximum are rejected before any device work
    rc = lib.mdbs_field_stats_static(2 ** 31, 1.0, C.c_void_p(phi.data_ptr()), C.c_void_p(alpha.data_ptr()),
                                     C.c_void_p(p.data_ptr()), C.c_void_p(out.data_ptr()), None)
    assert rc == mdbs.ERR_ARG
