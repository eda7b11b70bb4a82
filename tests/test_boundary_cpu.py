"""CPU checks of the C-ABI boundary: the library loads, exports every entry
point that include/mdbs.h declares, and its ctypes binding agrees with the
header's struct layouts.  No CUDA call is made."""
import ctypes as C
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mdbs.h")


@pytest.fixture(scope="module")
def built():
    from paper_2003_08374_gb300.build import build_library
    return build_library()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mdbs_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_function(built):
    names = declared_functions()
    assert "mdbs_step" in names and len(names) >= 10
    out = subprocess.run(["nm", "-D", "--defined-only", built], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (mdbs_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    lib = C.CDLL(built)
    for n in names:
        getattr(lib, n)


def test_binding_struct_layouts_match_header(built):
    from paper_2003_08374_gb300 import mdbs
    structs = {"mdbs_grid": mdbs.Grid, "mdbs_fluids": mdbs.Fluids, "mdbs_closures": mdbs.Closures,
               "mdbs_options": mdbs.Options, "mdbs_stats": mdbs.Stats, "mdbs_tuning": mdbs.Tuning}
    prog = '#include <stdio.h>\n#include <stddef.h>\n#include "mdbs.h"\nint main(void){\n'
    for s, cls in structs.items():
        prog += 'printf("%s %%zu\\n", sizeof(%s));\n' % (s, s)
        for f, _ in cls._fields_:
            prog += 'printf("%s.%s %%zu\\n", offsetof(%s, %s));\n' % (s, f, s, f)
    prog += "return 0;}\n"
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(prog)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    got = dict(l.split() for l in out.strip().splitlines())
    for s, cls in structs.items():
        assert int(got[s]) == C.sizeof(cls), s
        for f, _ in cls._fields_:
            assert int(got["%s.%s" % (s, f)]) == getattr(cls, f).offset, (s, f)


def test_bytes_required_is_host_only_and_monotone(built):
    from paper_2003_08374_gb300 import mdbs
    from paper_2003_08374_gb300 import workloads as W
    a = mdbs.bytes_required(W.Case(name="a", nx=32, ny=32, nz=32, h=1e-5))
    b = mdbs.bytes_required(W.Case(name="b", nx=64, ny=64, nz=64, h=1e-5))
    assert 0 < a < b
    assert b / (64 ** 3) < 1200  # device bytes per cell
    # mixed precision adds the FP32 hierarchy; BF16 coarse coefficients take 2 bytes, not 4
    g = W.Case(name="c", nx=64, ny=64, nz=64, h=1e-5)
    f64, f32, bf = (mdbs.bytes_required(g, precision=p) for p in (0, 1, 2))
    coarse = sum((64 >> l) ** 3 for l in range(1, 5))  # levels 32^3 .. 4^3
    assert f64 < f32 and f32 - bf >= 0.99 * 3 * 2 * coarse  # (less 256-byte alignment of the small levels)


def test_allocator_hook_and_batch_membership_argument_errors(built):
    """Host-only checks (no device call): exactly one NULL allocator function, and NULL
    batch or simulation handles, are argument errors; both NULL restores cudaMalloc."""
    from paper_2003_08374_gb300 import mdbs
    L = mdbs.lib()
    assert L.mdbs_set_allocator(mdbs.ALLOC_FN(lambda n, c: None), mdbs.FREE_FN(), None) == mdbs.ERR_ARG
    assert L.mdbs_set_allocator(mdbs.ALLOC_FN(), mdbs.FREE_FN(lambda p, c: None), None) == mdbs.ERR_ARG
    assert L.mdbs_set_allocator(mdbs.ALLOC_FN(), mdbs.FREE_FN(), None) == mdbs.OK
    assert L.mdbs_batch_add(None, None) == mdbs.ERR_ARG
    assert L.mdbs_batch_remove(None, None) == mdbs.ERR_ARG
