"""Host arithmetic of bench.py's rooflines: the multigrid hierarchy it assumes, the
algorithmic bytes and FP64 instructions per V-cycle, and the roofline fraction of the
finest-level sweep from a kernel-time record.  The reported fractions are only as
right as these models, so each is checked against numbers worked out by hand."""
import pytest

import bench


def test_hierarchy_matches_the_solvers_rule():
    """Every axis longer than 4 cells is halved, rounding up (the oracle's and the
    library's rule): 128^3 down to 4^3, and a ragged grid with a short axis."""
    assert bench.level_sizes((128, 128, 128)) == [(128,) * 3, (64,) * 3, (32,) * 3, (16,) * 3, (8,) * 3, (4,) * 3]
    assert bench.level_sizes((9, 6, 3)) == [(9, 6, 3), (5, 3, 3), (3, 3, 3)]
    assert bench.level_sizes((64, 64, 1))[-1] == (4, 4, 1)


def test_vcycle_bytes_by_hand_for_a_two_level_grid():
    """8^3 over 4^3, FP64, split sweeps, nu = (2, 2): the finest level moves one
    zero-guess half sweep (1.5 w), six full ones (2 w + 3 w each), the prolonging one
    (5 w + w/8) and the restriction (5 w + w/8) per cell; the 64-cell coarsest level
    reads its dense inverse and b, writes x (N^2 + 2 N words)."""
    w = 8
    levels = bench.vcycle_bytes((8, 8, 8), w, {"sweep_kz": 0, "tail_cells": 512})
    per_cell = 1.5 * w + 6 * 5 * w + (5 * w + w / 8) + (5 * w + w / 8)
    assert levels[0] == (512, pytest.approx(512 * per_cell))
    assert levels[1] == (64, (64 * 64 + 2 * 64) * w)


def test_fp64_instructions_by_hand_for_a_two_level_grid():
    """8^3 over 4^3, nu = (2, 2): 256 cells updated per half sweep at 1 (zero guess),
    7 (six full) and 13 (prolonging) FP64 instructions, 9 per colour-0 cell of the
    restriction, and 64^2 for the coarsest dense product."""
    instr = bench.vcycle_fp64_instructions((8, 8, 8))
    assert instr[0] == 256 * (1 + 6 * 7 + 13) + 256 * 9
    assert instr[1] == 64 * 64


def test_sweep_roofline_fraction_from_a_kernel_record():
    """128^3, FP64, split sweeps: 7 timed half sweeps per V-cycle average
    (6 x 5 w + 1.5 w) / 7 words per cell; 70 launches in 1.4 ms is 20 us a launch."""
    cells = 128 ** 3
    prof = {bench.DOMINANT: (1.4, 70)}
    r = bench.roofline(prof, cells, 8, fp64=True, tuning={"sweep_kz": 0}, nu=(2, 2))
    alg = (6 * 5 * 8 + 1.5 * 8) / 7 * cells
    assert r["alg_bytes_per_launch"] == pytest.approx(alg)
    assert r["avg_us"] == pytest.approx(20.0)
    gbs = alg / 20e-6 / 1e9
    frac_hbm = r["frac"] if r["unit"] == "GB/s" else r["hbm"]["frac"]
    peak = r["peak"] if r["unit"] == "GB/s" else r["hbm"]["peak"]
    assert frac_hbm == pytest.approx(gbs / peak)
    assert r["alg_bytes_full_sweep"] == 5 * 8 * cells
