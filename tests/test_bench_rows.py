"""Bench arithmetic that needs no GPU: the per-level HBM rows (algorithmic
bytes over the timed launch, flags for L2-resident launches, the rows of
launches that take several right-hand sides together) on a stand-in solver
with fixed sizes and times."""
import pytest

import bench


class FakeSolver:
    """Two levels of 2^21 and 2^20 cells and a small third; every kernel
    takes 100 us, level 1 is a cell-tile level, level 0 a brick level."""

    def __init__(self):
        self.calls = []

    def num_levels(self):
        return 3

    def level_sizes(self, l):
        return [(1 << 21, 1000, 4000), (1 << 20, 800, 3000), (1 << 10, 0, 0)][l]

    def stored_coefficients(self, l):
        return [1 << 21, 15 << 20, 27 << 10][l]

    def level_tile(self, l):
        return (4, 1 if l == 0 else 0)

    def time_kernel(self, kid, level, reps, stream):
        self.calls.append((kid, level))
        return 100.0


def test_hbm_rows_bytes_and_together_rows():
    sv = FakeSolver()
    out = bench.hbm_by_level(sv, "w", None, 1000.0, min_cells=1 << 20, nrhs=4)
    rows = {r["level"]: r for r in out["levels"]}
    assert sorted(rows) == [0, 1]                 # level 2 is below min_cells
    w, N1, sc1 = 4, 1 << 20, 15 << 20
    # one right-hand side: coefficients and three / four vectors
    assert rows[1]["residual"]["gbs"] == pytest.approx(w * (sc1 + 3 * N1) / 100e-6 / 1e9, rel=1e-3)
    assert rows[1]["relax"]["frac"] == pytest.approx(w * (sc1 + 4 * N1) / 100e-6 / 1e9 / 1000.0,
                                                     abs=1e-3)
    # together: the coefficients once, the vectors four times, per-side time
    tog = rows[1]["residual_rhs_together"]
    assert tog["rhs"] == 4 and tog["us_per_rhs"] == 25.0
    assert tog["gbs"] == pytest.approx(w * (sc1 + 3 * N1 * 4) / 100e-6 / 1e9, rel=1e-3)
    # the brick level has no together rows, and level 0 alone times the
    # pre-relaxation (level 1's is done by the restriction onto it)
    assert "residual_rhs_together" not in rows[0] and "relax0_u" in rows[0]
    assert "relax0_u" not in rows[1]
    assert (11, 1) in sv.calls and (12, 1) in sv.calls and (11, 0) not in sv.calls
    # launches moving less than ~3/4 of L2 are flagged
    assert rows[1]["restrict"].get("l2_resident") is True


def test_hbm_rows_single_rhs_has_no_together_rows():
    sv = FakeSolver()
    out = bench.hbm_by_level(sv, "w", None, 1000.0)
    assert all(not k.endswith("_together") for r in out["levels"] for k in r)
    assert all(kid < 11 for kid, _ in sv.calls)
