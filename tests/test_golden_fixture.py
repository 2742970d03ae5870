"""The paper's printed iteration counts (tests/golden/paper_iteration_counts.txt) are well formed
and consistent with the paper's own statements about them (CPU only)."""
import os

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = {"Table1", "Table2", "Table3", "Table4", "Table6", "Table8", "Table9"}


def rows():
    path = os.path.join(HERE, "golden", "paper_iteration_counts.txt")
    return [l.split() for l in open(path) if l.strip() and not l.startswith("#")]


def test_rows_are_well_formed():
    rs = rows()
    assert len(rs) >= 50
    for r in rs:
        assert len(r) == 10, r
        src, case, kn, M, order, slope, grid, solver, printed, tol = r
        assert src in SOURCES and case in {"lid", "eslid", "four", "heated"}
        assert float(kn) > 0 and 3 <= int(M) <= 25 and int(order) in (1, 2) and int(slope) in (0, 1, 2)
        assert int(grid) in (32, 64, 128, 256) and solver in {"NMG", "FS", "Euler"} and int(printed) > 0
        assert tol == "-" or tol.endswith("%") or tol.isdigit(), r
        if tol != "-":
            assert int(M) <= 16  # the library's largest order


def test_printed_orderings_the_paper_states():
    """Per case, Euler needs more steps than FS and FS more than NMG cycles (Sec. 4: FS takes about
    1/8 of the Euler iterations, NMG a few percent of FS)."""
    by = {}
    for src, case, kn, M, order, slope, grid, solver, printed, tol in rows():
        by.setdefault((src, case, kn, M, order, grid), {})[solver] = int(printed)
    both = 0
    for key, d in by.items():
        if "Euler" in d and "FS" in d:
            assert 4 * d["FS"] < d["Euler"] < 12 * d["FS"], key
            both += 1
        if "FS" in d and "NMG" in d:
            assert d["NMG"] < d["FS"] / 10, key
    assert both >= 6


@pytest.mark.parametrize("src,grids", [("Table1", (32, 64, 128, 256)), ("Table2", (32, 64, 128, 256))])
def test_fs_and_euler_grow_with_the_grid_nmg_stays_flat(src, grids):
    d = {}
    for s, case, kn, M, order, slope, grid, solver, printed, tol in rows():
        if s == src:
            d[(solver, int(grid))] = int(printed)
    nmg = [d[("NMG", g)] for g in grids]
    assert max(nmg) <= 2 * min(nmg)
    eu = [d[("Euler", g)] for g in grids if ("Euler", g) in d]
    assert all(b > 1.7 * a for a, b in zip(eu, eu[1:]))
