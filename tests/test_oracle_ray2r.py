"""The ray-mask table at R_ray = 2R (Sec. 4.2): begin and end cells on the 2R
grid, each row an R^3-bit mask that sets a mask cell iff the sweep test on the
2R grid sets one of its eight sub-cells.  Pinned against:

* a direct scan of the definition -- every sub-cell, t on an exact rational
  grid fine enough to land inside any feasible open interval -- on whole small
  tables and sampled rows of the R = 4 and R = 6 tables;
* containment: the 2R sweep between two sub-cells lies inside the R sweep
  between their enclosing cells, so a 2R row lies inside that R row;
* conservativeness: every R cell a segment passes through is in the row of
  the 2R cells of its ends;
* the 2R cell of a point: its enclosing R cell is the R-table cell, and away
  from cell borders it is the point's 2R-grid coordinate rounded down;
* traversal: with the 2R table culled hits equal plain hits, no ray needs
  more tests than with the R table, and ideal culling needs no more in total.
"""
import numpy as np
import pytest

import oracle


def _bits(rows, R):
    """bool[rows, R^3] from uint32[rows, W] masks."""
    b = np.unpackbits(np.ascontiguousarray(rows).view(np.uint8), axis=1, bitorder="little")
    return b[:, : R ** 3].astype(bool)


def _scan_row(R, b2, e2):
    """The definition on the 2R grid by a scan of t = k / M, folded to R."""
    R2 = 2 * R
    M = 2 * (R2 - 1) ** 2 + 1
    k = np.arange(M + 1)
    v = np.arange(R2)
    ok = [np.abs(M * (b2[a] - v)[:, None] + k[None, :] * (e2[a] - b2[a])) < M for a in range(3)]
    sub = (ok[0][None, None, :, :] & ok[1][None, :, None, :] & ok[2][:, None, None, :]).any(-1)
    z, y, x = np.nonzero(sub)  # sub[z, y, x]
    out = np.zeros(R ** 3, bool)
    out[(x // 2) + R * (y // 2) + R * R * (z // 2)] = True
    return out


def _cells(idx, n):
    return np.stack([idx % n, (idx // n) % n, idx // (n * n)], axis=-1)


@pytest.mark.parametrize("R,nrows", [(2, None), (4, 400), (6, 120)])
def test_rows_match_a_scan_of_the_definition(R, nrows):
    lut = oracle.raylut2r(R)
    R23 = (2 * R) ** 3
    rng = np.random.default_rng(R)
    rows = np.arange(R23 * R23) if nrows is None else rng.integers(0, R23 * R23, nrows)
    got = _bits(lut[rows], R)
    for i, row in enumerate(rows):
        b2, e2 = _cells(np.array([row // R23, row % R23]), 2 * R)
        assert np.array_equal(got[i], _scan_row(R, b2, e2)), (R, row)


@pytest.mark.parametrize("R", [4, 6])
def test_rows_lie_inside_the_R_rows_of_the_enclosing_cells(R):
    lut2, lut1 = oracle.raylut2r(R), oracle.raylut(R)
    R2, R3, R23 = 2 * R, R ** 3, (2 * R) ** 3
    rows = np.arange(R23 * R23) if R == 4 else \
        np.random.default_rng(11).integers(0, R23 * R23, 200000)
    b2, e2 = _cells(rows // R23, R2), _cells(rows % R23, R2)
    b1, e1 = b2 // 2, e2 // 2
    beg = b1[:, 0] + R * b1[:, 1] + R * R * b1[:, 2]
    end = e1[:, 0] + R * e1[:, 1] + R * R * e1[:, 2]
    inner, outer = lut2[rows], lut1[beg * R3 + end]
    assert not (inner & ~outer).any()
    # and it is tighter somewhere
    assert (inner != outer).any()
    # a segment inside one 2R cell sets just the R cell around it
    same = rows[rows // R23 == rows % R23]
    one = _bits(lut2[same], R).sum(1)
    assert (one == 1).all()


@pytest.mark.parametrize("R", [4, 6])
def test_every_cell_a_segment_crosses_is_in_its_row(R):
    lut = oracle.raylut2r(R)
    R2, R23 = 2 * R, (2 * R) ** 3
    rng = np.random.default_rng(100 + R)
    t = np.linspace(0.0, 1.0, 3001)
    for _ in range(400):
        # ends in R-grid coordinates; short and long segments
        p0 = rng.uniform(0, R, 3)
        p1 = p0 + rng.normal(0, rng.choice([0.3, 2.0]), 3)
        p1 = np.clip(p1, 0, R - 1e-9)
        b2, e2 = np.floor(2 * p0).astype(int), np.floor(2 * p1).astype(int)
        row = _bits(lut[[(b2[0] + R2 * b2[1] + R2 * R2 * b2[2]) * R23
                         + e2[0] + R2 * e2[1] + R2 * R2 * e2[2]]], R)[0]
        pts = p0[None, :] + t[:, None] * (p1 - p0)[None, :]
        c = np.clip(np.floor(pts).astype(int), 0, R - 1)
        crossed = np.unique(c[:, 0] + R * c[:, 1] + R * R * c[:, 2])
        assert row[crossed].all()


@pytest.mark.parametrize("R", [4, 6])
def test_cell2_encloses_in_the_R_cell_and_rounds_down(R):
    rng = np.random.default_rng(5)
    for _ in range(3000):
        lo = float(rng.uniform(-2, 2))
        hi = lo + float(rng.choice([1e-3, 0.5, 3.0]))
        o, d = float(rng.uniform(-4, 4)), float(rng.normal())
        t = float(rng.uniform(-1, 3))
        c1 = oracle.cell_at(t, o, d, lo, hi, R)
        c2 = oracle.cell2_at(t, o, d, lo, hi, R)
        assert 0 <= c2 < 2 * R and c2 // 2 == c1
        f1 = oracle.cell_t(t, o, d, lo, hi, R)
        f2 = oracle.cell2_t(t, o, d, lo, hi, R)
        assert 0 <= f2 < 2 * R and f2 // 2 == f1
        u = 2 * R * ((o + t * d) - lo) / (hi - lo)
        if abs(u - round(u)) > 1e-3:
            assert c2 == int(np.clip(np.floor(u), 0, 2 * R - 1))


@pytest.mark.parametrize("R", [4, 6])
def test_traversal_with_the_2R_table(hair_small, R):
    tris, rays = hair_small
    plain = oracle.OracleBVH(tris).trace(rays, 0, 0)
    ob = oracle.OracleBVH(tris).build_masks(R, 3)
    lut = ob.trace(rays, 0, 1)
    lut2 = ob.set_ray2r().trace(rays, 0, 1)
    ideal = ob.set_ray2r(False).set_ideal().trace(rays, 0, 1)
    ob.set_ideal(False)
    for o in (lut, lut2, ideal):
        assert np.array_equal(o["id"], plain["id"]) and np.array_equal(o["t"], plain["t"])
    tot = {k: int(o["counts"].astype(np.int64).sum()) for k, o in
           (("plain", plain), ("lut", lut), ("lut2", lut2), ("ideal", ideal))}
    # every 2R test culls at least what the R test culls, so no ray does more
    assert (lut2["counts"] <= lut["counts"]).all()
    assert tot["ideal"] <= tot["lut2"] < tot["lut"] < tot["plain"]
    # any hit keeps a real hit
    anyh = ob.set_ray2r().trace(rays, 1, 1)
    ob.set_ray2r(False)
    assert np.array_equal(anyh["id"] >= 0, plain["id"] >= 0)
