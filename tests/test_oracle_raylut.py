"""Pins of the oracle's ray-mask lookup table (Sec. 3.1.1, Alg. 1).

The table maps the discretised begin/end cells of a ray segment inside a box
to the cells the segment may cross; it is built with an AABB-AABB sweep test
"because the sweep represents all possible rays".  The oracle evaluates the
sweep condition exactly with rational interval arithmetic.  These tests pin
it to facts that do not come from the oracle itself:
  * brute force of the sweep over a grid of t fine enough to be exact,
  * real segments between random interior points of the two cells (every
    cell they cross must be in the mask: conservativeness),
  * a witness segment for every cell in the mask (tightness),
  * closed forms for the main diagonal and for axis-parallel sweeps,
  * symmetry and the bounding-box property.
"""
import numpy as np
import pytest

import oracle


def _cells(R):
    g = np.arange(R)
    z, y, x = np.meshgrid(g, g, g, indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel()], 1)  # index = x + R y + R^2 z


def _unpack(lut, R):
    R3 = R ** 3
    bits = np.unpackbits(lut.view(np.uint8), axis=1, bitorder="little")
    return bits[:, :R3].astype(bool)


def _brute(R):
    """Exact brute force of the sweep: t = k/M, M = 2(R-1)^2 + 1.  A non-empty
    feasible set either contains t = 0 or t = 1 or is an open interval whose
    ends are fractions with denominators <= R-1, hence of length
    >= 1/(R-1)^2 > 1/M, so it contains a grid point.  Integer arithmetic:
    |M(b - v) + k(e - b)| < M on every axis."""
    c = _cells(R)
    M = 2 * (R - 1) ** 2 + 1
    k = np.arange(M + 1)
    b = c[:, None, None, None, :]
    e = c[None, :, None, None, :]
    v = c[None, None, :, None, :]
    kk = k[None, None, None, :, None]
    ok = np.abs(M * (b - v) + kk * (e - b)) < M
    return ok.all(-1).any(-1).reshape(R ** 6, R ** 3)


@pytest.mark.parametrize("R", [2, 3, 4])
def test_lut_equals_brute_force(R):
    lut = _unpack(oracle.raylut(R), R)
    assert np.array_equal(lut, _brute(R))


@pytest.mark.parametrize("R", [4, 6, 8])
def test_diagonal_closed_form(R):
    # Sweep from cell (0,0,0) to (R-1,R-1,R-1): cell v is met iff some
    # s in [0, R-1] has |s - v_k| < 1 on all axes, i.e. max(v) - min(v) <= 1;
    # there are R + 6(R-1) = 7R - 6 such cells (22 at R = 4).
    lut = _unpack(oracle.raylut(R) if R <= 6 else _lut8(), R)
    R3 = R ** 3
    m = lut[0 * R3 + (R3 - 1)]
    c = _cells(R)
    expect = (c.max(1) - c.min(1)) <= 1
    assert np.array_equal(m, expect)
    assert m.sum() == 7 * R - 6
    if R == 4:
        assert m.sum() == 22


_LUT8 = None


def _lut8():
    global _LUT8
    if _LUT8 is None:
        _LUT8 = oracle.raylut(8)
    return _LUT8


@pytest.mark.parametrize("R", [4, 6])
def test_axis_parallel_and_point(R):
    lut = _unpack(oracle.raylut(R), R)
    R3 = R ** 3
    c = _cells(R)
    rng = np.random.default_rng(0)
    for _ in range(50):
        y, z = rng.integers(0, R, 2)
        b = 0 + R * y + R * R * z
        e = (R - 1) + R * y + R * R * z
        expect = (c[:, 1] == y) & (c[:, 2] == z)
        assert np.array_equal(lut[b * R3 + e], expect)
    # beg == end: the single cell
    for s in range(R3):
        row = lut[s * R3 + s]
        assert row.sum() == 1 and row[s]


@pytest.mark.parametrize("R", [4, 6])
def test_symmetry_endpoints_and_bbox(R):
    lut = _unpack(oracle.raylut(R), R)
    R3 = R ** 3
    L = lut.reshape(R3, R3, R3)
    assert np.array_equal(L, L.transpose(1, 0, 2))
    idx = np.arange(R3)
    assert L[idx[:, None], idx[None, :], idx[:, None]].all()  # beg set
    assert L[idx[:, None], idx[None, :], idx[None, :]].all()  # end set
    c = _cells(R)
    lo = np.minimum(c[:, None, :], c[None, :, :])
    hi = np.maximum(c[:, None, :], c[None, :, :])
    inside = ((c[None, None, :, :] >= lo[:, :, None, :])
              & (c[None, None, :, :] <= hi[:, :, None, :])).all(-1)
    assert not (L & ~inside).any()


@pytest.mark.parametrize("R", [4, 6])
def test_conservative_on_real_segments(R):
    """Every cell crossed by a segment between interior points of the begin
    and end cells is in the mask (the ray segment inside the box can start
    and end anywhere in those cells, Sec. 3.1.1)."""
    lut = _unpack(oracle.raylut(R), R)
    R3 = R ** 3
    rng = np.random.default_rng(1)
    n = 20000
    b = rng.integers(0, R, (n, 3))
    e = rng.integers(0, R, (n, 3))
    p0 = b + rng.uniform(1e-6, 1 - 1e-6, (n, 3))
    p1 = e + rng.uniform(1e-6, 1 - 1e-6, (n, 3))
    t = np.linspace(0.0, 1.0, 129)
    pts = p0[:, None, :] + t[None, :, None] * (p1 - p0)[:, None, :]
    cell = np.clip(np.floor(pts).astype(int), 0, R - 1)
    ci = cell[..., 0] + R * cell[..., 1] + R * R * cell[..., 2]
    row = (b[:, 0] + R * b[:, 1] + R * R * b[:, 2]) * R3 + (e[:, 0] + R * e[:, 1] + R * R * e[:, 2])
    assert lut[row[:, None], ci].all()


def test_tight_witness_segments():
    """Every cell in a mask is crossed, through its interior, by a segment
    joining interior points of the begin and end cells (R = 4, all pairs)."""
    R = 4
    R3 = R ** 3
    lut = _unpack(oracle.raylut(R), R)
    c = _cells(R).astype(np.float64)
    M = 2 * (R - 1) ** 2 + 1
    tg = np.arange(M + 1) / M
    for beg in range(R3):
        b = c[beg]
        for end in range(R3):
            e = c[end]
            vs = np.nonzero(lut[beg * R3 + end])[0]
            v = c[vs]                                       # (m, 3)
            pos = b[None, None, :] + tg[None, :, None] * (e - b)[None, None, :]
            ok = (np.abs(pos - v[:, None, :]) < 1).all(-1)  # (m, M+1)
            assert ok.any(1).all()
            ts = tg[ok.argmax(1)]
            cc = b[None, :] + ts[:, None] * (e - b)[None, :] - v
            lo = np.maximum(-0.5, -0.5 - cc)
            hi = np.minimum(0.5, 0.5 - cc)
            s = 0.5 * (lo + hi)
            p = b + 0.5 + s
            q = e + 0.5 + s
            w = p + ts[:, None] * (q - p)
            assert ((p > b) & (p < b + 1)).all() and ((q > e) & (q < e + 1)).all()
            assert ((w > v) & (w < v + 1)).all()


def test_single_cell_queries_match_table():
    R = 6
    lut = _unpack(oracle.raylut(R), R)
    rng = np.random.default_rng(2)
    for _ in range(200):
        b, e, v = rng.integers(0, R, (3, 3))
        row = (b[0] + R * b[1] + R * R * b[2]) * R ** 3 + (e[0] + R * e[1] + R * R * e[2])
        assert oracle.raylut_cell(R, b, e, v) == lut[row, v[0] + R * v[1] + R * R * v[2]]


def test_table_is_six_dimensional():
    import json, os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")))
    R = 4
    lut = oracle.raylut(R)
    # key = (beg cell xyz, end cell xyz): R^6 rows
    assert g["ray_lut_key_dims"]["dims"] == 6
    assert lut.shape[0] == R ** g["ray_lut_key_dims"]["dims"]
