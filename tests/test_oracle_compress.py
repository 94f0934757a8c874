"""Pins of the oracle's mask compression (Sec. 3.2.2 compression LUT, Sec.
3.2.3 requirement LUTs and Alg. 3).

Independent facts: the paper's own naive comparator (Table 3: brute-force
search for the tightest superset), numpy brute force over the table, the
table counts printed in Sec. 3.2.3 / 4.4, and hand-made importance cases.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2305_08343_gb300 import scenegen as sg

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")))


def _bits(m, R):
    return np.unpackbits(np.ascontiguousarray(m).view(np.uint8), axis=-1,
                         bitorder="little")[..., : R ** 3].astype(bool)


def _pack(bits):
    R3 = bits.shape[-1]
    W = (R3 + 31) // 32
    pad = np.zeros(bits.shape[:-1] + (W * 32,), bool)
    pad[..., :R3] = bits
    return np.packbits(pad, axis=-1, bitorder="little").view(np.uint32)


def _random_masks(R, n, rng):
    # sparse, structured masks (boxes and lines) like real object masks
    R3 = R ** 3
    out = np.zeros((n, R3), bool)
    g = np.arange(R)
    z, y, x = np.meshgrid(g, g, g, indexing="ij")
    x, y, z = x.ravel(), y.ravel(), z.ravel()
    for i in range(n):
        lo = rng.integers(0, R, 3)
        hi = np.minimum(lo + rng.integers(0, 3, 3), R - 1)
        out[i] = (x >= lo[0]) & (x <= hi[0]) & (y >= lo[1]) & (y <= hi[1]) & (z >= lo[2]) & (z <= hi[2])
        out[i] |= rng.random(R3) < 0.03
    return out


@pytest.mark.parametrize("R", [4, 6])
def test_requirement_lut_count_matches_paper(R):
    b = GOLD["requirement_luts"]["b"]
    clut = _pack(np.ones((1, R ** 3), bool))
    req = oracle.req_luts(clut, R, b)
    assert req.shape[0] == GOLD["requirement_luts"][f"count_R{R}"]
    assert req.shape[1] == GOLD["requirement_luts"]["entries"]


def test_compression_ratio_matches_paper():
    c = GOLD["compression"]
    for R in (4, 6):
        assert (R ** 3) // (8 * c["index_bytes"]) == c[f"ratio_R{R}"]
    assert c["lut_size"] == 2 ** (8 * c["index_bytes"])


@pytest.mark.parametrize("R", [4, 6, 8])
def test_alg3_equals_naive_and_is_tightest(R):
    rng = np.random.default_rng(R)
    bits = _random_masks(R, 3000, rng)
    masks = _pack(bits)
    boxes = np.tile(np.array([0, 0, 0, 1, 1, 1], np.float32), (len(masks), 1))
    boxes[:, 3:] += rng.uniform(0, 2, (len(masks), 3)).astype(np.float32)
    clut, imp = oracle.clut_build(masks, boxes, R, 256)
    K = clut.shape[0]
    assert K == 256
    cb = _bits(clut, R)
    pop = cb.sum(1)
    assert (np.diff(pop) >= 0).all(), "table not sorted by popcount"
    assert cb[-1].all() or cb.all(1).any(), "all-ones entry missing"
    assert len({c.tobytes() for c in clut}) == K, "duplicate entries"
    req = oracle.req_luts(clut, R, 8)
    for i in range(0, len(masks), 3):
        j = oracle.encode(masks[i], req, R, 8)
        assert j == oracle.encode_naive(masks[i], clut, R)
        sup = (cb | ~bits[i]).all(1)            # entries containing the mask
        assert sup[j]                            # conservative
        assert pop[j] == pop[sup].min()          # tightest
        assert j == np.nonzero(sup)[0][0]        # first in popcount order


def test_importance_selection_small_case():
    """Importance SA * O_m / R^3 (Sec. 3.2.2, the per-node term of Eq. 2):
    with room for 2 masks + the all-ones entry the two largest win."""
    R = 4
    bits = np.zeros((5, 64), bool)
    bits[0, :1] = True          # pop 1
    bits[1, :2] = True          # pop 2
    bits[2, :3] = True          # pop 3
    bits[3, 10:14] = True       # pop 4
    bits[4, :2] = True          # same as mask 1 (importance adds up)
    masks = _pack(bits)
    unit = np.array([0, 0, 0, 1, 1, 1], np.float32)        # SA = 6
    boxes = np.tile(unit, (5, 1))
    boxes[3, 3:] = [0.5, 0.5, 0.5]                         # SA = 1.5
    clut, imp = oracle.clut_build(masks, boxes, R, 3)
    # importances: m0 6/64, m1 2*(12/64), m2 18/64, m3 6/64 -> m1 (24) and m2 (18)
    cb = _bits(clut, R)
    assert cb.shape[0] == 3
    assert np.array_equal(cb[0], bits[1]) and np.array_equal(cb[1], bits[2])
    assert cb[2].all()
    assert np.isclose(imp[0], 2 * 6 * 2 / 64) and np.isclose(imp[1], 6 * 3 / 64)


@pytest.mark.parametrize("R", [4, 6])
def test_bvh_compressed_superset(R):
    tris = sg.hair(64, 16, False, seed=9)
    b = oracle.OracleBVH(tris).build_masks(R, L=3).compress(256, 8)
    m = b.masks()
    clut, idx = b.clut()
    dec = clut[idx.astype(np.int64)]
    assert not (m & ~dec).any(), "decoded mask is not a superset"
    # the encoded entry is the tightest superset in the table
    cb = _bits(clut, R)
    mb = _bits(m, R).reshape(-1, R ** 3)
    pop = cb.sum(1)
    for s in range(0, mb.shape[0], 7):
        sup = (cb | ~mb[s]).all(1)
        assert pop[idx.reshape(-1)[s]] == pop[sup].min()
