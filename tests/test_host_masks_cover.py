"""Pins of the product's own object masks, without the oracle.

The product's triangle-voxel test (the SAT in csrc/host/mask_math.h) is the
same separating-axis test the oracle restates, so the tests that compare the
two builds cannot catch a mistake both share.  These tests check the masks
the library exports against facts of the geometry instead:

  * every densely sampled point of every triangle lies in a set voxel of
    every ancestor slot's mask (conservative voxelization, Sec. 3.1.1,
    through the Alg. 2 fill for ancestors more than L levels up);
  * each decoded compressed mask (LUT entry of the slot's index, Alg. 3)
    contains the slot's uncompressed mask.
"""
import numpy as np
import pytest

from paper_2305_08343_gb300 import scenegen as sg
from paper_2305_08343_gb300 import subcull as sc


def _scene():
    return np.concatenate([sg.hair(48, 16, True, seed=61), sg.soup(1500, seed=62)])


def _pairs(ex, ntri):
    """(node, child index, triangle id) for every slot and every triangle
    below it."""
    child, count, perm = ex["child"], ex["count"], ex["perm"]
    nn = len(child)
    parent = np.full(nn, -1, np.int64)
    pc = np.zeros(nn, np.int64)
    for n in range(nn):
        for c in range(2):
            if count[n, c] == 0:
                parent[child[n, c]] = n
                pc[child[n, c]] = c
    out = []
    for n in range(nn):
        for c in range(2):
            if count[n, c] > 0:
                ids = perm[child[n, c]:child[n, c] + count[n, c]]
                m, k = n, c
                while m >= 0:
                    out.extend((m, k, int(t)) for t in ids)
                    m, k = parent[m], pc[m]
    return np.array(out, np.int64)


def _samples(tri, s=6):
    a, b, c = tri.reshape(3, 3).astype(np.float64)
    pts = []
    for i in range(s + 1):
        for j in range(s + 1 - i):
            u, v = i / s, j / s
            pts.append(a + u * (b - a) + v * (c - a))
    return np.array(pts)


@pytest.mark.parametrize("R,L", [(4, 3), (6, 3), (6, 1), (8, 3)])
def test_product_masks_cover_every_triangle_in_every_ancestor(R, L):
    tris = _scene()
    ex = sc.sc_bvh_build(tris, R, 0, L=L).export()
    pairs = _pairs(ex, len(tris))
    assert len(pairs) > 20000
    bits = np.unpackbits(ex["masks"].view(np.uint8), axis=-1, bitorder="little")[..., : R ** 3]
    S = np.stack([_samples(t) for t in tris])  # [ntri, s, 3]
    node, ch, tid = pairs[:, 0], pairs[:, 1], pairs[:, 2]
    box = ex["box"][node, ch].astype(np.float64)  # [P, 6]
    lo, hi = box[:, None, :3], box[:, None, 3:]
    p = S[tid]  # [P, s, 3]
    ext = hi - lo
    flat = ext <= 0
    u = np.where(flat, 0.0, (p - lo) / np.where(flat, 1.0, ext) * R)
    tol = 1e-7 * R
    a = np.clip(np.floor(u - tol), 0, R - 1).astype(np.int64)
    b = np.clip(np.floor(u + tol), 0, R - 1).astype(np.int64)
    a = np.where(flat, 0, a)
    b = np.where(flat, R - 1, b)
    m = bits[node, ch].astype(bool)  # [P, R^3]
    ok = np.zeros(p.shape[:2], bool)
    for dz in range(R):
        for dy in range(R):
            for dx in range(R):
                inside = ((a[..., 0] <= dx) & (dx <= b[..., 0]) & (a[..., 1] <= dy)
                          & (dy <= b[..., 1]) & (a[..., 2] <= dz) & (dz <= b[..., 2]))
                ok |= inside & m[:, None, dx + R * dy + R * R * dz]
    bad = np.argwhere(~ok)
    assert len(bad) == 0, f"{len(bad)} samples uncovered, first (pair, sample) {bad[:3].tolist()}"


@pytest.mark.parametrize("R", [4, 6, 8])
def test_product_decoded_masks_contain_the_originals(R):
    tris = _scene()
    ex = sc.sc_bvh_build(tris, R, 1).export()
    dec = ex["clut"][ex["cidx"].astype(np.int64)]
    assert np.array_equal(dec & ex["masks"], ex["masks"])
