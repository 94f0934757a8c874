"""Frontier and seeded traversal (learned proposal; not in the paper).

The seeded oracle is pinned to the plain oracle traversal (itself pinned to
brute force): for ANY class per ray -- random, out of range, the true
subtree -- its hits must be bit-identical, since the seed only changes t_max
and skips a subtree that phase 1 covered.  The product's frontier (host
code) must equal the oracle's."""
import numpy as np
import pytest

import oracle
from paper_2305_08343_gb300 import scenegen as sg
from paper_2305_08343_gb300 import subcull as sc


def _eq(a, b):
    return np.array_equal(np.asarray(a).view(np.int32), np.asarray(b).view(np.int32))


@pytest.fixture(scope="module")
def scene(hair_small):
    tris, rays = hair_small
    ob = oracle.OracleBVH(tris).build_masks(6, 3).compress(64, 8)
    return tris, rays, ob


@pytest.mark.parametrize("depth", [0, 1, 3, 8])
def test_frontier_partitions_triangles(scene, depth):
    tris, _, ob = scene
    fc, fn, fb, cls = ob.frontier(depth)
    assert 1 <= len(fc) <= 2 ** depth
    # every triangle belongs to exactly one frontier subtree; the subtree of
    # slot k holds exactly the triangles of class k, and they lie in its box
    counts = np.bincount(cls, minlength=len(fc))
    assert counts.sum() == len(tris) and np.all(counts > 0)
    v = tris.reshape(-1, 3, 3)
    lo = fb[cls][:, None, :3]
    hi = fb[cls][:, None, 3:]
    assert np.all(v >= lo) and np.all(v <= hi)
    if depth == 0:
        assert len(fc) == 1 and np.all(cls == 0)


@pytest.mark.parametrize("depth", [0, 2, 8])
def test_product_frontier_equals_oracle(scene, depth):
    tris, _, ob = scene
    fc, fn, fb, cls = ob.frontier(depth)
    b = sc.sc_bvh_build(tris, 6, 1)
    ent, pcls = sc.sc_bvh_frontier(b, depth)
    words = np.where(fn > 0, 0x80000000 | ((fn.astype(np.int64) - 1) << 28) | fc,
                     fc).astype(np.uint32)
    assert np.array_equal(ent[:, 6].view(np.uint32), words)
    assert np.all(ent[:, 7].view(np.uint32) == 0)
    assert _eq(ent[:, :6], fb)
    assert np.array_equal(pcls, cls)


@pytest.mark.parametrize("cull", [0, 1, 2])
def test_seeded_hits_equal_plain_for_any_class(scene, cull):
    tris, rays, ob = scene
    pl = ob.trace(rays, 0, cull)
    fc, fn, fb, cls = ob.frontier(8)
    rng = np.random.default_rng(5)
    true = np.where(pl["id"] >= 0, cls.astype(np.int32)[np.maximum(pl["id"], 0)], -1)
    for c in (rng.integers(-2, len(fc) + 2, len(rays)).astype(np.int32),
              true.astype(np.int32), np.zeros(len(rays), np.int32)):
        sd = ob.trace_seeded(rays, c, 8, cull=cull)
        assert _eq(sd["id"], pl["id"]) and _eq(sd["t"], pl["t"]) and _eq(sd["uv"], pl["uv"])
    # no seed at all: exactly the plain traversal, counts included
    sd = ob.trace_seeded(rays, np.full(len(rays), -1, np.int32), 8, cull=cull)
    assert np.array_equal(sd["counts"], pl["counts"])


def test_seeded_ties_keep_traversal_order():
    # Two triangles in the plane z = 0 with different centroids, so they sit
    # in different subtrees; rays through their overlap hit both at exactly
    # t = 1.  The seeded traversal must keep the one the plain traversal
    # meets first, whichever subtree the seed names.
    small = np.array([[-1, -1, 0, 1, -1, 0, 0, 1, 0]], np.float32)
    big = np.array([[-3, -1.5, 0, 3, -1.5, 0, 0, 6, 0]], np.float32)
    far = sg.soup(64, seed=9) + np.float32(5.0)
    tris = np.concatenate([small, far, big]).astype(np.float32)
    ob = oracle.OracleBVH(tris, max_leaf=1)
    rays = np.array([[0.1 * i, 0.05, -1, 0, 0, 0, 1, np.inf] for i in range(-4, 5)], np.float32)
    pl = ob.trace(rays, 0, 0)
    assert np.all(pl["t"] == 1.0)
    fc, fn, fb, cls = ob.frontier(3)
    assert cls[0] != cls[len(tris) - 1]  # the tie spans two subtrees
    for k in range(-1, len(fc)):
        sd = ob.trace_seeded(rays, np.full(len(rays), k, np.int32), 3, cull=0)
        assert _eq(sd["id"], pl["id"]) and _eq(sd["t"], pl["t"])


def test_seeded_depth_and_degenerate(scene):
    tris, rays, ob = scene
    pl = ob.trace(rays[:512], 0, 1)
    for depth in (0, 1, 5):
        fc = ob.frontier(depth)[0]
        c = np.arange(512, dtype=np.int32) % (len(fc) + 1)
        sd = ob.trace_seeded(rays[:512], c, depth, cull=1)
        assert _eq(sd["id"], pl["id"]) and _eq(sd["t"], pl["t"])
    one = oracle.OracleBVH(tris[:1])
    r = rays[:64]
    p1 = one.trace(r, 0, 0)
    s1 = one.trace_seeded(r, np.zeros(64, np.int32), 8, cull=0)
    assert _eq(s1["id"], p1["id"]) and _eq(s1["t"], p1["t"])
