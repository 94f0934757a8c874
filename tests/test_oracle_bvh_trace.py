"""Pins of the oracle's BVH (binned SAH, Sec. 4) and traversal (Alg. 4 with
Alg. 1, culling of Sec. 3.1.2).

Independent facts: brute force over all ray x triangle pairs (closest hit),
closed-form ray-triangle and ray-box results, structural validity of the
tree, the paper's conservativeness claim (culling never removes a true hit,
Sec. 3.1.1 / 3.2.3) and its consequence on counts, and dense sampling of the
clipped segment against the looked-up ray mask.
"""
import numpy as np
import pytest

import oracle
from paper_2305_08343_gb300 import scenegen as sg


def _tri_boxes(tris):
    v = tris.reshape(-1, 3, 3)
    return v.min(1), v.max(1)


def test_bvh_structure(hair_small):
    tris, _ = hair_small
    b = oracle.OracleBVH(tris)
    child, count, box = b.nodes()
    perm = b.perm()
    assert sorted(perm.tolist()) == list(range(len(tris)))
    assert (count <= 4).all()
    lo, hi = _tri_boxes(tris)
    seen = np.zeros(len(tris), int)
    order = []
    # pre-order walk: nodes appear as 0, 1, 2, ...
    stack = [0]
    while stack:
        n = stack.pop()
        order.append(n)
        for c in (1, 0):
            if count[n, c] == 0:
                assert child[n, c] > n
                stack.append(int(child[n, c]))
    assert order == list(range(b.num_nodes))
    for n in range(b.num_nodes):
        for c in range(2):
            if count[n, c] > 0:
                ids = perm[child[n, c]:child[n, c] + count[n, c]]
                seen[ids] += 1
                exp_lo, exp_hi = lo[ids].min(0), hi[ids].max(0)
            else:
                m = child[n, c]
                exp_lo = np.minimum(box[m, 0, :3], box[m, 1, :3])
                exp_hi = np.maximum(box[m, 0, 3:], box[m, 1, 3:])
            assert np.array_equal(box[n, c, :3], exp_lo) and np.array_equal(box[n, c, 3:], exp_hi)
    assert (seen == 1).all()
    # Eq. 1 cost is finite and better than a single big leaf
    assert b.sah() < len(tris)


def test_sah_separates_clusters():
    # two clusters of 8 triangles far apart: the root split separates them
    rng = np.random.default_rng(0)
    a = rng.uniform(0, 1, (8, 9)).astype(np.float32)
    bb = (rng.uniform(0, 1, (8, 9)) + 100).astype(np.float32)
    tris = np.vstack([bb[:4], a, bb[4:]])
    b = oracle.OracleBVH(tris)
    child, count, box = b.nodes()
    perm = b.perm()

    def leaves(n, c):
        if count[n, c] > 0:
            return list(perm[child[n, c]:child[n, c] + count[n, c]])
        m = child[n, c]
        return leaves(m, 0) + leaves(m, 1)
    left, right = set(leaves(0, 0)), set(leaves(0, 1))
    cl_a = set(range(4, 12))
    assert left == cl_a or right == cl_a


def test_ray_triangle_closed_form():
    tri = np.array([0, 0, 0, 1, 0, 0, 0, 1, 0], np.float32)
    ray = np.array([0.25, 0.25, 1, 0, 0, 0, -1, np.inf], np.float32)
    ok, t, u, v = oracle.ray_tri(ray, tri)
    assert ok and t == 1.0 and u == 0.25 and v == 0.25
    ray2 = np.array([0.75, 0.75, 1, 0, 0, 0, -1, np.inf], np.float32)   # outside
    assert not oracle.ray_tri(ray2, tri)[0]
    ray3 = np.array([0.5, 0.5, 1, 0, 0, 0, -1, np.inf], np.float32)     # on edge u+v=1
    assert oracle.ray_tri(ray3, tri)[0]
    assert not oracle.ray_tri(ray, tri, tcur=1.0)[0]                     # strict t < tcur
    ray4 = np.array([0.25, 0.25, 1, 1.0, 0, 0, -1, np.inf], np.float32)  # tmin = 1
    assert not oracle.ray_tri(ray4, tri)[0]


def test_slab_closed_form():
    box = np.array([1, 1, 1, 2, 2, 2], np.float32)
    ray = np.array([0, 1.5, 1.5, 0, 1, 0, 0, np.inf], np.float32)
    ok, tn, tf = oracle.slab(ray, box)
    assert ok and tn == 1.0 and tf == 2.0
    ok, tn, tf = oracle.slab(ray, box, tcur=0.5)
    assert not ok
    ray_in = np.array([1.5, 1.5, 1.5, 0, 0, 0, 1, np.inf], np.float32)
    ok, tn, tf = oracle.slab(ray_in, box)
    assert ok and tn == 0.0 and tf == 0.5


@pytest.mark.parametrize("R", [4, 6, 8])
def test_traversal_cell_is_alg1_exactly(R):
    """The culling test's cell (or_cell_at, the traversal's default) is Alg. 1
    applied to the point p = o + t d formed in float32 (a product, then a
    sum): it equals or_cell of that point on every sample, with no
    tolerance.  numpy's float32 scalar arithmetic forms p independently."""
    rng = np.random.default_rng(3 + R)
    for _ in range(20000):
        lo, hi = np.sort(rng.uniform(-2, 2, 2)).astype(np.float32)
        if rng.random() < 0.05:
            hi = lo  # flat box: the extent floor of 1e-30
        o, d = np.float32(rng.uniform(-3, 3)), np.float32(rng.normal())
        t = np.float32(rng.uniform(0, 4))
        p = np.float32(o + np.float32(t * d))
        assert oracle.cell_at(t, o, d, lo, hi, R) == oracle.cell(p, lo, hi, R)


def test_fused_cell_option_differs_only_at_cell_borders():
    """The fused form (an option of the traversal, or_cell_t) evaluates the
    same coordinate with one rounding; it may differ from Alg. 1 only where
    the exact coordinate lies within rounding of a cell border."""
    rng = np.random.default_rng(3)
    diff = 0
    for _ in range(20000):
        lo, hi = np.sort(rng.uniform(-2, 2, 2)).astype(np.float32)
        o, d, t = np.float32(rng.uniform(-3, 3)), np.float32(rng.normal()), np.float32(rng.uniform(0, 4))
        a, b = oracle.cell_at(t, o, d, lo, hi, 6), oracle.cell_t(t, o, d, lo, hi, 6)
        if a != b:
            q = (float(o) + float(t) * float(d) - float(lo)) * 6 / (float(hi) - float(lo))
            assert abs(q - round(q)) < 1e-4
            diff += 1
    assert diff < 20


def test_cell_index_alg1():
    # Alg. 1: floor(R/extent * (p - lower)), clamped to [0, R-1]
    assert oracle.cell(0.0, 0.0, 1.0, 4) == 0
    assert oracle.cell(0.25, 0.0, 1.0, 4) == 1
    assert oracle.cell(0.999, 0.0, 1.0, 4) == 3
    assert oracle.cell(1.0, 0.0, 1.0, 4) == 3      # min(., R-1)
    assert oracle.cell(-1e-7, 0.0, 1.0, 4) == 0    # clamp at 0
    assert oracle.cell(5.0, 5.0, 5.0, 6) == 0      # flat box


def _check_against_brute(tris, rays, near_tie_rel=1e-6):
    """Closest hits equal brute force: t on every ray, the triangle id on
    every ray without an exact tie (equal t, where brute force takes the
    lowest index and traversal the first met).  Rays whose second-closest
    hit lies within near_tie_rel of the closest are listed separately."""
    b = oracle.OracleBVH(tris)
    o = b.trace(rays, 0, 0)
    bt, bid, t2 = oracle.brute(tris, rays, 0)
    assert np.array_equal(o["t"], bt)
    with np.errstate(invalid="ignore"):
        near = (t2 - bt) <= near_tie_rel * np.abs(bt)
    exact = (t2 == bt) & (bid >= 0)
    diff = o["id"] != bid
    assert not (diff & ~exact).any(), "hit id differs on a ray without an exact tie"
    print(f"\n{len(rays)} rays: {int(near.sum())} near-tie (second hit within "
          f"{near_tie_rel:g}), {int(exact.sum())} exact ties, {int(diff.sum())} ids differ "
          f"(exact ties only): rays {np.nonzero(near)[0][:10].tolist()}")
    return b, o


def test_plain_traversal_equals_brute_force_hair(hair_small):
    tris, rays = hair_small
    _check_against_brute(tris, rays)


def test_plain_traversal_equals_brute_force_soup():
    tris = sg.soup(4096, seed=21)
    rays = sg.random_rays(4096, seed=22)
    b, o = _check_against_brute(tris, rays)
    assert (o["id"] >= 0).sum() > 10


def test_plain_traversal_equals_brute_force_ground():
    tris = sg.hair(64, 16, True, seed=23)
    rays = sg.pinhole(48, 32)
    b, o = _check_against_brute(tris, rays)
    assert (o["id"] == len(tris) - 1).any() or (o["id"] == len(tris) - 2).any()


@pytest.mark.parametrize("R,L", [(4, 3), (6, 3), (6, 1), (8, 3)])
def test_culling_keeps_hits_and_reduces_counts(hair_small, R, L):
    tris, rays = hair_small
    b = oracle.OracleBVH(tris).build_masks(R, L=L).compress(256, 8)
    plain = b.trace(rays, 0, 0)
    for cull in (1, 2):
        o = b.trace(rays, 0, cull)
        assert np.array_equal(o["id"], plain["id"])
        assert np.array_equal(o["t"], plain["t"])
        assert (o["counts"] <= plain["counts"]).all()
    unc = b.trace(rays, 0, 1)
    assert unc["counts"].sum() < plain["counts"].sum()


def test_culling_keeps_hits_soup_bounce_like():
    tris = sg.soup(8192, seed=31)
    rays = sg.random_rays(8192, seed=32)
    b = oracle.OracleBVH(tris).build_masks(6, L=3).compress(256, 8)
    plain = b.trace(rays, 0, 0)
    for cull in (1, 2):
        o = b.trace(rays, 0, cull)
        assert np.array_equal(o["id"], plain["id"]) and np.array_equal(o["t"], plain["t"])
        assert (o["counts"] <= plain["counts"]).all()


def test_any_hit_consistency():
    tris = sg.soup(4096, seed=41)
    rays = sg.random_rays(2048, seed=42)
    b = oracle.OracleBVH(tris).build_masks(6, L=3)
    cl = b.trace(rays, 0, 0)
    for cull in (0, 1):
        an = b.trace(rays, 1, cull)
        assert np.array_equal(an["id"] >= 0, cl["id"] >= 0)
        hit = cl["id"] >= 0
        assert (an["t"][hit] >= cl["t"][hit]).all()
        assert (an["counts"] <= cl["counts"]).all() if cull == 0 else True


def test_edge_cases():
    # empty scene
    rays = sg.pinhole(8, 4)
    b = oracle.OracleBVH(np.zeros((0, 9), np.float32))
    o = b.trace(rays)
    assert (o["id"] == -1).all() and np.isinf(o["t"]).all() and (o["counts"] == 0).all()
    # one triangle: the root is a leaf (no box test)
    tri = np.array([[-1, -1, 0, 1, -1, 0, 0, 1, 0]], np.float32)
    b = oracle.OracleBVH(tri)
    assert b.num_nodes == 0
    o = b.trace(rays)
    assert (o["counts"][:, 0] == 0).all() and (o["counts"][:, 1] == 1).all()
    assert (o["id"] == 0).any()
    # identical triangles (no SAH split possible): median split, all found
    tris = np.tile(tri, (9, 1))
    b = oracle.OracleBVH(tris)
    assert b.num_nodes >= 2
    o = b.trace(rays)
    bt, bid, _ = oracle.brute(tris, rays)
    assert np.array_equal(o["t"], bt)


@pytest.mark.parametrize("form", [0, 1])
def test_ray_mask_covers_sampled_segment(form):
    """C9: for random boxes and rays, every densely sampled point of the true
    clipped segment lies within a small distance of a cell set in the ray
    mask looked up from the float segment ends (Alg. 1 as written, form 0,
    and the fused option, form 1)."""
    R = 6
    lut = oracle.raylut(R)
    bits = np.unpackbits(lut.view(np.uint8), axis=1, bitorder="little")[:, : R ** 3].astype(bool)
    rng = np.random.default_rng(5)
    checked = 0
    for _ in range(4000):
        lo = rng.uniform(-1, 1, 3).astype(np.float32)
        hi = (lo + rng.uniform(0.01, 1, 3)).astype(np.float32)
        o = rng.uniform(-2, 2, 3)
        tgt = lo + rng.uniform(0, 1, 3) * (hi - lo)
        d = tgt - o
        d /= np.linalg.norm(d)
        ray = np.array([*o, 0, *d, np.inf], np.float32)
        ok, tn, tf = oracle.slab(ray, np.concatenate([lo, hi]))
        if not ok:
            continue
        cell = oracle.cell_t if form else oracle.cell_at
        cb = [cell(tn, ray[k], ray[4 + k], lo[k], hi[k], R) for k in range(3)]
        ce = [cell(tf, ray[k], ray[4 + k], lo[k], hi[k], R) for k in range(3)]
        row = (cb[0] + R * cb[1] + R * R * cb[2]) * R ** 3 + (ce[0] + R * ce[1] + R * R * ce[2])
        m = bits[row].reshape(R, R, R)  # [z, y, x]
        od, dd = ray[:3].astype(np.float64), ray[4:7].astype(np.float64)
        ts = np.linspace(tn, tf, 64)
        ext = (hi.astype(np.float64) - lo) / R
        tol = 1e-5 * ext
        for t in ts:
            p = od + t * dd
            rngs = []
            for k in range(3):
                a = int(np.clip(np.floor((p[k] - tol[k] - lo[k]) / ext[k]), 0, R - 1))
                z = int(np.clip(np.floor((p[k] + tol[k] - lo[k]) / ext[k]), 0, R - 1))
                rngs.append(range(a, z + 1))
            assert any(m[z, y, x] for x in rngs[0] for y in rngs[1] for z in rngs[2])
        checked += 1
    assert checked > 1000


def test_dense_mask_skip_keeps_hits_and_orders_counts(hair_small):
    """Skipping the test for dense masks only keeps children: hits are the
    same for every threshold, counts lie between the fully tested culled
    traversal and the plain one, and fewer masks are tested."""
    tris, rays = hair_small
    b = oracle.OracleBVH(tris).build_masks(6, L=3).compress(256, 8)
    plain = b.trace(rays, 0, 0)
    for cull in (1, 2):
        full = b.trace(rays, 0, cull)
        prev = full
        for skip in (180, 144, 100, 36, 0):
            o = b.trace(rays, 0, cull, skip_bits=skip)
            assert np.array_equal(o["id"], plain["id"]) and np.array_equal(o["t"], plain["t"])
            assert (o["counts"] >= full["counts"]).all() and (o["counts"] <= plain["counts"]).all()
            assert o["mask_tests"].sum() <= prev["mask_tests"].sum()
            prev = o
        assert prev["mask_tests"].sum() == 0 and np.array_equal(prev["counts"], plain["counts"])
        for stride in (2, 3):
            o = b.trace(rays, 0, cull, stride=stride)
            assert np.array_equal(o["id"], plain["id"]) and np.array_equal(o["t"], plain["t"])
            assert (o["counts"] >= full["counts"]).all() and (o["counts"] <= plain["counts"]).all()
        prev = full
        for leaf_min in (2, 3, 4, 5):
            o = b.trace(rays, 0, cull, leaf_min=leaf_min)
            assert np.array_equal(o["id"], plain["id"]) and np.array_equal(o["t"], plain["t"])
            assert (o["counts"] >= full["counts"]).all() and (o["counts"] <= plain["counts"]).all()
            assert o["mask_tests"].sum() <= prev["mask_tests"].sum()
            # nodes are culled the same way; only leaf triangles can be added
            assert np.array_equal(o["counts"][:, 0], full["counts"][:, 0])
            prev = o


def test_exact_and_near_ties_against_brute_force():
    """A duplicated triangle (exact tie: any of the two is right) and a copy
    moved about one float step (2.5e-7 at t = 3) along the ray: a near tie
    that is not exact, so the closer copy must win."""
    base = sg.hair(64, 16, False, seed=29)
    tri = np.array([[-0.5, -0.5, 0.0, 0.5, -0.5, 0.0, 0.0, 0.5, 0.0]], np.float32)
    near = tri.copy()
    near[0, 2::3] += np.float32(2.5e-7)  # z of the three vertices
    tris = np.concatenate([base, tri, tri, near]).astype(np.float32)
    rays = np.zeros((64, 8), np.float32)
    g = np.linspace(-0.2, 0.2, 8, dtype=np.float32)
    rays[:, 0] = np.repeat(g, 8)
    rays[:, 1] = np.tile(g, 8)
    rays[:, 2] = 3.0
    rays[:, 6] = -1.0           # towards -z
    rays[:, 7] = np.inf
    b, o = _check_against_brute(tris, rays)
    n = len(base)
    on = (o["id"] >= n)
    assert on.sum() > 40
    # the moved copy is closer to rays coming from +z: it is the hit
    assert (o["id"][on] == n + 2).all()
    # without it, the two copies tie exactly: either is right
    b2, o2 = _check_against_brute(tris[:-1], rays)
    assert np.isin(o2["id"][on], [n, n + 1]).all()
