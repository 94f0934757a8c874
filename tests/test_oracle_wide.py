"""4-wide traversal in the oracle: the collapse keeps every binary child
slot exactly once, and the traversal's hits equal brute force and the
binary traversal's, culled or not, with culled counts <= plain."""
import numpy as np
import pytest

import oracle
from paper_2305_08343_gb300 import scenegen as sg


def test_collapse_covers_every_slot_once(hair_small):
    tris, _ = hair_small
    ob = oracle.OracleBVH(tris)
    w = ob.wide()
    assert np.all((w["n"] >= 2) & (w["n"] <= 4))
    ex_child, ex_count = ob_children(ob)
    seen = set()
    for q in range(len(w["n"])):
        for i in range(w["n"][q]):
            p, c = int(w["parent"][q, i]), int(w["child"][q, i])
            seen.add((p, c))
            inner = ex_count[p, c] == 0
            assert (w["next"][q, i] > q) == inner and (w["next"][q, i] < 0) == (not inner)
    # the binary nodes that become 4-wide nodes: the root and every inner
    # 4-wide child; their inner slots are pulled up (replaced by the two
    # slots below them), every other binary slot is a 4-wide child once
    made = {0} | {int(ex_child[p, c]) for (p, c) in seen if ex_count[p, c] == 0}
    pulled = {(n, c) for n in made for c in (0, 1) if ex_count[n, c] == 0}
    all_slots = {(p, c) for p in range(len(ex_count)) for c in (0, 1)}
    assert seen | pulled == all_slots and not (seen & pulled)


def ob_children(ob):
    n = ob.num_nodes
    child = np.zeros((n, 2), np.int32)
    count = np.zeros((n, 2), np.int32)
    box = np.zeros((n, 2, 6), np.float32)
    oracle.lib().or_bvh_nodes(ob._h, oracle._ptr(child, oracle.C.c_int32),
                              oracle._ptr(count, oracle.C.c_int32),
                              oracle._ptr(box, oracle.C.c_float))
    return child, count


@pytest.mark.parametrize("cull", [0, 1, 2])
def test_wide_hits_equal_binary_and_brute_force(hair_small, cull):
    tris, rays = hair_small
    ob = oracle.OracleBVH(tris).build_masks(6, 3).compress(256, 8)
    two = ob.trace(rays, 0, cull)
    four = ob.trace(rays, 0, cull, width=4)
    assert np.array_equal(four["id"], two["id"]) and np.array_equal(four["t"], two["t"])
    plain4 = ob.trace(rays, 0, 0, width=4)
    assert (four["counts"] <= plain4["counts"]).all()
    assert four["counts"][:, 0].sum() > 0


def test_wide_soup_brute_force_and_any_hit():
    tris = sg.soup(3000, seed=21)
    rays = sg.random_rays(2000, seed=22)
    ob = oracle.OracleBVH(tris).build_masks(4, 3)
    t, hid, t2 = oracle.brute(tris, rays, 0)
    o = ob.trace(rays, 0, 1, width=4)
    assert np.array_equal(o["t"], t)
    ok = t2 != t
    assert np.array_equal(o["id"][ok], hid[ok])
    a = ob.trace(rays, 1, 1, width=4)
    assert np.array_equal(a["id"] >= 0, hid >= 0)


def test_wide_leaf_root_and_single_triangle():
    one = np.array([[0, 0, 0, 1, 0, 0, 0, 1, 0]], np.float32)
    ob = oracle.OracleBVH(one)
    rays = np.array([[0.2, 0.2, -1, 0, 0, 0, 1, np.inf], [2, 2, -1, 0, 0, 0, 1, np.inf]],
                    np.float32)
    o = ob.trace(rays, 0, 0, width=4)
    assert o["id"].tolist() == [0, -1] and o["counts"][:, 0].tolist() == [0, 0]
