"""Refit for moved triangles (sc_bvh_refit; dynamic scenes, whose mask
updates the paper leaves to future work) against the oracle's refit
(OracleBVH.refit: every slot box recomputed from scratch as the union of the
triangle boxes below it, then the masks of every slot and, when compressed,
Alg. 3 for every slot against the kept LUT).  The product recomputes only
the slots above moved triangles, so equality also checks which slots it
marks.  Cases: one moved strand (the dilation eps unchanged), the whole
scene scaled (eps changes: every slot), no motion (nothing changes), and
boxes checked directly as unions of their subtree's triangle boxes; culled
traversal after a refit keeps every hit."""
import numpy as np
import pytest

import oracle
from paper_2305_08343_gb300 import scenegen as sg
from paper_2305_08343_gb300 import subcull as sc

STRANDS, SEGS = 300, 16


@pytest.fixture(scope="module")
def scene():
    return sg.hair(STRANDS, SEGS, True, seed=12)


def _move_strand(tris, k, off=(0.01, 0.0, -0.005)):
    t = tris.copy()
    per = 2 * SEGS
    t[k * per:(k + 1) * per] += np.tile(np.asarray(off, np.float32), 3)
    return t


def _oracle_refit(tris0, tris1, R, comp):
    ob = oracle.OracleBVH(tris0).build_masks(R, 3)
    if comp:
        ob.compress(256, 8)
    ob.refit(tris1).build_masks(R, 3)
    if comp:
        ob.reencode()
    return ob


def _same_as_oracle(b, ob, comp):
    ex = b.export()
    child, count, box = ob.nodes()
    assert np.array_equal(ex["child"], child) and np.array_equal(ex["count"], count)
    assert np.array_equal(ex["box"], box)
    assert np.array_equal(np.array(b.info().root_box[:], np.float32), ob.root()[2])
    assert np.array_equal(ex["masks"], ob.masks())
    assert b.info().eps == ob.eps
    if comp:
        clut, cidx = ob.clut()
        assert np.array_equal(ex["clut"], clut) and np.array_equal(ex["cidx"], cidx)


@pytest.mark.parametrize("R,comp", [(6, 0), (6, 1), (4, 1), (8, 0)])
def test_one_strand_moved(scene, R, comp):
    t1 = _move_strand(scene, 137)
    b = sc.sc_bvh_build(scene, R, comp)
    info = sc.sc_bvh_refit(b, t1)
    assert info.moved_tris == 2 * SEGS
    # only the slots above the strand's leaves: a small part of the tree
    assert 0 < info.dirty_nodes < b.info().num_nodes // 10
    _same_as_oracle(b, _oracle_refit(scene, t1, R, comp), comp)


@pytest.mark.parametrize("comp", [0, 1])
def test_scene_scaled_every_slot_recomputed(scene, comp):
    t1 = (scene * np.float32(1.5)).astype(np.float32)
    b = sc.sc_bvh_build(scene, 6, comp)
    info = sc.sc_bvh_refit(b, t1)
    assert info.moved_tris == len(scene) - np.all(scene == 0, axis=1).sum()
    assert info.dirty_nodes == b.info().num_nodes  # eps changed with the scene's extent
    _same_as_oracle(b, _oracle_refit(scene, t1, 6, comp), comp)


def test_no_motion_changes_nothing(scene):
    b = sc.sc_bvh_build(scene, 6, 1)
    before = b.export()
    info = sc.sc_bvh_refit(b, scene.copy())
    assert info.moved_tris == 0 and info.dirty_nodes == 0
    after = b.export()
    for k in before:
        assert np.array_equal(before[k], after[k]), k


def test_boxes_are_unions_of_their_triangles(scene):
    t1 = _move_strand(_move_strand(scene, 5, (0.2, -0.1, 0.05)), 250, (-0.03, 0.02, 0.0))
    b = sc.sc_bvh_build(scene, 0, 0)
    sc.sc_bvh_refit(b, t1)
    ex = b.export()
    lo = t1.reshape(-1, 3, 3).min(1)
    hi = t1.reshape(-1, 3, 3).max(1)

    def span(child, count):  # leaf positions below a slot
        if count > 0:
            return child, child + count
        a, _ = span(ex["child"][child, 0], ex["count"][child, 0])
        _, z = span(ex["child"][child, 1], ex["count"][child, 1])
        return a, z

    for n in range(len(ex["child"])):
        for c in range(2):
            a, z = span(ex["child"][n, c], ex["count"][n, c])
            ids = ex["perm"][a:z]
            want = np.concatenate([lo[ids].min(0), hi[ids].max(0)])
            assert np.array_equal(ex["box"][n, c], want)


def test_traversal_after_refit_keeps_hits(scene):
    t1 = _move_strand(scene, 40, (0.05, 0.02, 0.0))
    ob = _oracle_refit(scene, t1, 6, 0)
    rays = sg.pinhole(96, 64)
    culled = ob.trace(rays, 0, 1)
    _, ids, _ = oracle.brute(t1, rays, 0)
    plain = ob.trace(rays, 0, 0)
    assert np.array_equal(culled["id"], plain["id"]) and np.array_equal(culled["t"], plain["t"])
    assert np.array_equal(culled["id"] >= 0, ids >= 0)


def test_refit_errors(scene):
    b = sc.sc_bvh_build(scene, 6, 0)
    with pytest.raises(sc.SubcullError) as e:
        sc.sc_bvh_refit(b, scene[:-1])
    assert e.value.code == sc.SC_ERR_ARG
    bad = scene.copy()
    bad[3, 2] = np.inf
    with pytest.raises(sc.SubcullError) as e:
        sc.sc_bvh_refit(b, bad)
    assert e.value.code == sc.SC_ERR_ARG


def test_refit_then_checkpoint_round_trip(scene, tmp_path):
    t1 = _move_strand(scene, 77)
    b = sc.sc_bvh_build(scene, 6, 1)
    sc.sc_bvh_refit(b, t1)
    path = str(tmp_path / "refit.ckpt")
    sc.sc_bvh_save(b, path)
    c = sc.sc_bvh_load(path)
    ea, ec = b.export(), c.export()
    for k in ea:
        assert np.array_equal(ea[k], ec[k]), k
    # the loaded BVH refits further like the original
    t2 = _move_strand(t1, 78)
    ia, ic = sc.sc_bvh_refit(b, t2), sc.sc_bvh_refit(c, t2)
    assert (ia.moved_tris, ia.dirty_nodes) == (ic.moved_tris, ic.dirty_nodes)
    ea, ec = b.export(), c.export()
    for k in ea:
        assert np.array_equal(ea[k], ec[k]), k


def test_refit_edge_cases():
    # no triangles
    b = sc.sc_bvh_build(np.zeros((0, 9), np.float32), 6, 0)
    i = sc.sc_bvh_refit(b, np.zeros((0, 9), np.float32))
    assert (i.moved_tris, i.dirty_nodes) == (0, 0)
    # one triangle: the root is a leaf, its box moves with it
    t = np.array([[0, 0, 0, 1, 0, 0, 0, 1, 0]], np.float32)
    t2 = t + np.float32(0.5)
    b = sc.sc_bvh_build(t, 6, 1)
    i = sc.sc_bvh_refit(b, t2)
    assert (i.moved_tris, i.dirty_nodes) == (1, 0)
    ob = oracle.OracleBVH(t).build_masks(6, 3)
    ob.refit(t2)
    assert np.array_equal(np.array(b.info().root_box[:], np.float32), ob.root()[2])
    # five triangles: one node, compressed
    t5 = sg.soup(5, seed=2)
    m = t5.copy()
    m[2] += np.float32(0.1)
    b = sc.sc_bvh_build(t5, 6, 1)
    i = sc.sc_bvh_refit(b, m)
    assert (i.moved_tris, i.dirty_nodes) == (1, 1)
    _same_as_oracle(b, _oracle_refit(t5, m, 6, 1), 1)
