"""The product's host side (libsubcull: BVH builder, masks, ray-mask table,
compression, C-ABI) against the CPU oracle, on the CPU.

Integer and bit results must match exactly: tree topology, boxes, leaf
order, object masks, compression table and indices, ray-mask table.
"""
import ctypes as C
import os
import re

import numpy as np
import pytest

import oracle
from paper_2305_08343_gb300 import scenegen as sg
from paper_2305_08343_gb300 import subcull as sc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _scenes():
    yield "hair65k", sg.hair(2048, 16, False, seed=1)
    yield "hair_ground", sg.hair(300, 16, True, seed=2)
    yield "soup", sg.soup(20000, seed=3)
    yield "identical", np.tile(np.array([[0, 0, 0, 1, 0, 0, 0, 1, 0]], np.float32), (37, 1))
    yield "single", np.array([[0, 0, 0, 1, 0, 0, 0, 1, 0]], np.float32)
    yield "empty", np.zeros((0, 9), np.float32)


@pytest.mark.parametrize("name,tris", list(_scenes()), ids=lambda x: x if isinstance(x, str) else "")
def test_tree_matches_oracle(name, tris):
    b = sc.sc_bvh_build(tris, 0, 0)
    ex = b.export()
    ob = oracle.OracleBVH(tris)
    child, count, box = ob.nodes()
    rc, rn, rbox = ob.root()
    assert ex["root"].tolist() == [rc, rn]
    assert np.array_equal(ex["child"], child)
    assert np.array_equal(ex["count"], count)
    assert np.array_equal(ex["box"], box)
    assert np.array_equal(ex["perm"], ob.perm())
    info = b.info()
    assert info.num_nodes == ob.num_nodes and info.max_depth == ob.max_depth
    if len(tris):
        assert np.array_equal(np.array(info.root_box[:], np.float32), rbox)


@pytest.mark.parametrize("R,L", [(4, 3), (6, 3), (6, 1), (8, 3), (6, 5)])
def test_masks_match_oracle(R, L):
    for tris in (sg.hair(400, 16, True, seed=4), sg.soup(6000, seed=5)):
        b = sc.sc_bvh_build(tris, R, 1, L=L)
        ex = b.export()
        ob = oracle.OracleBVH(tris).build_masks(R, L=L).compress(256, 8)
        assert np.array_equal(ex["masks"], ob.masks())
        clut, cidx = ob.clut()
        assert np.array_equal(ex["clut"], clut)
        assert np.array_equal(ex["cidx"], cidx)
        assert b.info().eps == ob.eps


@pytest.mark.parametrize("R", [2, 3, 4, 6, 8])
def test_raylut_matches_oracle(R):
    assert np.array_equal(sc.sc_raylut(R), oracle.raylut(R))


@pytest.mark.parametrize("R", [2, 3, 4, 6])
def test_raylut2r_matches_oracle(R):
    assert np.array_equal(sc.sc_raylut2r(R), oracle.raylut2r(R))


def test_thread_count_does_not_change_the_build():
    tris = sg.hair(3000, 16, True, seed=6)
    a = sc.sc_bvh_build(tris, 6, 1, threads=1).export()
    b = sc.sc_bvh_build(tris, 6, 1, threads=7).export()
    for k in a:
        assert np.array_equal(a[k], b[k]), k


def test_scene_generation_through_abi_matches_module():
    t1 = sc.sc_scene_generate(sc.SC_SCENE_HAIR, 100, 16, 1, seed=9)
    assert np.array_equal(t1, sg.hair(100, 16, True, seed=9))
    t2 = sc.sc_scene_generate(sc.SC_SCENE_SOUP, 5000, seed=9)
    assert np.array_equal(t2, sg.soup(5000, seed=9))
    r1 = sc.sc_rays_generate(sc.SC_RAYS_PINHOLE, 64, 40)
    assert np.array_equal(r1, sg.pinhole(64, 40))
    r2 = sc.sc_rays_generate(sc.SC_RAYS_RANDOM, count=3000, seed=4)
    assert np.array_equal(r2, sg.random_rays(3000, seed=4))


def _declared_symbols():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(sc_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return names


def test_library_exports_every_declared_symbol():
    names = _declared_symbols()
    assert {"sc_trace", "sc_bvh_build", "sc_bvh_upload", "sc_scene_generate"} <= names
    L = sc.lib()
    missing = [n for n in sorted(names) if not hasattr(L, n)]
    assert not missing, missing
    assert L.sc_abi_version() == sc.SC_ABI_VERSION == 2


def test_errors_are_reported_not_raised_through_the_abi():
    tris = sg.hair(4, 16, False)
    with pytest.raises(sc.SubcullError) as e:
        sc.sc_bvh_build(tris, 5, 0)
    assert e.value.code == -6 and "grid_res" in str(e.value)
    bad = tris.copy()
    bad[3, 4] = np.nan
    with pytest.raises(sc.SubcullError) as e:
        sc.sc_bvh_build(bad, 6, 0)
    assert e.value.code == -1
    with pytest.raises(sc.SubcullError):
        sc.sc_bvh_build(tris, 0, 1)  # compression without masks
    with pytest.raises(sc.SubcullError) as e:  # rejected before any device call
        sc.sc_bvh_build(tris, 0, 0, gpu_bvh=1, bins=64)
    assert e.value.code == -6 and "32 bins" in str(e.value)
    b = sc.sc_bvh_build(tris, 0, 0)
    with pytest.raises(sc.SubcullError) as e:
        sc.sc_bvh_device_bytes(b, sc.SC_LAYOUT_MASKED)
    assert e.value.code == -7
    # NULL device pointers are rejected before any CUDA call
    n = C.c_void_p()
    code = sc.lib().sc_bvh_upload(b.handle, 0, None, 0, None, C.byref(n))
    assert code == -1


def test_device_image_sizes():
    import json
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_numbers.json")))["bvh4_node_bytes"]
    # Sec. 3.2.4: a w-wide node holds w boxes (24 B) and w child words (4 B);
    # masks add w * R^3/8 bytes uncompressed, w * 1 byte compressed.
    w, R = g["width"], g["R"]
    assert w * (24 + 4) == g["plain"]
    assert w * (24 + 4) + w * R ** 3 // 8 == g["uncompressed"]
    assert w * (24 + 4) + w * 1 == g["compressed"]
    # this BVH2's records: the same content for w = 2 rounded up to 16-B
    # vectors (64 B; the compressed index fits in the padding), plus the
    # two masks padded to 8/32/64 B when uncompressed.
    tris = sg.hair(64, 16, False)
    for R, unc in ((4, 80), (6, 128), (8, 192)):
        for comp, nb in ((0, unc), (1, 64)):
            b = sc.sc_bvh_build(tris, R, comp)
            nn = b.info().num_nodes
            plain = sc.sc_bvh_device_bytes(b, sc.SC_LAYOUT_PLAIN)
            masked = sc.sc_bvh_device_bytes(b, sc.SC_LAYOUT_MASKED)
            assert plain % 256 == 0 and masked % 256 == 0
            assert masked - plain >= nn * (nb - 64)


def test_ray2r_image_sizes_and_limits():
    """SC_LAYOUT_MASKED_RAY2R adds the (2R)^6-row table (one mask stride per
    row) to SC_LAYOUT_MASKED, for uncompressed masks at R = 4 and 6 only."""
    tris = sg.hair(64, 16, False)
    for R, stride in ((4, 8), (6, 32)):
        b = sc.sc_bvh_build(tris, R, 0)
        extra = (sc.sc_bvh_device_bytes(b, sc.SC_LAYOUT_MASKED_RAY2R)
                 - sc.sc_bvh_device_bytes(b, sc.SC_LAYOUT_MASKED))
        rows = (2 * R) ** 6
        assert rows * stride <= extra < rows * stride + 256
    for R, comp in ((8, 0), (6, 1)):
        b = sc.sc_bvh_build(tris, R, comp)
        with pytest.raises(sc.SubcullError) as e:
            sc.sc_bvh_device_bytes(b, sc.SC_LAYOUT_MASKED_RAY2R)
        assert e.value.code == sc.SC_ERR_UNSUPPORTED


def test_probe_and_refit_argument_errors_without_a_device():
    L = sc.lib()
    # NULL buffers are refused before any device call
    assert L.sc_l2_read(None, 16, 1, None, None) == sc.SC_ERR_ARG
    assert L.sc_bvh_refit(None, None, 0, None) == sc.SC_ERR_ARG
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except ImportError:
        has_gpu = False
    if not has_gpu:
        assert L.sc_l2_probe_blocks() == 0
