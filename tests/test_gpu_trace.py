"""GPU traversal (libsubcull, sm_103a) against the CPU oracle, through the
C-ABI.

The oracle builds its own BVH, masks, ray-mask table and compression LUT
from the same seeded triangles (it shares no code with the product) and
traces the same rays.  Required agreement (Alg. 4 with Alg. 1, culling of
Sec. 3.1.2): hit triangle ids and per-ray slab / triangle test counts
bit-exact; hit t within 1e-6 relative (the path is expected to be exact and
the test reports it); culled hits identical to plain hits; culled counts
<= plain counts.
"""
import ctypes as C

import numpy as np
import pytest

import oracle
from paper_2305_08343_gb300 import scenegen as sg
from paper_2305_08343_gb300 import subcull as sc

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

T_REL = 1e-6


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")


def gpu_trace(bvh, rays, mode, cull, lut_mode=sc.SC_LUT_AUTO, layout=None, refill=0):
    _need_gpu()
    lay = layout if layout is not None else (sc.SC_LAYOUT_MASKED if cull else sc.SC_LAYOUT_PLAIN)
    d = sc.DeviceBVH(bvh, lay)
    r = torch.from_numpy(np.ascontiguousarray(rays)).cuda()
    hits, counts = sc.trace(d, r, mode, cull, opts=sc._opts(lut_mode=lut_mode, refill=refill))
    torch.cuda.synchronize()
    t, i, u, v = sc.split_hits(hits)
    return dict(t=t.copy(), id=i.copy(), uv=np.stack([u, v], 1),
                counts=counts.cpu().numpy().view(np.uint32).copy())


def oracle_trace(tris, rays, R, comp, mode, cull, skip_bits=None, stride=1, leaf_min=0):
    ob = oracle.OracleBVH(tris)
    if R:
        ob.build_masks(R, 3)
        if comp:
            ob.compress(256, 8)
    return ob.trace(rays, mode, (2 if comp else 1) if cull else 0, skip_bits=skip_bits,
                    stride=stride, leaf_min=leaf_min)


def assert_parity(g, o, what=""):
    bad_id = np.nonzero(g["id"] != o["id"])[0]
    assert bad_id.size == 0, f"{what}: {bad_id.size} hit ids differ, first rays {bad_id[:8]}"
    hit = o["id"] >= 0
    assert np.array_equal(np.isinf(g["t"]), np.isinf(o["t"]))
    rel = np.abs(g["t"][hit] - o["t"][hit]) / np.maximum(np.abs(o["t"][hit]), 1e-30)
    assert (rel <= T_REL).all(), f"{what}: t differs by {rel.max()}"
    bad_c = np.nonzero((g["counts"] != o["counts"]).any(1))[0]
    assert bad_c.size == 0, (f"{what}: counts differ on {bad_c.size} rays, e.g. ray {bad_c[:4]}: "
                             f"gpu {g['counts'][bad_c[:4]].tolist()} oracle {o['counts'][bad_c[:4]].tolist()}")
    # exactness beyond the required tolerance (reported through the assert)
    assert np.array_equal(g["t"][hit], o["t"][hit]) and np.array_equal(g["uv"][hit], o["uv"][hit])


@pytest.fixture(scope="module")
def c1():
    """2,048 strands x 16 segments x 2 = 65,536 thin tilted triangles,
    256x256 pinhole rays (the small hair configuration)."""
    return sg.hair(2048, 16, False, seed=1), sg.pinhole(256, 256)


@pytest.mark.parametrize("comp", [0, 1])
def test_hair65k_parity_culled_and_plain(c1, comp):
    tris, rays = c1
    b = sc.sc_bvh_build(tris, 6, comp)
    plain_g = gpu_trace(b, rays, 0, 0)
    cull_g = gpu_trace(b, rays, 0, 1)
    plain_o = oracle_trace(tris, rays, 0, 0, 0, 0)
    cull_o = oracle_trace(tris, rays, 6, comp, 0, 1)
    assert_parity(plain_g, plain_o, "plain")
    assert_parity(cull_g, cull_o, "culled")
    assert np.array_equal(cull_g["id"], plain_g["id"]) and np.array_equal(cull_g["t"], plain_g["t"])
    assert (cull_g["counts"] <= plain_g["counts"]).all()
    assert cull_g["counts"].sum() < plain_g["counts"].sum()


@pytest.mark.parametrize("R", [4, 6, 8])
@pytest.mark.parametrize("comp,lut", [(0, sc.SC_LUT_GLOBAL), (0, sc.SC_LUT_SHARED),
                                      (1, sc.SC_LUT_GLOBAL), (1, sc.SC_LUT_SHARED),
                                      (1, sc.SC_LUT_BITTABLE)])
@pytest.mark.parametrize("layout", [sc.SC_LAYOUT_MASKED, sc.SC_LAYOUT_MASKED_COMPACT])
def test_resolutions_lut_modes_layouts(hair_small, R, comp, lut, layout):
    tris, rays = hair_small
    b = sc.sc_bvh_build(tris, R, comp)
    g = gpu_trace(b, rays, 0, 1, lut_mode=lut, layout=layout)
    o = oracle_trace(tris, rays, R, comp, 0, 1)
    assert_parity(g, o, f"R={R} comp={comp} lut={lut} layout={layout}")


@pytest.mark.parametrize("mode", [0, 1])
def test_factored_tables_through_l1(hair_small, mode):
    """SC_LUT_FACTORED_L1: the Helly-factored 2-D tables read from the image
    through L1 give the oracle's hits and per-ray counts."""
    tris, rays = hair_small
    b = sc.sc_bvh_build(tris, 6, 0)
    g = gpu_trace(b, rays, mode, 1, lut_mode=sc.SC_LUT_FACTORED_L1)
    o = oracle_trace(tris, rays, 6, 0, mode, 1)
    assert_parity(g, o, f"factored L1 mode={mode}")


@pytest.mark.parametrize("R,comp,layout", [(4, 0, None), (6, 1, None),
                                           (6, 0, sc.SC_LAYOUT_MASKED_COMPACT)])
def test_factored_tables_through_l1_rejects_other_images(hair_small, R, comp, layout):
    tris, rays = hair_small
    b = sc.sc_bvh_build(tris, R, comp)
    with pytest.raises(sc.SubcullError, match="L1-read factored"):
        gpu_trace(b, rays, 0, 1, lut_mode=sc.SC_LUT_FACTORED_L1, layout=layout)


@pytest.mark.parametrize("skip", [150, 100, 40])
@pytest.mark.parametrize("comp", [0, 1])
def test_dense_mask_skip_threshold(hair_small, skip, comp):
    tris, rays = hair_small
    b = sc.sc_bvh_build(tris, 6, comp, skip_bits=skip)
    g = gpu_trace(b, rays, 0, 1)
    assert_parity(g, oracle_trace(tris, rays, 6, comp, 0, 1, skip_bits=skip), f"skip={skip}")


@pytest.mark.parametrize("stride,skip", [(2, 0), (3, 150)])
@pytest.mark.parametrize("comp", [0, 1])
def test_test_stride(hair_small, stride, skip, comp):
    tris, rays = hair_small
    b = sc.sc_bvh_build(tris, 6, comp, skip_bits=skip, test_stride=stride)
    g = gpu_trace(b, rays, 0, 1)
    o = oracle_trace(tris, rays, 6, comp, 0, 1, skip_bits=skip or None, stride=stride)
    assert_parity(g, o, f"stride={stride} skip={skip}")


@pytest.mark.parametrize("leaf_min,stride", [(2, 1), (3, 1), (4, 2)])
@pytest.mark.parametrize("comp", [0, 1])
def test_leaf_min(hair_small, leaf_min, stride, comp):
    tris, rays = hair_small
    b = sc.sc_bvh_build(tris, 6, comp, leaf_min_tris=leaf_min, test_stride=stride)
    g = gpu_trace(b, rays, 0, 1)
    o = oracle_trace(tris, rays, 6, comp, 0, 1, stride=stride, leaf_min=leaf_min)
    assert_parity(g, o, f"leaf_min={leaf_min} stride={stride}")


@pytest.mark.parametrize("max_leaf", [1, 8])
@pytest.mark.parametrize("comp", [0, 1])
def test_leaf_sizes(hair_small, max_leaf, comp):
    tris, rays = hair_small
    b = sc.sc_bvh_build(tris, 6, comp, max_leaf=max_leaf)
    ob = oracle.OracleBVH(tris, max_leaf=max_leaf).build_masks(6, 3)
    if comp:
        ob.compress(256, 8)
    assert_parity(gpu_trace(b, rays, 0, 1), ob.trace(rays, 0, 2 if comp else 1),
                  f"max_leaf={max_leaf}")
    assert_parity(gpu_trace(b, rays, 0, 0), ob.trace(rays, 0, 0), f"plain max_leaf={max_leaf}")


@pytest.mark.parametrize("refill", [1, 4, 16, 32])
def test_refill_threshold_does_not_change_results(hair_small, refill):
    tris, rays = hair_small
    b = sc.sc_bvh_build(tris, 6, 1)
    o = oracle_trace(tris, rays, 6, 1, 0, 1)
    assert_parity(gpu_trace(b, rays, 0, 1, refill=refill), o, f"refill={refill}")
    assert_parity(gpu_trace(b, rays, 0, 0, refill=refill), oracle_trace(tris, rays, 0, 0, 0, 0),
                  f"plain refill={refill}")


@pytest.mark.parametrize("mode", [0, 1])
def test_soup_random_rays_closest_and_any(mode):
    tris = sg.soup(16384, seed=13)
    rays = sg.random_rays(8192 + 17, seed=14)   # ragged tail
    b = sc.sc_bvh_build(tris, 6, 0)
    for cull in (0, 1):
        g = gpu_trace(b, rays, mode, cull)
        o = oracle_trace(tris, rays, 6 if cull else 0, 0, mode, cull)
        assert_parity(g, o, f"soup mode={mode} cull={cull}")


def test_ground_and_inside_origins():
    tris = sg.hair(500, 16, True, seed=15)
    rays = sg.random_rays(5000, seed=16)
    rays[:, :3] = rays[:, :3] * 3.0 - 1.5          # origins inside the hair volume
    rays[::3, 3] = 1e-4                             # some rays with tmin > 0
    rays[::5, 7] = 0.7                              # and a finite tmax
    b = sc.sc_bvh_build(tris, 6, 1)
    for cull in (0, 1):
        g = gpu_trace(b, rays, 0, cull)
        o = oracle_trace(tris, rays, 6 if cull else 0, 1, 0, cull)
        assert_parity(g, o, f"ground cull={cull}")


@pytest.mark.parametrize("n", [0, 1, 31, 33, 1000])
def test_ragged_ray_counts(hair_small, n):
    tris, rays = hair_small
    b = sc.sc_bvh_build(tris, 6, 0)
    r = rays[:n].copy()
    if n == 0:
        d = sc.DeviceBVH(b, sc.SC_LAYOUT_MASKED)
        hits, counts = sc.trace(d, torch.zeros((0, 8), dtype=torch.float32, device="cuda"), 0, 1)
        assert hits.shape[0] == 0
        return
    assert_parity(gpu_trace(b, r, 0, 1), oracle_trace(tris, r, 6, 0, 0, 1), f"n={n}")


def test_degenerate_scenes():
    rays = sg.pinhole(40, 20)
    one = np.array([[-1, -1, 0, 1, -1, 0, 0, 1, 0]], np.float32)
    for tris in (one, np.tile(one, (9, 1))):
        b = sc.sc_bvh_build(tris, 6, 0)
        for cull in (0, 1):
            assert_parity(gpu_trace(b, rays, 0, cull),
                          oracle_trace(tris, rays, 6 if cull else 0, 0, 0, cull), "degenerate")
    empty = np.zeros((0, 9), np.float32)
    b = sc.sc_bvh_build(empty, 6, 0)
    g = gpu_trace(b, rays, 0, 1)
    assert (g["id"] == -1).all() and np.isinf(g["t"]).all() and (g["counts"] == 0).all()


def test_deep_tree_is_rejected_before_launch():
    """A BVH deeper than the kernel's 64-entry stack is refused on the host
    (SC_ERR_UNSUPPORTED) instead of being launched."""
    ks = np.arange(-24, 25)
    x = (33.0 ** ks).astype(np.float32)
    ta = np.zeros((len(ks), 9), np.float32)
    ta[:, 0], ta[:, 3], ta[:, 6], ta[:, 7] = x, x * 1.01, x, x * 0.01
    tb = np.zeros((len(ks), 9), np.float32)
    tb[:, 1], tb[:, 4], tb[:, 7], tb[:, 8] = x, x * 1.01, x, x * 0.01
    tris = np.vstack([ta, tb])
    b = sc.sc_bvh_build(tris, 6, 0)
    assert b.info().max_depth + 1 > 64
    d = sc.DeviceBVH(b, sc.SC_LAYOUT_MASKED)
    r = torch.from_numpy(sg.pinhole(8, 4)).cuda()
    with pytest.raises(sc.SubcullError) as e:
        sc.trace(d, r, 0, 1)
    assert e.value.code == -6


def test_cull_requires_masked_image(hair_small):
    tris, rays = hair_small
    b = sc.sc_bvh_build(tris, 6, 0)
    d = sc.DeviceBVH(b, sc.SC_LAYOUT_PLAIN)
    r = torch.from_numpy(rays[:64]).cuda()
    with pytest.raises(sc.SubcullError) as e:
        sc.trace(d, r, 0, 1)
    assert e.value.code == -7
    # plain traversal works on the masked image too (same results)
    g1 = gpu_trace(b, rays, 0, 0, layout=sc.SC_LAYOUT_MASKED)
    g2 = gpu_trace(b, rays, 0, 0, layout=sc.SC_LAYOUT_PLAIN)
    assert np.array_equal(g1["id"], g2["id"]) and np.array_equal(g1["counts"], g2["counts"])


def test_trace_host_end_to_end(hair_small):
    """sc_trace_host: host rays in, host hits out (the e2e form)."""
    tris, rays = hair_small
    b = sc.sc_bvh_build(tris, 6, 1)
    d = sc.DeviceBVH(b, sc.SC_LAYOUT_MASKED)
    n = rays.shape[0]
    h_rays = torch.from_numpy(rays).pin_memory()
    h_hits = torch.empty((n, 4), dtype=torch.float32).pin_memory()
    h_counts = torch.empty((n, 2), dtype=torch.int32).pin_memory()
    d_rays = torch.empty((n, 8), dtype=torch.float32, device="cuda")
    d_hits = torch.empty((n, 4), dtype=torch.float32, device="cuda")
    d_counts = torch.empty((n, 2), dtype=torch.int32, device="cuda")
    work = torch.empty(sc.sc_trace_workspace_bytes(), dtype=torch.uint8, device="cuda")
    sc.sc_trace_host(d, h_rays, h_hits, h_counts, 0, 1, d_rays, d_hits, d_counts, work)
    t, i, u, v = sc.split_hits(h_hits)
    o = oracle_trace(tris, rays, 6, 1, 0, 1)
    assert np.array_equal(i, o["id"])
    assert np.array_equal(h_counts.numpy().view(np.uint32), o["counts"])


@pytest.mark.parametrize("R,comp", [(0, 0), (4, 0), (6, 0), (6, 1), (8, 1), (4, 1)])
@pytest.mark.parametrize("mode", [0, 1])
def test_wide_nodes_match_oracle(hair_small, R, comp, mode):
    """4-wide images against the oracle's 4-wide traversal: hits and counts
    bit-exact; hits equal to the binary traversal's."""
    tris, rays = hair_small
    b = sc.sc_bvh_build(tris, R, comp)
    ob = oracle.OracleBVH(tris)
    if R:
        ob.build_masks(R, 3)
        if comp:
            ob.compress(256, 8)
    lay = sc.SC_LAYOUT_MASKED4 if R else sc.SC_LAYOUT_PLAIN4
    cull = 1 if R else 0
    g = gpu_trace(b, rays, mode, cull, layout=lay)
    o = ob.trace(rays, mode, (2 if comp else 1) if cull else 0, width=4)
    assert_parity(g, o, f"4-wide R={R} comp={comp} mode={mode}")
    if mode == 0:
        two = ob.trace(rays, 0, 0)
        assert np.array_equal(g["id"], two["id"])
    if R:  # the plain kernel on the masked 4-wide image
        assert_parity(gpu_trace(b, rays, mode, 0, layout=lay), ob.trace(rays, mode, 0, width=4),
                      "plain on masked 4-wide")


def test_wide_nodes_soup_and_ground():
    tris = np.concatenate([sg.soup(8000, seed=41), sg.hair(64, 16, True, seed=2)])
    rays = np.concatenate([sg.random_rays(3000, seed=42), sg.pinhole(48, 32)])
    b = sc.sc_bvh_build(tris, 6, 0)
    ob = oracle.OracleBVH(tris).build_masks(6, 3)
    assert_parity(gpu_trace(b, rays, 0, 1, layout=sc.SC_LAYOUT_MASKED4),
                  ob.trace(rays, 0, 1, width=4), "4-wide soup")
