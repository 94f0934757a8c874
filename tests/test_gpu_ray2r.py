"""Culled traversal with the ray-mask table at R_ray = 2R (Sec. 4.2; images in
SC_LAYOUT_MASKED_RAY2R) against the CPU oracle with its own 2R table
(OracleBVH.set_ray2r), through the C-ABI.  Hit ids, t, u, v and per-ray
counts must agree bit for bit in:
* the single-batch kernel, closest and any hit, R = 4 and 6;
* the wave pipeline, every wave, including tuned block / stack variants;
* the seeded traversal.
The same image traced with SC_LUT_GLOBAL gives the R-table results, and no
ray needs more tests with the 2R table than with the R table."""
import numpy as np
import pytest

import oracle
from paper_2305_08343_gb300 import scenegen as sg
from paper_2305_08343_gb300 import subcull as sc

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

LAYOUT = sc.SC_LAYOUT_MASKED_RAY2R


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")


def _bits(a):
    return np.ascontiguousarray(a).view(np.int32)


def _gpu(b, rays, mode, lut=sc.SC_LUT_AUTO):
    d = sc.DeviceBVH(b, LAYOUT)
    r = torch.from_numpy(np.ascontiguousarray(rays)).cuda()
    hits, counts = sc.trace(d, r, mode, 1, opts=sc._opts(lut_mode=lut))
    torch.cuda.synchronize()
    return hits.cpu().numpy(), counts.cpu().numpy().view(np.uint32)


def _oracle(tris, R, two_r=True):
    ob = oracle.OracleBVH(tris).build_masks(R, 3)
    return ob.set_ray2r() if two_r else ob


def _same(h, c, o):
    assert np.array_equal(_bits(h[:, 1]), o["id"])
    assert np.array_equal(_bits(h[:, 0]), _bits(o["t"]))
    hit = o["id"] >= 0
    assert np.array_equal(_bits(h[hit, 2:]), _bits(o["uv"][hit]))
    bad = np.nonzero((c != o["counts"]).any(1))[0]
    assert bad.size == 0, f"counts differ on {bad.size} rays, e.g. {bad[:4]}"


@pytest.fixture(scope="module")
def scene():
    """2,048 strands x 16 segments x 2 + ground, 200x150 pinhole rays (a
    ragged count: not a multiple of the warp or block)."""
    return sg.hair(2048, 16, True, seed=1), sg.pinhole(200, 150)[:29999]


@pytest.mark.parametrize("R", [4, 6])
@pytest.mark.parametrize("mode", [sc.SC_CLOSEST, sc.SC_ANY])
def test_single_batch_matches_oracle(scene, R, mode):
    _need_gpu()
    tris, rays = scene
    b = sc.sc_bvh_build(tris, R, 0)
    h2, c2 = _gpu(b, rays, mode)
    _same(h2, c2, _oracle(tris, R).trace(rays, mode, 1))
    # the R table of the same image, and the 2R table's tighter culling
    h1, c1 = _gpu(b, rays, mode, sc.SC_LUT_GLOBAL)
    _same(h1, c1, _oracle(tris, R, False).trace(rays, mode, 1))
    assert np.array_equal(_bits(h1[:, :2]), _bits(h2[:, :2]))
    assert (c2 <= c1).all() and c2.sum() < c1.sum()


def _oracle_waves(tris, rays, bounces, seed, R):
    ob = _oracle(tris, R)
    waves, cur, path = [], rays, np.arange(len(rays))
    for w in range(bounces + 1):
        o = ob.trace(cur, 0, 1)
        waves.append(dict(path=path, **o))
        if w < bounces:
            cur, path = oracle.bounce_wave(cur, o["t"], o["id"], tris, seed, w + 1, path)
    return waves


@pytest.mark.parametrize("R,cfg", [(4, {}), (6, {}), (6, dict(block=256, stack=32)),
                                   (6, dict(block=64, wave_chunk=777))])
def test_waves_match_oracle(R, cfg):
    _need_gpu()
    tris = sg.hair(400, 16, True, seed=31)
    rays = sg.pinhole(64, 48)
    b = sc.sc_bvh_build(tris, R, 0)
    d = sc.DeviceBVH(b, LAYOUT)
    r = torch.from_numpy(rays).cuda()
    bufs, sizes = sc.trace_waves(d, r, 2, 1234, 1, opts=sc._opts(**cfg))
    torch.cuda.synchronize()
    o = _oracle_waves(tris, rays, 2, 1234, R)
    for w in range(3):
        m = int(sizes[w])
        path = bufs.path[w][:m].cpu().numpy()
        g_id = _bits(bufs.hits[w][:m].cpu().numpy()[:, 1])
        g_cnt = bufs.counts[w][:m].cpu().numpy().view(np.uint32)
        gord, oord = np.argsort(path, kind="stable"), np.argsort(o[w]["path"], kind="stable")
        assert np.array_equal(path[gord], o[w]["path"][oord]), f"wave {w}: different rays"
        assert np.array_equal(g_id[gord], o[w]["id"][oord]), f"wave {w}: hit ids differ"
        assert np.array_equal(g_cnt[gord], o[w]["counts"][oord]), f"wave {w}: counts differ"
    assert len(o[1]["path"]) > 100 and len(o[2]["path"]) > 10


def test_seeded_matches_oracle():
    _need_gpu()
    tris, rays = sg.hair(1024, 16, True, seed=21), sg.pinhole(96, 64)[:4000]
    b = sc.sc_bvh_build(tris, 6, 0)
    d = sc.DeviceBVH(b, LAYOUT)
    ent, _ = sc.sc_bvh_frontier(b, 8)
    cls = np.random.default_rng(17).integers(-2, ent.shape[0] + 2, rays.shape[0]).astype(np.int32)
    n = rays.shape[0]
    hits = torch.full((n, 4), -7.0, dtype=torch.float32, device="cuda")
    counts = torch.zeros((n, 2), dtype=torch.int32, device="cuda")
    work = torch.empty(sc.sc_trace_workspace_bytes(), dtype=torch.uint8, device="cuda")
    sc.sc_trace_seeded(d, torch.from_numpy(rays).cuda(), torch.from_numpy(cls).cuda(),
                       torch.from_numpy(ent).cuda(), hits, counts, 1, work)
    sc.sc_status_poll(work)
    o = _oracle(tris, 6).trace_seeded(rays, cls, 8, cull=1)
    _same(hits.cpu().numpy(), counts.cpu().numpy().view(np.uint32), o)


def test_2r_lookup_needs_the_2r_image():
    _need_gpu()
    tris, rays = sg.hair(64, 16, True, seed=3), sg.pinhole(32, 32)
    b = sc.sc_bvh_build(tris, 6, 0)
    d = sc.DeviceBVH(b, sc.SC_LAYOUT_MASKED)
    r = torch.from_numpy(rays).cuda()
    with pytest.raises(sc.SubcullError) as e:
        sc.trace(d, r, 0, 1, opts=sc._opts(lut_mode=sc.SC_LUT_RAY2R))
    assert e.value.code == sc.SC_ERR_ARG
