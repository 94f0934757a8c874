"""Parity at the full benchmark sizes, in the launch configuration bench.py
times (the wave pipeline with the autotuner's choice of block, stack,
refill and wave chunk).

* Every ray: culled hits bit-identical to plain hits (per path), culled
  per-ray counts <= plain counts, every wave and every bounce included.
* Sampled rays, computed one by one on the CPU:
  - 1M hair: the oracle's own BVH and masks trace evenly spaced primary
    rays and bounce rays (the bounce rays recomputed by the oracle from the
    GPU's primary hits): hit id, t, u, v and counts bit-identical;
  - 12.1M hair and the 4M soup: brute force over every triangle: hit t
    bit-identical, hit id identical unless another triangle ties exactly.
"""

import numpy as np
import pytest

import oracle
from paper_2305_08343_gb300 import scenegen as sg
from paper_2305_08343_gb300 import subcull as sc

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SEED = 2305


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")


def _bits(a):
    return np.ascontiguousarray(a).view(np.int32)


def _run_waves(d, r, bounces, cull, opts):
    n = r.shape[0]
    bufs = sc.WaveBuffers(n, bounces, with_counts=True, device="cuda", with_rays=True)
    sc.sc_trace_waves(d, r, bounces, SEED, cull, bufs.outs(), bufs.ws, opts)
    sizes = sc.sc_waves_poll(bufs.ws, bounces)
    sizes[0] = n
    out = []
    for w in range(bounces + 1):
        m = int(sizes[w])
        out.append(dict(hits=bufs.hits[w][:m].cpu().numpy(), path=bufs.path[w][:m].cpu().numpy(),
                        counts=bufs.counts[w][:m].cpu().numpy().view(np.uint32),
                        rays=bufs.rays[w][:m].cpu().numpy()))
    return out


def _tuned_waves(bvh, layout, rays, bounces):
    """Culled waves with the autotuned configuration, plain waves likewise."""
    d = sc.DeviceBVH(bvh, layout)
    dp = sc.DeviceBVH(bvh, sc.SC_LAYOUT_PLAIN)
    r = torch.from_numpy(rays).cuda()
    n = rays.shape[0]
    tune = sc.WaveBuffers(n, bounces, with_counts=False, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    oc, _ = sc.sc_autotune_waves(d, r, bounces, SEED, 1, tune, None, 2, flush)
    op, _ = sc.sc_autotune_waves(dp, r, bounces, SEED, 0, tune, None, 2, flush)
    del tune, flush
    culled = _run_waves(d, r, bounces, 1, oc)
    plain = _run_waves(dp, r, bounces, 0, op)
    return culled, plain


def _check_culled_equals_plain(culled, plain):
    for w, (c, p) in enumerate(zip(culled, plain)):
        oc, op = np.argsort(c["path"], kind="stable"), np.argsort(p["path"], kind="stable")
        assert np.array_equal(c["path"][oc], p["path"][op]), f"wave {w}: paths differ"
        assert np.array_equal(_bits(c["hits"][oc]), _bits(p["hits"][op])), f"wave {w}: hits differ"
        assert np.array_equal(_bits(c["rays"][oc]), _bits(p["rays"][op])), f"wave {w}: rays differ"
        assert (c["counts"][oc] <= p["counts"][op]).all(), f"wave {w}: culled counts > plain"


def _check_brute(tris, rays, hits, near_tie_rel=1e-6):
    t, hid, t2 = oracle.brute(tris, rays, 0)
    g_t, g_id = hits[:, 0], _bits(hits[:, 1])
    assert np.array_equal(_bits(g_t), _bits(t)), "closest t differs from brute force"
    tie = t2 == t
    assert np.array_equal(g_id[~tie], hid[~tie]), "closest triangle differs from brute force"
    for i in np.nonzero(tie & (hid >= 0))[0]:  # exact ties: any tied triangle is right
        ok, tt, _, _ = oracle.ray_tri(rays[i], tris[g_id[i]])
        assert ok and tt == t[i]
    with np.errstate(invalid="ignore"):
        near = (t2 - t) <= near_tie_rel * np.abs(t)
    print(f"\n{len(rays)} sampled rays: {int(near.sum())} near-tie (second hit within "
          f"{near_tie_rel:g}), {int((tie & (hid >= 0)).sum())} exact ties")


def test_hair1m_full_size_sampled_oracle_parity():
    """1,048,578 triangles (32,768 hair strands + ground), 1920x1080 primary
    rays + one diffuse bounce wave, R = 6 uncompressed masks."""
    _need_gpu()
    tris = sg.hair(32768, 16, True, seed=2)
    rays = sg.pinhole(1920, 1080)
    bvh = sc.sc_bvh_build(tris, 6, 0)
    culled, plain = _tuned_waves(bvh, sc.SC_LAYOUT_MASKED, rays, 1)
    _check_culled_equals_plain(culled, plain)
    ob = oracle.OracleBVH(tris).build_masks(6, 3)
    # primary wave: out position = primary ray index
    w0 = culled[0]
    idx = np.linspace(0, len(rays) - 1, 1500).astype(np.int64)
    assert np.array_equal(w0["path"][idx], idx)
    o = ob.trace(rays[idx], 0, 1)
    assert np.array_equal(_bits(w0["hits"][idx, 1]), o["id"])
    assert np.array_equal(_bits(w0["hits"][idx, 0]), _bits(o["t"]))
    assert np.array_equal(_bits(w0["hits"][idx, 2:]), _bits(o["uv"]))
    assert np.array_equal(w0["counts"][idx], o["counts"])
    # bounce wave: the oracle rebuilds each sampled bounce ray from the
    # primary hit of its path, then traces it
    w1 = culled[1]
    assert len(w1["path"]) > 100000
    pos = np.linspace(0, len(w1["path"]) - 1, 1500).astype(np.int64)
    pid = w1["path"][pos]
    ht0, id0 = w0["hits"][pid, 0], _bits(w0["hits"][pid, 1])
    brays = np.stack([oracle.bounce(rays[p], float(t), tris[i], SEED, int(p), 1)
                      for p, t, i in zip(pid, ht0, id0)])
    assert np.array_equal(_bits(brays), _bits(w1["rays"][pos]))
    ob_ = ob.trace(brays, 0, 1)
    assert np.array_equal(_bits(w1["hits"][pos, 1]), ob_["id"])
    assert np.array_equal(_bits(w1["hits"][pos, 0]), _bits(ob_["t"]))
    assert np.array_equal(w1["counts"][pos], ob_["counts"])


def test_hair12m_full_size_properties_and_brute_force():
    """12,100,000 hair triangles, 1920x1080 primary rays + two bounce waves,
    R = 6 LUT-compressed masks (the batched configuration)."""
    _need_gpu()
    tris = sg.hair(378125, 16, False, seed=4)
    rays = sg.pinhole(1920, 1080)
    bvh = sc.sc_bvh_build(tris, 6, 1)
    culled, plain = _tuned_waves(bvh, sc.SC_LAYOUT_MASKED, rays, 2)
    _check_culled_equals_plain(culled, plain)
    assert all(len(w["path"]) > 4096 for w in culled)
    idx = np.linspace(0, len(rays) - 1, 40).astype(np.int64)
    _check_brute(tris, rays[idx], culled[0]["hits"][idx])
    for w in (1, 2):
        pos = np.linspace(0, len(culled[w]["path"]) - 1, 12).astype(np.int64)
        _check_brute(tris, culled[w]["rays"][pos], culled[w]["hits"][pos])


def test_soup4m_full_size_closest_and_any_hit():
    """2^22 soup triangles, 2^23 random rays, closest hit (the bench's
    zero-bounce wave) and any hit, R = 6 uncompressed masks."""
    _need_gpu()
    tris = sg.soup(1 << 22, seed=3)
    rays = sg.random_rays(1 << 23, seed=3)
    bvh = sc.sc_bvh_build(tris, 6, 0)
    culled, plain = _tuned_waves(bvh, sc.SC_LAYOUT_MASKED, rays, 0)
    _check_culled_equals_plain(culled, plain)
    idx = np.linspace(0, len(rays) - 1, 48).astype(np.int64)
    _check_brute(tris, rays[idx], culled[0]["hits"][idx])
    # any hit: a reported hit is a real hit of that triangle; a miss is a miss
    d = sc.DeviceBVH(bvh, sc.SC_LAYOUT_MASKED)
    r = torch.from_numpy(rays).cuda()
    hits, _ = sc.trace(d, r, sc.SC_ANY, 1, with_counts=False)
    torch.cuda.synchronize()
    h = hits.cpu().numpy()
    del hits, r
    sample = np.linspace(0, len(rays) - 1, 256).astype(np.int64)
    ids = _bits(h[sample, 1])
    _, closest, _ = oracle.brute(tris, rays[sample], 0)
    for k, i in enumerate(sample):
        if ids[k] < 0:
            assert closest[k] < 0
        else:
            ok, tt, _, _ = oracle.ray_tri(rays[i], tris[ids[k]])
            assert ok and _bits(np.float32([tt]))[0] == _bits(h[i:i + 1, 0])[0]


def test_hair12m_full_size_oracle_counts():
    """12.1M hair with compressed masks, built as the bench builds it (tree
    and masks on the GPU), in the bench's wave configuration (primary rays
    and two bounce waves, autotuned): sampled primary, first- and
    second-bounce rays against the oracle's own BVH, masks and compression
    LUT (its threaded build) -- bounce rays, hit id, t, u, v and per-ray
    counts bit-exact."""
    _need_gpu()
    tris = sg.hair(378125, 16, False, seed=4)
    rays = sg.pinhole(1920, 1080)
    bvh = sc.sc_bvh_build(tris, 6, 1, gpu_bvh=1, gpu_masks=1)
    culled, plain = _tuned_waves(bvh, sc.SC_LAYOUT_MASKED, rays, 2)
    _check_culled_equals_plain(culled, plain)
    del plain
    ob = oracle.OracleBVH(tris).build_masks(6, 3).compress(256, 8)

    def check(w, idx, r):
        o = ob.trace(r, 0, 2)
        assert np.array_equal(_bits(w["hits"][idx, 1]), o["id"])
        assert np.array_equal(_bits(w["hits"][idx, 0]), _bits(o["t"]))
        assert np.array_equal(_bits(w["hits"][idx, 2:]), _bits(o["uv"]))
        assert np.array_equal(w["counts"][idx], o["counts"])

    w0 = culled[0]
    idx = np.linspace(0, len(rays) - 1, 600).astype(np.int64)
    check(w0, idx, rays[idx])
    by_path = [None] + [{int(p): k for k, p in enumerate(culled[w]["path"])} for w in (1, 2)]
    prev = w0
    for wave in (1, 2):
        w = culled[wave]
        assert len(w["path"]) > 100000
        pos = np.linspace(0, len(w["path"]) - 1, 300).astype(np.int64)
        pid = w["path"][pos]
        # the ray of the previous wave on each sampled path, and its hit
        k = pid if wave == 1 else np.array([by_path[1][int(p)] for p in pid])
        src = rays[pid] if wave == 1 else prev["rays"][k]
        ht, hid = prev["hits"][k, 0], _bits(prev["hits"][k, 1])
        brays = np.stack([oracle.bounce(src[q], float(ht[q]), tris[hid[q]], SEED, int(pid[q]),
                                        wave) for q in range(len(pid))])
        assert np.array_equal(_bits(brays), _bits(w["rays"][pos]))
        check(w, pos, brays)
        prev = w
