"""The wave pipeline (primary rays + diffuse bounce waves in one cooperative
launch) against the CPU oracle: the oracle traces the primaries, spawns the
bounce rays of every hit with the same generator (keyed by path id) and
traces them; the GPU waves, keyed by path id, must hold the same rays'
results: hit ids and per-ray counts exact, t within 1e-6 relative."""
import numpy as np
import pytest

import oracle
from paper_2305_08343_gb300 import scenegen as sg
from paper_2305_08343_gb300 import subcull as sc

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _oracle_waves(tris, rays, bounces, seed, R, comp, cull, skip_bits=None, width=2):
    ob = oracle.OracleBVH(tris)
    if R:
        ob.build_masks(R, 3)
        if comp:
            ob.compress(256, 8)
    mode = (2 if comp else 1) if cull else 0
    waves = []
    cur, path = rays, np.arange(len(rays))
    for w in range(bounces + 1):
        o = ob.trace(cur, 0, mode, skip_bits=skip_bits, width=width)
        waves.append(dict(path=path, **o))
        if w < bounces:
            cur, path = oracle.bounce_wave(cur, o["t"], o["id"], tris, seed, w + 1, path)
    return waves


def _gpu_waves(tris, rays, bounces, seed, R, comp, cull, layout=None, lut=sc.SC_LUT_AUTO,
               **opts):
    b = sc.sc_bvh_build(tris, R, comp)
    lay = layout if layout is not None else (sc.SC_LAYOUT_MASKED if cull else sc.SC_LAYOUT_PLAIN)
    d = sc.DeviceBVH(b, lay)
    r = torch.from_numpy(rays).cuda()
    bufs, sizes = sc.trace_waves(d, r, bounces, seed, cull, opts=sc._opts(lut_mode=lut, **opts))
    torch.cuda.synchronize()
    out = []
    for w in range(bounces + 1):
        m = int(sizes[w])
        t, i, u, v = sc.split_hits(bufs.hits[w][:m])
        path = bufs.path[w][:m].cpu().numpy()
        cnt = bufs.counts[w][:m].cpu().numpy().view(np.uint32)
        order = np.argsort(path, kind="stable")
        out.append(dict(path=path[order], t=t[order], id=i[order], counts=cnt[order]))
    return out


@pytest.mark.parametrize("cull,comp,layout,lut", [
    (0, 0, None, 0), (1, 0, 1, 0), (1, 0, 2, 0), (1, 1, 1, sc.SC_LUT_BITTABLE),
    (1, 1, 2, sc.SC_LUT_BITTABLE), (1, 1, 1, sc.SC_LUT_GLOBAL)])
def test_waves_match_oracle(cull, comp, layout, lut):
    tris = sg.hair(400, 16, True, seed=31)
    rays = sg.pinhole(64, 48)
    g = _gpu_waves(tris, rays, 2, 1234, 6, comp, cull, layout, lut)
    o = _oracle_waves(tris, rays, 2, 1234, 6, comp, cull)
    for w in range(3):
        op = o[w]["path"]
        assert np.array_equal(g[w]["path"], np.sort(op)), f"wave {w}: different rays"
        order = np.argsort(op, kind="stable")
        assert np.array_equal(g[w]["id"], o[w]["id"][order]), f"wave {w}: hit ids differ"
        assert np.array_equal(g[w]["counts"], o[w]["counts"][order]), f"wave {w}: counts differ"
        assert np.array_equal(g[w]["t"], o[w]["t"][order])
    assert len(o[1]["path"]) > 100 and len(o[2]["path"]) > 10


@pytest.mark.parametrize("comp,lut", [(0, sc.SC_LUT_SHARED), (1, sc.SC_LUT_SHARED),
                                      (1, sc.SC_LUT_BITTABLE), (0, sc.SC_LUT_GLOBAL)])
def test_waves_r4_lookup_variants(comp, lut):
    tris = sg.hair(400, 16, True, seed=34)
    rays = sg.pinhole(64, 48)
    g = _gpu_waves(tris, rays, 2, 77, 4, comp, 1, None, lut)
    o = _oracle_waves(tris, rays, 2, 77, 4, comp, 1)
    for w in range(3):
        order = np.argsort(o[w]["path"], kind="stable")
        assert np.array_equal(g[w]["path"], np.sort(o[w]["path"]))
        assert np.array_equal(g[w]["id"], o[w]["id"][order])
        assert np.array_equal(g[w]["counts"], o[w]["counts"][order])


@pytest.mark.parametrize("lut", [sc.SC_LUT_SHARED, sc.SC_LUT_FACTORED_L1])
@pytest.mark.parametrize("cfg", [dict(), dict(block=64, stack=32), dict(block=256, stack=64)])
def test_waves_r6_factored_tables(lut, cfg):
    """R = 6, uncompressed masks, stored scales: the Helly-factored ray-mask
    tables in shared memory or read through L1, in several block / stack
    shapes of the wave pipeline, against the oracle."""
    tris = sg.hair(400, 16, True, seed=36)
    rays = sg.pinhole(64, 48)
    g = _gpu_waves(tris, rays, 2, 91, 6, 0, 1, sc.SC_LAYOUT_MASKED, lut, **cfg)
    o = _oracle_waves(tris, rays, 2, 91, 6, 0, 1)
    for w in range(3):
        order = np.argsort(o[w]["path"], kind="stable")
        assert np.array_equal(g[w]["path"], np.sort(o[w]["path"])), f"wave {w} {cfg}"
        assert np.array_equal(g[w]["id"], o[w]["id"][order])
        assert np.array_equal(g[w]["counts"], o[w]["counts"][order])


@pytest.mark.parametrize("cfg", [dict(wave_chunk=1000), dict(wave_chunk=777, block=64, stack=32),
                                 dict(block=256, stack=32, refill=16), dict(block=64, refill=1)])
@pytest.mark.parametrize("cull,comp", [(1, 1), (1, 0), (0, 0)])
def test_waves_chunks_blocks_stacks(cfg, cull, comp):
    """Chunked waves (the wave size), block sizes and stack depths: per-path
    results must not depend on the configuration."""
    tris = sg.hair(300, 16, True, seed=35)
    rays = sg.pinhole(80, 40)
    g = _gpu_waves(tris, rays, 2, 5, 6, comp, cull, None, sc.SC_LUT_AUTO, **cfg)
    o = _oracle_waves(tris, rays, 2, 5, 6, comp, cull)
    for w in range(3):
        order = np.argsort(o[w]["path"], kind="stable")
        assert np.array_equal(g[w]["path"], np.sort(o[w]["path"])), f"wave {w} {cfg}"
        assert np.array_equal(g[w]["id"], o[w]["id"][order])
        assert np.array_equal(g[w]["counts"], o[w]["counts"][order])


def test_autotuner_returns_a_valid_config():
    tris = sg.hair(300, 16, True, seed=36)
    rays = sg.pinhole(256, 256)
    b = sc.sc_bvh_build(tris, 6, 1)
    d = sc.DeviceBVH(b, sc.SC_LAYOUT_MASKED_COMPACT)
    r = torch.from_numpy(rays).cuda()
    bufs = sc.WaveBuffers(r.shape[0], 2, with_counts=False)
    best, rows = sc.sc_autotune_waves(d, r, 2, 9, 1, bufs, reps=1)
    assert len(rows) >= 9 and best.block in (64, 128, 256) and best.stack in (32, 64)
    assert min(x[-1] for x in rows) > 0
    # the tuned configuration gives the same results as the default one
    b1, s1 = sc.trace_waves(d, r, 2, 9, 1, opts=best)
    b2, s2 = sc.trace_waves(d, r, 2, 9, 1)
    assert list(s1) == list(s2)
    assert torch.equal(b1.hits[0].view(torch.int32), b2.hits[0].view(torch.int32))


@pytest.mark.parametrize("comp,cull", [(1, 1), (0, 1), (0, 0)])
def test_autotuner_considers_the_stack_ring(comp, cull):
    """On images with kernel variants the tuner also times the shared-memory
    stack ring, the 9-block occupancy bound and the shared-memory hit slot
    (block 128, stack 64); whatever it picks traces the same."""
    tris = sg.hair(300, 16, True, seed=37)
    rays = sg.pinhole(128, 128)
    b = sc.sc_bvh_build(tris, 6, comp)
    d = sc.DeviceBVH(b, sc.SC_LAYOUT_MASKED if cull else sc.SC_LAYOUT_PLAIN)
    r = torch.from_numpy(rays).cuda()
    bufs = sc.WaveBuffers(r.shape[0], 2, with_counts=False)
    best, rows = sc.sc_autotune_waves(d, r, 2, 9, cull, bufs, reps=1)
    S, O, H = sc.SC_VARIANT_SSTACK, sc.SC_VARIANT_OCC9, sc.SC_VARIANT_HSLOT
    placed = {S, O, O | S, H, H | O, H | O | S}
    ring = [x for x in rows if x[4] != 0]
    assert {x[4] for x in ring} == placed and all(x[0] == 128 and x[1] == 64 for x in ring)
    assert best.variant in placed | {0}
    others = [sc._opts(block=128, stack=64, variant=v) for v in sorted(placed)]
    for o in [best] + others:
        b1, s1 = sc.trace_waves(d, r, 2, 9, cull, opts=o)
        b2, s2 = sc.trace_waves(d, r, 2, 9, cull)
        assert list(s1) == list(s2)
        for w in range(3):
            m = int(s1[w])
            ia, ib = torch.argsort(b1.path[w][:m]), torch.argsort(b2.path[w][:m])
            assert torch.equal(b1.hits[w][:m].view(torch.int32)[ia],
                               b2.hits[w][:m].view(torch.int32)[ib])


@pytest.mark.parametrize("lut", [sc.SC_LUT_SHARED, sc.SC_LUT_FACTORED_L1, sc.SC_LUT_GLOBAL])
def test_autotuner_with_lookup_modes(lut):
    """The tuner adds its stack / occupancy candidates only where those
    kernels exist for the image and lookup mode; with the factored tables it
    tunes the factored kernels alone, and the result traces the same."""
    tris = sg.hair(300, 16, True, seed=38)
    rays = sg.pinhole(96, 96)
    b = sc.sc_bvh_build(tris, 6, 0)
    d = sc.DeviceBVH(b, sc.SC_LAYOUT_MASKED)
    r = torch.from_numpy(rays).cuda()
    bufs = sc.WaveBuffers(r.shape[0], 2, with_counts=False)
    best, rows = sc.sc_autotune_waves(d, r, 2, 9, 1, bufs, sc._opts(lut_mode=lut), reps=1)
    placed = [x for x in rows if x[4] != 0]
    assert (len(placed) > 0) == (lut == sc.SC_LUT_GLOBAL)
    b1, s1 = sc.trace_waves(d, r, 2, 9, 1, opts=best)
    b2, s2 = sc.trace_waves(d, r, 2, 9, 1)
    assert list(s1) == list(s2)
    for w in range(3):
        m = int(s1[w])
        ia, ib = torch.argsort(b1.path[w][:m]), torch.argsort(b2.path[w][:m])
        assert torch.equal(b1.hits[w][:m].view(torch.int32)[ia],
                           b2.hits[w][:m].view(torch.int32)[ib])


def test_waves_culled_equals_plain_and_sizes():
    tris = sg.hair(800, 16, True, seed=32)
    rays = sg.pinhole(96, 64)
    a = _gpu_waves(tris, rays, 3, 99, 6, 1, 1)
    b = _gpu_waves(tris, rays, 3, 99, 6, 1, 0)
    for w in range(4):
        assert np.array_equal(a[w]["path"], b[w]["path"])
        assert np.array_equal(a[w]["id"], b[w]["id"]) and np.array_equal(a[w]["t"], b[w]["t"])
        assert (a[w]["counts"] <= b[w]["counts"]).all()
    # each wave is compacted: only hits of the previous wave spawn rays
    for w in range(1, 4):
        assert len(a[w]["path"]) == int((b[w - 1]["id"] >= 0).sum())


def test_waves_edge_cases():
    tris = sg.hair(50, 16, False, seed=33)
    b = sc.sc_bvh_build(tris, 6, 0)
    d = sc.DeviceBVH(b, sc.SC_LAYOUT_MASKED)
    # no bounces: same as a plain trace
    rays = sg.pinhole(40, 24)
    r = torch.from_numpy(rays).cuda()
    bufs, sizes = sc.trace_waves(d, r, 0, 1, 1)
    h, c = sc.trace(d, r, 0, 1)
    assert torch.equal(bufs.hits[0].view(torch.int32), h.view(torch.int32))
    # rays that all miss: empty bounce waves
    miss = rays.copy()
    miss[:, 4:7] = [0, 1, 0]
    miss[:, :3] = [0, 5, 0]
    bufs, sizes = sc.trace_waves(d, torch.from_numpy(miss).cuda(), 2, 1, 1)
    assert sizes.tolist() == [len(miss), 0, 0]
    with pytest.raises(sc.SubcullError):
        sc.trace_waves(d, r, sc.SC_MAX_BOUNCES + 1, 1, 1)


def test_wait_timeout_is_reported_and_the_context_survives():
    """Failure detection without a fault: with a 1 ns limit the grid
    barrier between waves gives up at once, every block records the timeout
    and returns, sc_waves_poll reports SC_ERR_TIMEOUT, and the next launch
    on the same context and buffers gives the normal results."""
    tris = sg.hair(2048, 16, True, seed=5)
    rays = sg.pinhole(256, 256)
    b = sc.sc_bvh_build(tris, 6, 0)
    d = sc.DeviceBVH(b, sc.SC_LAYOUT_MASKED)
    r = torch.from_numpy(rays).cuda()
    bufs = sc.WaveBuffers(r.shape[0], 2, with_counts=True)
    sc.sc_trace_waves(d, r, 2, 99, 1, bufs.outs(), bufs.ws, sc._opts(wait_timeout_ns=1))
    with pytest.raises(sc.SubcullError) as e:
        sc.sc_waves_poll(bufs.ws, 2)
    assert e.value.code == sc.SC_ERR_TIMEOUT
    # same context, same buffers, default limit: a normal run
    _, sizes = sc.trace_waves(d, r, 2, 99, 1, bufs)
    ref = sc.WaveBuffers(r.shape[0], 2, with_counts=True)
    _, ref_sizes = sc.trace_waves(d, r, 2, 99, 1, ref)
    torch.cuda.synchronize()
    assert np.array_equal(sizes, ref_sizes) and sizes[1] > 0
    for w in range(3):
        m = int(sizes[w])
        a = bufs.hits[w][:m].cpu().numpy().view(np.int32)
        c = ref.hits[w][:m].cpu().numpy().view(np.int32)
        pa = bufs.path[w][:m].cpu().numpy()
        pc = ref.path[w][:m].cpu().numpy()
        oa, oc = np.argsort(pa, kind="stable"), np.argsort(pc, kind="stable")
        assert np.array_equal(pa[oa], pc[oc]) and np.array_equal(a[oa], c[oc])


@pytest.mark.parametrize("cull,comp,lut", [(0, 0, 0), (1, 0, 0), (1, 1, sc.SC_LUT_BITTABLE),
                                           (1, 1, sc.SC_LUT_GLOBAL)])
@pytest.mark.parametrize("block", [128, 256])
def test_wide_waves_match_oracle(cull, comp, lut, block):
    tris = sg.hair(400, 16, True, seed=31)
    rays = sg.pinhole(64, 48)
    lay = sc.SC_LAYOUT_MASKED4 if cull else sc.SC_LAYOUT_PLAIN4
    g = _gpu_waves(tris, rays, 2, 1234, 6, comp, cull, lay, lut, block=block, stack=64)
    o = _oracle_waves(tris, rays, 2, 1234, 6, comp, cull, width=4)
    for w in range(3):
        assert np.array_equal(g[w]["path"], o[w]["path"]), w
        assert np.array_equal(g[w]["id"], o[w]["id"]), w
        assert np.array_equal(g[w]["t"], o[w]["t"]), w
        assert np.array_equal(g[w]["counts"], o[w]["counts"]), w


def test_waves_host_entry_point_matches_device_pipeline():
    """sc_trace_waves_host (host rays in, each wave's entries copied back)
    gives, per wave, the sizes, paths, hits and counts of sc_trace_waves on
    device buffers."""
    tris = sg.hair(500, 16, True, seed=37)
    rays = sg.pinhole(96, 48)
    b = sc.sc_bvh_build(tris, 6, 1)
    d = sc.DeviceBVH(b, sc.SC_LAYOUT_MASKED)
    r = torch.from_numpy(rays).cuda()
    ref, sizes = sc.trace_waves(d, r, 2, 11, 1)
    torch.cuda.synchronize()
    n = rays.shape[0]
    h_rays = torch.from_numpy(rays).pin_memory()
    h_outs = [(torch.full((n, 4), -9.0).pin_memory(), torch.full((n,), -9, dtype=torch.int32).pin_memory(),
               torch.full((n, 2), -9, dtype=torch.int32).pin_memory(), None) for _ in range(3)]
    bufs = sc.WaveBuffers(n, 2, with_counts=True)
    d_rays = torch.empty((n, 8), dtype=torch.float32, device="cuda")
    got = sc.sc_trace_waves_host(d, h_rays, 2, 11, 1, h_outs, d_rays, bufs.outs(), bufs.ws)
    assert list(got) == list(sizes)
    for w in range(3):
        m = int(sizes[w])
        hp, hh, hc = h_outs[w][1][:m].numpy(), h_outs[w][0][:m].numpy(), h_outs[w][2][:m].numpy()
        rp = ref.path[w][:m].cpu().numpy()
        rh = ref.hits[w][:m].cpu().numpy()
        rc = ref.counts[w][:m].cpu().numpy()
        a, b_ = np.argsort(hp, kind="stable"), np.argsort(rp, kind="stable")
        assert np.array_equal(hp[a], rp[b_])
        assert np.array_equal(hh[a].view(np.int32), rh[b_].view(np.int32))
        assert np.array_equal(hc[a], rc[b_])
        if m < n:
            assert (h_outs[w][1][m:].numpy() == -9).all()  # nothing past the wave
