"""Kernel variants (sc_trace_opts.variant) against the CPU oracle.

The load-scheduling, stack and bounce-sort options must not change any
result: hit ids, t, u, v and per-ray node and triangle test counts are
compared element by element with the oracle's traversal (Alg. 4 with the
Alg. 1 cells as written).  The fused cell option is compared with the
oracle's fused mode (set_cellform(1)).  Single batches and the wave
pipeline (by path id, several chunks), culled with compressed masks and the
bit table, culled with uncompressed masks and the full table, and plain.
"""
import numpy as np
import pytest

import oracle
from paper_2305_08343_gb300 import scenegen as sg
from paper_2305_08343_gb300 import subcull as sc

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

F, P, S, T, O, D = (sc.SC_VARIANT_FUSED_CELLS, sc.SC_VARIANT_PAIR, sc.SC_VARIANT_SPEC,
                    sc.SC_VARIANT_TOS, sc.SC_VARIANT_SORT, sc.SC_VARIANT_DEFER)
VARIANTS = [F, P, S, T, S | T, O, S | T | O, F | S | T | O, D, sc.SC_VARIANT_LAZY,
            sc.SC_VARIANT_SSTACK, sc.SC_VARIANT_TABLE_L1, sc.SC_VARIANT_OCC9,
            sc.SC_VARIANT_OCC9 | sc.SC_VARIANT_SSTACK, sc.SC_VARIANT_OCC10,
            sc.SC_VARIANT_OCC10 | sc.SC_VARIANT_SSTACK, sc.SC_VARIANT_HSLOT,
            sc.SC_VARIANT_HSLOT | sc.SC_VARIANT_OCC9,
            sc.SC_VARIANT_HSLOT | sc.SC_VARIANT_OCC9 | sc.SC_VARIANT_SSTACK]
# (cull mode of the oracle, compressed, lookup)
CONFIGS = [(2, 1, sc.SC_LUT_BITTABLE), (1, 0, sc.SC_LUT_GLOBAL), (0, 0, sc.SC_LUT_AUTO)]


@pytest.fixture(scope="module")
def scene():
    tris = sg.hair(600, 16, True, seed=41)
    return tris, sg.pinhole(72, 40)


def _oracle(tris, comp, cull, fused):
    ob = oracle.OracleBVH(tris)
    if cull:
        ob.build_masks(6, 3)
        if comp:
            ob.compress(256, 8)
        ob.set_cellform(1 if fused else 0)
    return ob


def _device(tris, comp, cull):
    b = sc.sc_bvh_build(tris, 6 if cull else 0, comp)
    return sc.DeviceBVH(b, sc.SC_LAYOUT_MASKED if cull else sc.SC_LAYOUT_PLAIN)


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("cull,comp,lut", CONFIGS)
@pytest.mark.parametrize("mode", [sc.SC_CLOSEST, sc.SC_ANY])
def test_single_batch_variants_match_oracle(scene, variant, cull, comp, lut, mode):
    tris, rays = scene
    ob = _oracle(tris, comp, cull, variant & F)
    o = ob.trace(rays, mode, cull)
    d = _device(tris, comp, cull)
    r = torch.from_numpy(rays).cuda()
    hits, counts = sc.trace(d, r, mode, 1 if cull else 0,
                            opts=sc._opts(lut_mode=lut, variant=variant))
    torch.cuda.synchronize()
    t, i, u, v = sc.split_hits(hits)
    cnt = counts.cpu().numpy().view(np.uint32)
    assert np.array_equal(i, o["id"])
    assert np.array_equal(cnt, o["counts"])
    assert np.array_equal(t, o["t"])
    assert np.array_equal(np.stack([u, v], 1), o["uv"])


def _oracle_waves(ob, tris, rays, bounces, seed, cull):
    cur, path = rays, np.arange(len(rays))
    out = []
    for w in range(bounces + 1):
        o = ob.trace(cur, 0, cull)
        out.append(dict(path=path, **o))
        if w < bounces:
            cur, path = oracle.bounce_wave(cur, o["t"], o["id"], tris, seed, w + 1, path)
    return out


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("cull,comp,lut", CONFIGS)
@pytest.mark.parametrize("chunk", [0, 1100])
def test_wave_variants_match_oracle(scene, variant, cull, comp, lut, chunk):
    tris, rays = scene
    ob = _oracle(tris, comp, cull, variant & F)
    o = _oracle_waves(ob, tris, rays, 2, 4321, cull)
    d = _device(tris, comp, cull)
    r = torch.from_numpy(rays).cuda()
    bufs, sizes = sc.trace_waves(d, r, 2, 4321, 1 if cull else 0,
                                 opts=sc._opts(lut_mode=lut, variant=variant, wave_chunk=chunk))
    torch.cuda.synchronize()
    for w in range(3):
        m = int(sizes[w])
        t, i, _, _ = sc.split_hits(bufs.hits[w][:m])
        path = bufs.path[w][:m].cpu().numpy()
        cnt = bufs.counts[w][:m].cpu().numpy().view(np.uint32)
        g = np.argsort(path, kind="stable")
        k = np.argsort(o[w]["path"], kind="stable")
        assert np.array_equal(path[g], o[w]["path"][k]), f"wave {w}: different rays"
        assert np.array_equal(i[g], o[w]["id"][k]), f"wave {w}: hit ids differ"
        assert np.array_equal(cnt[g], o[w]["counts"][k]), f"wave {w}: counts differ"
        assert np.array_equal(t[g], o[w]["t"][k])
    assert int(sizes[1]) > 200 and int(sizes[2]) > 20


def test_unbuilt_variants_are_rejected(scene):
    tris, rays = scene
    r = torch.from_numpy(rays).cuda()
    b = sc.sc_bvh_build(tris, 4, 0)
    d = sc.DeviceBVH(b, sc.SC_LAYOUT_MASKED)
    with pytest.raises(sc.SubcullError) as e:
        sc.trace(d, r, sc.SC_CLOSEST, 1, opts=sc._opts(variant=sc.SC_VARIANT_SPEC))
    assert e.value.code == -6  # SC_ERR_UNSUPPORTED
    d6 = _device(tris, 1, 1)
    with pytest.raises(sc.SubcullError) as e:
        sc.trace(d6, r, sc.SC_CLOSEST, 1, opts=sc._opts(variant=sc.SC_VARIANT_PAIR | 64))
    assert e.value.code == -6
    with pytest.raises(sc.SubcullError) as e:
        sc.trace_waves(d6, r, 1, 1, 1, opts=sc._opts(variant=sc.SC_VARIANT_SPEC, block=256))
    assert e.value.code == -6
