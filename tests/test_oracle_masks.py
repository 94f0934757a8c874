"""Pins of the oracle's object masks (Sec. 3.1.1 voxelization, Sec. 3.2.1 /
Alg. 2 hierarchical fill, the L parameter).

Independent facts used:
  * triangle-box overlap by polygon clipping (Sutherland-Hodgman) instead of
    separating axes;
  * dense barycentric samples of the triangle (every sampled point's cells
    must be set: conservativeness);
  * Alg. 2 invariant: every parent cell touching an occupied child voxel is
    filled;
  * L = infinity equals direct voxelization of every descendant triangle
    (Sec. 3.2.1), and every finite L is a superset of it.
"""
import numpy as np
import pytest

import oracle
from paper_2305_08343_gb300 import scenegen as sg


def clip_nonempty(tri, bmin, bmax, grow=0.0):
    """Clip the triangle polygon by the six half-spaces of the box."""
    poly = [np.asarray(p, np.float64) for p in tri.reshape(3, 3)]
    for k in range(3):
        for sgn, bound in ((1.0, bmin[k] - grow), (-1.0, bmax[k] + grow)):
            out = []
            n = len(poly)
            for i in range(n):
                a, b = poly[i], poly[(i + 1) % n]
                fa, fb = sgn * (a[k] - bound), sgn * (b[k] - bound)
                if fa >= 0:
                    out.append(a)
                if (fa >= 0) != (fb >= 0):
                    t = fa / (fa - fb)
                    out.append(a + t * (b - a))
            poly = out
            if not poly:
                return False
    return True


def test_tri_box_vs_clipping():
    rng = np.random.default_rng(0)
    bmin, bmax = np.zeros(3), np.ones(3)
    disagree = 0
    for i in range(3000):
        kind = i % 3
        if kind == 0:
            tri = rng.uniform(-0.6, 1.6, 9)
        elif kind == 1:  # thin sliver near the box
            a = rng.uniform(-0.3, 1.3, 3)
            d = rng.normal(size=3)
            w = rng.normal(size=3)
            tri = np.concatenate([a, a + d, a + 0.5 * d + 1e-3 * w])
        else:  # axis-aligned triangle
            tri = rng.uniform(-0.6, 1.6, 9)
            k = rng.integers(0, 3)
            tri.reshape(3, 3)[:, k] = rng.uniform(-0.2, 1.2)
        sat = oracle.tri_box(tri, bmin, bmax)
        clip = clip_nonempty(tri, bmin, bmax)
        if sat != clip:
            # only grazing contacts may differ between the two methods
            assert clip_nonempty(tri, bmin, bmax, 1e-9) and not clip_nonempty(tri, bmin, bmax, -1e-9)
            disagree += 1
    assert disagree <= 3


def test_tri_box_touching_counts():
    # triangle in the plane x = 1 touching the face of the unit box
    tri = np.array([1, 0.2, 0.2, 1, 0.8, 0.2, 1, 0.5, 0.8], np.float64)
    assert oracle.tri_box(tri, np.zeros(3), np.ones(3))
    tri2 = tri.copy()
    tri2[0::3] = 1.0 + 1e-9
    assert not oracle.tri_box(tri2, np.zeros(3), np.ones(3))


def _voxel_boxes(lo, hi, R, eps):
    lo = lo.astype(np.float64)
    ext = hi.astype(np.float64) - lo
    i = np.arange(R + 1)
    edges = lo[:, None] + (ext[:, None] * i[None, :]) / R  # (3, R+1)
    return edges[:, :-1] - eps, edges[:, 1:] + eps


def _samples(tri, n=40):
    a, b = np.meshgrid(np.linspace(0, 1, n), np.linspace(0, 1, n))
    m = a + b <= 1
    a, b = a[m], b[m]
    v = tri.reshape(3, 3).astype(np.float64)
    return v[0] + a[:, None] * (v[1] - v[0]) + b[:, None] * (v[2] - v[0])


@pytest.mark.parametrize("R", [4, 6, 8])
@pytest.mark.parametrize("eps", [0.0, 1e-3])
def test_voxelize_covers_samples_and_is_tight(R, eps):
    rng = np.random.default_rng(R)
    for it in range(40):
        tri = rng.uniform(0, 1, 9).astype(np.float32)
        if it % 4 == 0:
            tri.reshape(3, 3)[:, it % 3] = np.float32(0.5)  # axis-aligned
        lo = tri.reshape(3, 3).min(0) - rng.uniform(0, 0.2, 3).astype(np.float32)
        hi = tri.reshape(3, 3).max(0) + rng.uniform(0, 0.2, 3).astype(np.float32)
        m = oracle.voxelize(tri, lo, hi, R, eps)
        bits = np.unpackbits(m.view(np.uint8), bitorder="little")[: R ** 3].astype(bool)
        b0, b1 = _voxel_boxes(lo, hi, R, eps)
        pts = _samples(tri)
        inside = [(pts[:, k, None] >= b0[k][None, :]) & (pts[:, k, None] <= b1[k][None, :])
                  for k in range(3)]
        # cell (x,y,z) contains point p if all three axes do
        cont = (inside[0][:, None, None, :] & inside[1][:, None, :, None]
                & inside[2][:, :, None, None]).reshape(len(pts), -1)
        assert not (cont & ~bits[None, :]).any(), "a sample's cell is not set"
        # tightness: each set voxel really overlaps the triangle (clipping)
        for v in np.nonzero(bits)[0]:
            x, y, z = v % R, (v // R) % R, v // (R * R)
            bmin = np.array([b0[0][x], b0[1][y], b0[2][z]])
            bmax = np.array([b1[0][x], b1[1][y], b1[2][z]])
            assert clip_nonempty(tri.astype(np.float64), bmin, bmax, 1e-9)


def test_boundary_plane_sets_both_layers():
    # A triangle lying exactly on the plane between layers 1 and 2 (R = 4,
    # box [0,4]^3) touches both layers.
    R = 4
    tri = np.array([0.5, 2.0, 0.5, 3.5, 2.0, 0.5, 0.5, 2.0, 3.5], np.float32)
    m = oracle.voxelize(tri, np.zeros(3, np.float32), np.full(3, 4, np.float32), R, 0.0)
    bits = np.unpackbits(m.view(np.uint8), bitorder="little")[: R ** 3].reshape(R, R, R)
    assert bits[:, 1, :].any() and bits[:, 2, :].any()
    assert not bits[:, 0, :].any() and not bits[:, 3, :].any()


@pytest.mark.parametrize("R", [4, 6])
@pytest.mark.parametrize("eps", [0.0, 2e-3])
def test_fill_covers_child_voxels(R, eps):
    """Alg. 2: each occupied child voxel fills every parent cell it touches
    (its eps-neighbourhood, with eps > 0)."""
    rng = np.random.default_rng(7 + R)
    for it in range(30):
        plo = rng.uniform(-1, 0, 3).astype(np.float32)
        phi = (plo + rng.uniform(0.5, 2, 3)).astype(np.float32)
        clo = (plo + (phi - plo) * rng.uniform(0, 0.5, 3)).astype(np.float32)
        chi = (clo + (phi - clo) * rng.uniform(0.05, 1, 3)).astype(np.float32)
        cm = rng.integers(0, 2 ** 32, oracle.mask_words(R), dtype=np.uint64).astype(np.uint32)
        cm &= rng.integers(0, 2 ** 32, cm.shape, dtype=np.uint64).astype(np.uint32)
        pm = oracle.fill(np.zeros_like(cm), plo, phi, cm, clo, chi, R, eps)
        cb = np.unpackbits(cm.view(np.uint8), bitorder="little")[: R ** 3].astype(bool)
        pb = np.unpackbits(pm.view(np.uint8), bitorder="little")[: R ** 3].astype(bool)
        c0, c1 = _voxel_boxes(clo, chi, R, 0.0)
        p0, p1 = _voxel_boxes(plo, phi, R, 0.0)
        for v in np.nonzero(cb)[0]:
            x, y, z = v % R, (v // R) % R, v // (R * R)
            vmin = np.array([c0[0][x], c0[1][y], c0[2][z]]) - eps * 0.999
            vmax = np.array([c1[0][x], c1[1][y], c1[2][z]]) + eps * 0.999
            pts = vmin + rng.uniform(0, 1, (64, 3)) * (vmax - vmin)
            pts = np.vstack([pts, vmin, vmax])
            for p in pts:
                if (p < plo).any() or (p > phi).any():
                    continue
                cells = [np.nonzero((p[k] >= p0[k]) & (p[k] <= p1[k]))[0] for k in range(3)]
                for cx in cells[0]:
                    for cy in cells[1]:
                        for cz in cells[2]:
                            assert pb[cx + R * cy + R * R * cz]


def test_fill_flat_parent_axis_fills_all_layers():
    R = 4
    plo = np.array([0, 0, 0], np.float32)
    phi = np.array([1, 0, 1], np.float32)  # flat in y
    cm = np.zeros(oracle.mask_words(R), np.uint32)
    cm[0] = 1  # voxel (0,0,0)
    pm = oracle.fill(np.zeros_like(cm), plo, phi, cm, plo, phi, R, 0.0)
    pb = np.unpackbits(pm.view(np.uint8), bitorder="little")[: R ** 3].reshape(R, R, R)
    assert pb[0, :, 0].all()  # [z, y, x]


def _slot_tris(child, count, perm, node, c):
    """Triangle positions below slot (node, c)."""
    out = []
    stack = [(int(child[node, c]), int(count[node, c]))]
    while stack:
        ch, n = stack.pop()
        if n > 0:
            out.extend(perm[ch:ch + n])
        else:
            stack.append((int(child[ch, 0]), int(count[ch, 0])))
            stack.append((int(child[ch, 1]), int(count[ch, 1])))
    return out


@pytest.mark.parametrize("R", [4, 6])
def test_L_infinity_is_exact_and_L_is_superset(R):
    tris = sg.hair(24, 16, False, seed=5)
    b_inf = oracle.OracleBVH(tris).build_masks(R, L=64)
    m_inf = b_inf.masks()
    child, count, box = b_inf.nodes()
    perm = b_inf.perm()
    eps = b_inf.eps
    for node in range(b_inf.num_nodes):
        for c in range(2):
            direct = np.zeros(oracle.mask_words(R), np.uint32)
            for t in _slot_tris(child, count, perm, node, c):
                oracle.voxelize(tris[t], box[node, c, :3], box[node, c, 3:], R, eps, direct)
            assert np.array_equal(direct, m_inf[node, c])
    for L in (1, 2, 3):
        mL = oracle.OracleBVH(tris).build_masks(R, L=L).masks()
        assert not (m_inf & ~mL).any(), f"L={L} is not a superset of the exact mask"
    # L = 1 fills from direct children only: coarser on average
    m1 = oracle.OracleBVH(tris).build_masks(R, L=1).masks()
    pc = lambda m: np.unpackbits(m.view(np.uint8)).sum()
    assert pc(m1) >= pc(m_inf)


def test_triangle_mask_covers_triangle_in_all_ancestors():
    """C9 invariant: for every ancestor slot of a triangle, the slot's mask
    covers densely sampled points of the triangle (L = 3, R = 6)."""
    R = 6
    tris = sg.hair(16, 16, True, seed=6)
    b = oracle.OracleBVH(tris).build_masks(R, L=3)
    m = b.masks()
    child, count, box = b.nodes()
    perm = b.perm()
    for node in range(b.num_nodes):
        for c in range(2):
            bits = np.unpackbits(m[node, c].view(np.uint8), bitorder="little")[: R ** 3].astype(bool)
            lo, hi = box[node, c, :3], box[node, c, 3:]
            e0, e1 = _voxel_boxes(lo, hi, R, 0.0)
            for t in _slot_tris(child, count, perm, node, c)[::3]:
                for p in _samples(tris[t], 8):
                    idx = []
                    for k in range(3):
                        ii = np.nonzero((p[k] >= e0[k]) & (p[k] <= e1[k]))[0]
                        if len(ii) == 0:  # flat or rounding: nearest layer
                            ii = [int(np.clip(np.searchsorted(e0[k], p[k]) - 1, 0, R - 1))]
                        idx.append(ii)
                    assert any(bits[x + R * y + R * R * z]
                               for x in idx[0] for y in idx[1] for z in idx[2])
