"""Checks of the seeded input generators against their own definitions
(these produce inputs only; they hold none of the method's arithmetic)."""
import math

import numpy as np

from paper_2305_08343_gb300 import scenegen as sg


def test_elementary_functions():
    for x in np.linspace(-60, 60, 2001):
        s, c = sg.sincos(float(x))
        assert abs(s - math.sin(x)) < 1e-13 and abs(c - math.cos(x)) < 1e-13
    for x in np.linspace(-12, 3, 301):
        assert abs(sg.exp(float(x)) / math.exp(x) - 1) < 1e-14


def test_hair_shape_and_determinism():
    S, G = 50, 16
    a = sg.hair(S, G, True, seed=3)
    b = sg.hair(S, G, True, seed=3)
    assert a.shape == (S * G * 2 + 2, 9) and np.array_equal(a, b)
    assert not np.array_equal(a, sg.hair(S, G, True, seed=4))
    v = a[:-2].reshape(S, G, 2, 3, 3).astype(np.float64)
    # ribbon: A-, A+ of segment k are at the helix point +- half width
    am, ap = v[:, :, 0, 0], v[:, :, 0, 1]
    mid = 0.5 * (am + ap)
    assert np.allclose(np.linalg.norm(ap - am, axis=-1), 1e-3, rtol=1e-3)
    # root point: |n + 0.02 w| with w orthogonal to the unit normal n
    assert np.allclose(np.linalg.norm(mid[:, 0], axis=-1), math.sqrt(1 + 0.02 ** 2), atol=1e-6)
    # consecutive helix samples advance 0.5/16 along n
    n = mid[:, 0] / np.linalg.norm(mid[:, 0], axis=-1, keepdims=True)
    axial = np.einsum("skc,sc->sk", mid, n)
    assert np.allclose(np.diff(axial, axis=1), 0.5 / G, atol=1e-3)
    # ground quad at y = -1.2
    assert np.all(a[-2:].reshape(-1, 3)[:, 1] == np.float32(-1.2))


def test_soup():
    t = sg.soup(2000, seed=3)
    v = t.reshape(-1, 3, 3).astype(np.float64)
    assert (v > -0.11).all() and (v < 1.11).all()
    sl = v[0::2]
    ell = np.linalg.norm(sl[:, 1] - sl[:, 0], axis=-1)
    assert ell.min() >= 0.99e-4 and ell.max() <= 1.01e-1
    h = np.linalg.norm(sl[:, 2] - 0.5 * (sl[:, 0] + sl[:, 1]), axis=-1)
    big = ell > 1e-2  # float32 rounding dominates the 1e-7 heights of tiny slivers
    assert np.allclose(h[big] / ell[big], 1e-3, rtol=2e-2)
    assert ((h / ell) > 5e-4).all() and ((h / ell) < 2e-3).all()
    sb = v[1::2]
    e1 = sb[:, 1] - sb[:, 0]
    e2 = sb[:, 2] - sb[:, 0]
    assert ((np.abs(e1) > 0).sum(1) == 1).all() and ((np.abs(e2) > 0).sum(1) == 1).all()


def test_rays():
    r, pix = sg.pinhole(40, 20, with_pixels=True)
    assert sorted(pix.tolist()) == list(range(800))
    d = r[:, 4:7].astype(np.float64)
    assert np.allclose(np.linalg.norm(d, axis=1), 1, atol=1e-6)
    assert (r[:, :3] == np.array([0, 0, 3], np.float32)).all() and np.isinf(r[:, 7]).all()
    # first 32 rays form one 8x4 tile
    xs, ys = pix[:32] % 40, pix[:32] // 40
    assert xs.max() - xs.min() == 7 and ys.max() - ys.min() == 3
    # vertical field of view 40 degrees: top/bottom rows at +-20 deg (pixel centres)
    top = r[pix == 20][0]
    ang = math.degrees(math.atan2(top[5], -top[6]))
    assert abs(ang - math.degrees(math.atan(math.tan(math.radians(20)) * (1 - 1 / 20)))) < 1e-4
    q = sg.random_rays(5000, seed=7)
    assert (q[:, :3] >= 0).all() and (q[:, :3] < 1).all()
    assert np.allclose(np.linalg.norm(q[:, 4:7].astype(np.float64), axis=1), 1, atol=1e-6)
    assert abs(q[:, 4:7].mean()) < 0.05
    j = sg.pinhole(8, 4, jitter_seed=5)
    assert not np.array_equal(j, sg.pinhole(8, 4))
