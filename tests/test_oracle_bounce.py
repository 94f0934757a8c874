"""Pins of the oracle's diffuse bounce rays (wave workloads; not in the
paper): the counter-based hash of Jarzynski & Olano (JCGT 2020) and
cosine-weighted directions about the geometric normal."""
import numpy as np

import oracle


def test_hash_is_a_permutation_sample():
    # the hash is a composition of bijections of 32-bit words (LCG step,
    # xorshift, odd multiply, xorshift), so distinct inputs never collide
    v = [oracle.pcg_hash(i) for i in range(1 << 16)]
    assert len(set(v)) == 1 << 16
    u = np.array(v, np.float64) / 2 ** 32
    assert abs(u.mean() - 0.5) < 0.01 and abs(u.var() - 1 / 12) < 0.005


def test_bounce_geometry_and_cosine_distribution():
    tri = np.array([0, 0, 0, 1, 0, 0, 0, 1, 0], np.float32)   # plane z = 0, normal +z
    ray = np.array([0.2, 0.3, 1, 0, 0, 0, -1, np.inf], np.float32)
    cos = []
    for rid in range(20000):
        b = oracle.bounce(ray, 1.0, tri, 7, rid, 1)
        assert b is not None
        assert b[0] == np.float32(0.2) and b[1] == np.float32(0.3) and b[2] == 0.0
        assert b[3] == np.float32(1e-4) and np.isinf(b[7])
        d = b[4:7].astype(np.float64)
        assert abs(np.linalg.norm(d) - 1) < 1e-6
        cos.append(d[2])
    cos = np.array(cos)
    assert (cos >= 0).all()                       # hemisphere facing the incoming ray
    assert abs(cos.mean() - 2 / 3) < 0.01         # E[cos] of a cosine-weighted lobe
    # cos^2 = 1 - |disk point|^2 is uniform on [0, 1] for a uniform disk point
    h, _ = np.histogram(cos ** 2, bins=10, range=(0, 1))
    assert (np.abs(h / len(cos) - 0.1) < 0.01).all()
    # from below the normal flips (direction faces the incoming side)
    ray_b = np.array([0.2, 0.3, -1, 0, 0, 0, 1, np.inf], np.float32)
    b = oracle.bounce(ray_b, 1.0, tri, 7, 5, 1)
    assert b[6] <= 0


def test_bounce_degenerate_and_streams():
    deg = np.array([0, 0, 0, 1, 1, 1, 2, 2, 2], np.float32)
    ray = np.array([0, 0, 1, 0, 0, 0, -1, np.inf], np.float32)
    assert oracle.bounce(ray, 1.0, deg, 1, 0, 1) is None
    tri = np.array([0, 0, 0, 1, 0, 0, 0, 1, 0], np.float32)
    a = oracle.bounce(ray, 1.0, tri, 1, 3, 1)
    assert np.array_equal(a, oracle.bounce(ray, 1.0, tri, 1, 3, 1))   # deterministic
    assert not np.array_equal(a, oracle.bounce(ray, 1.0, tri, 1, 4, 1))  # per path
    assert not np.array_equal(a, oracle.bounce(ray, 1.0, tri, 1, 3, 2))  # per bounce
    assert not np.array_equal(a, oracle.bounce(ray, 1.0, tri, 2, 3, 1))  # per seed
