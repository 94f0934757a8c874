"""The binned-SAH tree built on the GPU (sc_build_opts.gpu_bvh) is the host
build's tree -- which test_host_vs_oracle.py ties to the oracle's own
builder -- node for node: the root slot, both child slots of every node
(child index or leaf range, triangle count, box) and the triangle order.

The scenes reach both phases of the GPU builder (level-by-level splits of
ranges over 2,048 triangles, and one-warp subtrees below that), leaf sizes
1..8 and 2..32 bins, and the degenerate cases: no triangles, a single leaf,
a single small subtree, equal centroids on every axis (the half split at
every node) and on two axes (one usable axis)."""
import numpy as np
import pytest

from paper_2305_08343_gb300 import scenegen as sg
from paper_2305_08343_gb300 import subcull as sc

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")


def _equal_trees(tris, **kw):
    host = sc.sc_bvh_build(tris, 0, 0, **kw)
    dev = sc.sc_bvh_build(tris, 0, 0, gpu_bvh=1, **kw)
    hi, di = host.info(), dev.info()
    assert (hi.num_nodes, hi.max_depth) == (di.num_nodes, di.max_depth)
    assert list(hi.root_box) == list(di.root_box)
    h, d = host.export(), dev.export()
    assert np.array_equal(h["root"], d["root"])
    for k in ("child", "count", "perm"):
        assert np.array_equal(h[k], d[k]), k
    # boxes by value (a zero bound may differ only in sign)
    assert np.array_equal(h["box"], d["box"])
    return hi, di


def _line(n, seed):
    """Triangles whose centroids differ only in x (one usable axis)."""
    rng = np.random.default_rng(seed)
    x = np.sort(rng.uniform(-1, 1, n)).astype(np.float32)
    t = np.zeros((n, 9), np.float32)
    t[:, 0] = x - 0.01
    t[:, 3] = x + 0.01
    t[:, 6] = x
    t[:, 1], t[:, 4], t[:, 7] = -0.5, -0.5, 0.5
    t[:, 2], t[:, 5], t[:, 8] = -0.5, 0.5, 0.0
    return t[rng.permutation(n)]


SCENES = {
    "hair_ground_65k": lambda: sg.hair(2048, 16, True, seed=1),
    "soup_100k": lambda: sg.soup(100000, seed=8),
    "hair_512": lambda: sg.hair(16, 16, False, seed=3),
}


@pytest.mark.parametrize("scene", sorted(SCENES))
@pytest.mark.parametrize("max_leaf,bins", [(4, 32), (1, 32), (8, 16), (4, 2), (3, 7)])
def test_gpu_tree_equals_host(scene, max_leaf, bins):
    _need_gpu()
    _equal_trees(SCENES[scene](), max_leaf=max_leaf, bins=bins)


@pytest.mark.parametrize("n", [1, 3, 4, 5, 31, 2048, 2049, 6000])
def test_gpu_tree_sizes_at_phase_borders(n):
    _need_gpu()
    _equal_trees(sg.soup(n, seed=n))


def test_gpu_tree_empty():
    _need_gpu()
    b = sc.sc_bvh_build(np.zeros((0, 9), np.float32), 0, 0, gpu_bvh=1)
    assert b.info().num_nodes == 0
    assert list(b.export()["root"]) == [-1, 0]


def test_gpu_tree_equal_centroids_half_splits():
    _need_gpu()
    one = sg.soup(1, seed=4)
    _, di = _equal_trees(np.repeat(one, 5000, axis=0))
    assert di.num_nodes > 1000


def test_gpu_tree_one_usable_axis():
    _need_gpu()
    _equal_trees(_line(20000, seed=6))
    _equal_trees(_line(700, seed=7), max_leaf=2, bins=5)


def test_gpu_tree_feeds_masks_compression_and_traversal():
    """The GPU tree with GPU masks and compression gives the host build's
    masks, LUT and hits (the masks' level order uses each node's depth)."""
    _need_gpu()
    tris = sg.hair(1024, 16, True, seed=5)
    a = sc.sc_bvh_build(tris, 6, 1)
    b = sc.sc_bvh_build(tris, 6, 1, gpu_bvh=1, gpu_masks=1)
    ea, eb = a.export(), b.export()
    for k in ("child", "count", "perm", "masks", "clut", "cidx"):
        assert np.array_equal(ea[k], eb[k]), k
    rays = torch.from_numpy(sg.pinhole(96, 64)).cuda()
    ha, ca = sc.trace(sc.DeviceBVH(a, sc.SC_LAYOUT_MASKED), rays, sc.SC_CLOSEST, 2)
    hb, cb = sc.trace(sc.DeviceBVH(b, sc.SC_LAYOUT_MASKED), rays, sc.SC_CLOSEST, 2)
    torch.cuda.synchronize()
    assert torch.equal(ha.view(torch.int32), hb.view(torch.int32))
    assert torch.equal(ca, cb)


def test_gpu_tree_full_size_hair12m():
    """12,100,000 hair triangles: the same tree, and the build time of both."""
    _need_gpu()
    tris = sg.hair(378125, 16, False, seed=4)
    hi, di = _equal_trees(tris)
    print(f"\n12.1M tree: host {hi.ms_bvh:.0f} ms, GPU {di.ms_bvh:.0f} ms, "
          f"{di.num_nodes} nodes, depth {di.max_depth}")
