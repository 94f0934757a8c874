"""Plain CPU oracle for BVH traversal with subspace culling.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py`` (its CPU-baseline leg and ``--impl reference``) may import this
package.  It wraps ``oracle.c``, a slow, direct restatement of the paper
(Yoshimura & Harada, "Subspace Culling for Ray-Box Intersection", 2023) that
shares no code with the GPU path, and the fp64 numpy MLP reference in
``oracle/mlp.py``.

Functions whose result is not pinned to an independent fact by a test are
listed here: none (every function below is exercised against brute force, a
closed form, an invariant or a second method in ``tests/test_oracle_*.py``).
"""
from __future__ import annotations

import ctypes as C
import os
import platform
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", platform.machine() or "unknown", "liboracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-pthread", "-ffp-contract=off",
          "-fno-fast-math", "-fno-strict-aliasing"]


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_build/liboracle.so (gcc, plain C)."""
    src = os.path.join(_HERE, "oracle.c")
    hdr = os.path.join(_HERE, "oracle.h")
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= max(os.path.getmtime(src), os.path.getmtime(hdr))):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", *CFLAGS, src, "-o", tmp, "-lm", "-lpthread"])
    os.replace(tmp, _SO)
    return _SO


def _P(t):
    return C.POINTER(t)


def lib():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        L = C.CDLL(build())
        f, d, i32, i64, u32, u8 = (C.c_float, C.c_double, C.c_int32, C.c_int64,
                                   C.c_uint32, C.c_uint8)
        vp = C.c_void_p
        sig = {
            "or_mask_words": (C.c_int, [C.c_int]),
            "or_raylut_cell": (C.c_int, [C.c_int, _P(C.c_int), _P(C.c_int), _P(C.c_int)]),
            "or_raylut": (None, [C.c_int, _P(u32)]),
            "or_raylut2r_rows": (None, [C.c_int, i64, i64, _P(u32)]),
            "or_cell2_t": (C.c_int, [f, f, f, f, f, C.c_int]),
            "or_bvh_set_raylut2r": (None, [vp, _P(u32)]),
            "or_bvh_refit": (C.c_int, [vp, _P(f)]),
            "or_bvh_reencode": (C.c_int, [vp]),
            "or_tri_box": (C.c_int, [_P(d), _P(d), _P(d)]),
            "or_voxelize": (None, [_P(f), _P(f), _P(f), C.c_int, d, _P(u32)]),
            "or_fill": (None, [_P(u32), _P(f), _P(f), _P(u32), _P(f), _P(f), C.c_int, d]),
            "or_clut_build": (C.c_int, [_P(u32), _P(f), i64, C.c_int, C.c_int, _P(u32), _P(d)]),
            "or_req_luts": (None, [_P(u32), C.c_int, C.c_int, C.c_int, _P(u32)]),
            "or_encode": (C.c_int, [_P(u32), _P(u32), C.c_int, C.c_int]),
            "or_encode_naive": (C.c_int, [_P(u32), _P(u32), C.c_int, C.c_int]),
            "or_bvh_build": (vp, [_P(f), i64, C.c_int, C.c_int]),
            "or_bvh_free": (None, [vp]),
            "or_bvh_num_nodes": (i64, [vp]),
            "or_bvh_max_depth": (C.c_int, [vp]),
            "or_bvh_root": (None, [vp, _P(i32), _P(i32), _P(f)]),
            "or_bvh_nodes": (None, [vp, _P(i32), _P(i32), _P(f)]),
            "or_bvh_perm": (None, [vp, _P(i32)]),
            "or_bvh_sah": (d, [vp, d, d]),
            "or_scene_eps": (d, [_P(f), i64, d]),
            "or_bvh_masks": (C.c_int, [vp, _P(f), C.c_int, C.c_int, d]),
            "or_bvh_get_masks": (None, [vp, _P(u32)]),
            "or_bvh_compress": (C.c_int, [vp, C.c_int, C.c_int]),
            "or_bvh_get_clut": (None, [vp, _P(u32), _P(u8)]),
            "or_trace_range": (C.c_int, [vp, _P(f), _P(f), i64, i64, C.c_int, C.c_int,
                                         C.c_int, C.c_int, C.c_int, _P(f), _P(i32), _P(f),
                                         _P(u32), _P(u32)]),
            "or_brute": (None, [_P(f), i64, _P(f), i64, C.c_int, _P(f), _P(i32), _P(f)]),
            "or_ray_tri": (C.c_int, [_P(f), _P(f), f, _P(f), _P(f), _P(f)]),
            "or_slab": (C.c_int, [_P(f), _P(f), f, _P(f), _P(f)]),
            "or_cell": (C.c_int, [f, f, f, C.c_int]),
            "or_cell_t": (C.c_int, [f, f, f, f, f, C.c_int]),
            "or_cell_at": (C.c_int, [f, f, f, f, f, C.c_int]),
            "or_cell2_at": (C.c_int, [f, f, f, f, f, C.c_int, C.c_int]),
            "or_bvh_set_cellform": (None, [vp, C.c_int]),
            "or_set_threads": (None, [C.c_int, i64]),
            "or_bvh_frontier": (C.c_int, [vp, C.c_int, _P(i32), _P(i32), _P(f), _P(u8)]),
            "or_trace_seeded": (C.c_int, [vp, _P(f), _P(f), i64, C.c_int, C.c_int, C.c_int,
                                          C.c_int, _P(i32), _P(i32), _P(i32), _P(f), C.c_int,
                                          _P(f),
                                          _P(i32), _P(f), _P(u32)]),
            "or_bvh_set_ideal": (None, [vp, C.c_int]),
            "or_bvh_wide": (i64, [vp]),
            "or_bvh_wide_export": (None, [vp, _P(i32), _P(i64), _P(i32), _P(i64)]),
            "or_trace4_range": (C.c_int, [vp, _P(f), _P(f), i64, i64, C.c_int, C.c_int,
                                          C.c_int, C.c_int, C.c_int, _P(f), _P(i32), _P(f),
                                          _P(u32), _P(u32)]),
            "or_pcg_hash": (u32, [u32]),
            "or_bounce_hash": (u32, [u32, u32, u32, u32]),
            "or_bounce": (C.c_int, [_P(f), f, _P(f), u32, u32, u32, _P(f)]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
        return L


def _ptr(a: np.ndarray, t):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_P(t))


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def set_threads(threads: int = 0, task_tris: int = 0):
    """Threads of the oracle's build (0: every online core) and the largest
    triangle range built as one subtree task (0: automatic).  Results do not
    depend on either."""
    lib().or_set_threads(int(threads), int(task_tris))


def mask_words(R: int) -> int:
    return (R * R * R + 31) // 32


# ------------------------------------------------------------ ray-mask LUT --

def raylut_cell(R: int, b, e, v) -> bool:
    arr = [(C.c_int * 3)(*map(int, x)) for x in (b, e, v)]
    return bool(lib().or_raylut_cell(R, *arr))


def raylut(R: int) -> np.ndarray:
    """Full ray-mask table, uint32[R^3 * R^3, W]; row = beg * R^3 + end."""
    R3 = R ** 3
    out = np.zeros((R3 * R3, mask_words(R)), dtype=np.uint32)
    lib().or_raylut(R, _ptr(out, C.c_uint32))
    return out


_LUT2R = {}


def raylut2r(R: int, threads: int = 0) -> np.ndarray:
    """Ray-mask table at R_ray = 2R (Sec. 4.2), uint32[(2R)^6, W]: row
    beg * (2R)^3 + end, beg and end cells of the 2R grid, each row an
    R^3-bit mask.  Rows are split across threads; the table is kept per R."""
    if R in _LUT2R:
        return _LUT2R[R]
    from concurrent.futures import ThreadPoolExecutor
    rows = (2 * R) ** 6
    out = np.zeros((rows, mask_words(R)), dtype=np.uint32)
    nt = threads or (os.cpu_count() or 1)
    cuts = np.linspace(0, rows, nt + 1).astype(np.int64)
    with ThreadPoolExecutor(nt) as ex:
        list(ex.map(lambda i: lib().or_raylut2r_rows(R, int(cuts[i]), int(cuts[i + 1]),
                                                     _ptr(out, C.c_uint32)), range(nt)))
    _LUT2R[R] = out
    return out


# ------------------------------------------------------------- voxel masks --

def tri_box(tri9, bmin, bmax) -> bool:
    t = np.ascontiguousarray(tri9, dtype=np.float64).reshape(9)
    lo = np.ascontiguousarray(bmin, dtype=np.float64)
    hi = np.ascontiguousarray(bmax, dtype=np.float64)
    return bool(lib().or_tri_box(_ptr(t, C.c_double), _ptr(lo, C.c_double),
                                 _ptr(hi, C.c_double)))


def voxelize(tri9, lo, hi, R: int, eps: float, mask: np.ndarray | None = None):
    m = np.zeros(mask_words(R), np.uint32) if mask is None else mask
    t, l, h = _f32(tri9).reshape(9), _f32(lo), _f32(hi)
    lib().or_voxelize(_ptr(t, C.c_float), _ptr(l, C.c_float), _ptr(h, C.c_float),
                      R, float(eps), _ptr(m, C.c_uint32))
    return m


def fill(mask, plo, phi, cmask, clo, chi, R: int, eps: float):
    cm = np.ascontiguousarray(cmask, dtype=np.uint32)
    a = [_f32(x) for x in (plo, phi, clo, chi)]
    lib().or_fill(_ptr(mask, C.c_uint32), _ptr(a[0], C.c_float), _ptr(a[1], C.c_float),
                  _ptr(cm, C.c_uint32), _ptr(a[2], C.c_float), _ptr(a[3], C.c_float),
                  R, float(eps))
    return mask


# ------------------------------------------------------------- compression --

def clut_build(masks: np.ndarray, boxes: np.ndarray, R: int, K: int = 256):
    W = mask_words(R)
    m = np.ascontiguousarray(masks, dtype=np.uint32).reshape(-1, W)
    bx = _f32(boxes).reshape(-1, 6)
    out = np.zeros((K, W), np.uint32)
    imp = np.zeros(K, np.float64)
    k = lib().or_clut_build(_ptr(m, C.c_uint32), _ptr(bx, C.c_float), m.shape[0], R, K,
                            _ptr(out, C.c_uint32), _ptr(imp, C.c_double))
    return out[:k].copy(), imp[:k].copy()


def req_luts(clut: np.ndarray, R: int, b: int = 8) -> np.ndarray:
    nchunk = -(-R ** 3 // b)
    out = np.zeros((nchunk, 1 << b, 8), np.uint32)
    c = np.ascontiguousarray(clut, dtype=np.uint32)
    lib().or_req_luts(_ptr(c, C.c_uint32), c.shape[0], R, b, _ptr(out, C.c_uint32))
    return out


def encode(mask, req, R: int, b: int = 8) -> int:
    m = np.ascontiguousarray(mask, dtype=np.uint32)
    return int(lib().or_encode(_ptr(m, C.c_uint32), _ptr(req, C.c_uint32), R, b))


def encode_naive(mask, clut, R: int) -> int:
    m = np.ascontiguousarray(mask, dtype=np.uint32)
    c = np.ascontiguousarray(clut, dtype=np.uint32)
    return int(lib().or_encode_naive(_ptr(m, C.c_uint32), _ptr(c, C.c_uint32),
                                     c.shape[0], R))


# ---------------------------------------------------------------- BVH + trace --

class OracleBVH:
    """Binned-SAH BVH2 with object masks, built and traced by the oracle."""

    def __init__(self, tris: np.ndarray, max_leaf: int = 4, bins: int = 32):
        self.tris = _f32(tris).reshape(-1, 9)
        self.ntri = self.tris.shape[0]
        self._h = lib().or_bvh_build(_ptr(self.tris, C.c_float), self.ntri, max_leaf, bins)
        self.R = 0
        self.K = 0

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().or_bvh_free(h)
            self._h = None

    @property
    def num_nodes(self) -> int:
        return int(lib().or_bvh_num_nodes(self._h))

    @property
    def max_depth(self) -> int:
        return int(lib().or_bvh_max_depth(self._h))

    def root(self):
        c, n = C.c_int32(), C.c_int32()
        box = np.zeros(6, np.float32)
        lib().or_bvh_root(self._h, C.byref(c), C.byref(n), _ptr(box, C.c_float))
        return c.value, n.value, box

    def nodes(self):
        nn = self.num_nodes
        child = np.zeros((nn, 2), np.int32)
        count = np.zeros((nn, 2), np.int32)
        box = np.zeros((nn, 2, 6), np.float32)
        if nn:
            lib().or_bvh_nodes(self._h, _ptr(child, C.c_int32), _ptr(count, C.c_int32),
                               _ptr(box, C.c_float))
        return child, count, box

    def perm(self):
        p = np.zeros(max(self.ntri, 1), np.int32)
        lib().or_bvh_perm(self._h, _ptr(p, C.c_int32))
        return p[: self.ntri]

    def sah(self, ct: float = 1.0, ci: float = 1.0) -> float:
        return float(lib().or_bvh_sah(self._h, ct, ci))

    def build_masks(self, R: int, L: int = 3, eps_rel: float = 2.0 ** -16):
        eps = scene_eps(self.tris, eps_rel)
        rc = lib().or_bvh_masks(self._h, _ptr(self.tris, C.c_float), R, L, eps)
        if rc != 0:
            raise ValueError(f"or_bvh_masks failed ({rc})")
        self.R, self.L, self.eps = R, L, eps
        return self

    def masks(self) -> np.ndarray:
        out = np.zeros((max(self.num_nodes, 1), 2, mask_words(self.R)), np.uint32)
        lib().or_bvh_get_masks(self._h, _ptr(out, C.c_uint32))
        return out[: self.num_nodes]

    def compress(self, K: int = 256, bits: int = 8):
        k = lib().or_bvh_compress(self._h, K, bits)
        if k < 0:
            raise ValueError("or_bvh_compress failed")
        self.K = k
        return self

    def clut(self):
        c = np.zeros((max(self.K, 1), mask_words(self.R)), np.uint32)
        idx = np.zeros((max(self.num_nodes, 1), 2), np.uint8)
        lib().or_bvh_get_clut(self._h, _ptr(c, C.c_uint32), _ptr(idx, C.c_uint8))
        return c[: self.K], idx[: self.num_nodes]

    def trace(self, rays: np.ndarray, mode: int = 0, cull: int = 0,
              r_begin: int = 0, r_end: int | None = None, out=None, skip_bits: int | None = None,
              stride: int = 1, leaf_min: int = 0, width: int = 2):
        """Alg. 4.  cull: 0 plain, 1 uncompressed masks, 2 compressed masks.
        skip_bits: children whose mask has at least this many bits set are
        kept untested (default R^3: only all-ones masks); stride: inner
        children are tested only at depths that are multiples of it;
        leaf_min: leaf children with fewer triangles are kept untested.
        Returns dict(t, id, uv, counts[n,2], mask_tests)."""
        if skip_bits is None:
            skip_bits = max(self.R, 1) ** 3
        rays = _f32(rays).reshape(-1, 8)
        n = rays.shape[0]
        r_end = n if r_end is None else r_end
        if out is None:
            out = dict(t=np.zeros(n, np.float32), id=np.zeros(n, np.int32),
                       uv=np.zeros((n, 2), np.float32),
                       counts=np.zeros((n, 2), np.uint32),
                       mask_tests=np.zeros(n, np.uint32))
        fn = lib().or_trace4_range if width == 4 else lib().or_trace_range
        rc = fn(self._h, _ptr(self.tris, C.c_float), _ptr(rays, C.c_float),
                                  r_begin, r_end, mode, cull, skip_bits, stride, leaf_min,
                                  _ptr(out["t"], C.c_float),
                                  _ptr(out["id"], C.c_int32), _ptr(out["uv"], C.c_float),
                                  _ptr(out["counts"], C.c_uint32),
                                  _ptr(out["mask_tests"], C.c_uint32))
        if rc != 0:
            raise ValueError(f"or_trace failed ({rc})")
        return out


def _frontier(self, depth: int = 8):
    """(child, count, box[k][6], class_of_tri) of the depth-`depth` frontier."""
    cap = 1 << depth
    fc = np.zeros(cap, np.int32)
    fn = np.zeros(cap, np.int32)
    fb = np.zeros((cap, 6), np.float32)
    cls = np.zeros(max(self.ntri, 1), np.uint8)
    k = lib().or_bvh_frontier(self._h, depth, _ptr(fc, C.c_int32), _ptr(fn, C.c_int32),
                              _ptr(fb, C.c_float), _ptr(cls, C.c_uint8))
    return fc[:k], fn[:k], fb[:k], cls[: self.ntri]


def _trace_seeded(self, rays, cls, depth: int = 8, cull: int = 0, skip_bits=None, stride=1,
                  leaf_min=0):
    """Seeded closest-hit traversal over the depth-`depth` frontier; cls[i]
    outside [0, frontier size) traces ray i without a seed."""
    rays = _f32(rays).reshape(-1, 8)
    n = rays.shape[0]
    fc, fn, fb, _ = self.frontier(depth)
    fb = np.ascontiguousarray(fb)
    c = np.ascontiguousarray(cls, dtype=np.int32)
    if skip_bits is None:
        skip_bits = max(self.R, 1) ** 3
    t = np.zeros(n, np.float32)
    hid = np.zeros(n, np.int32)
    uv = np.zeros((n, 2), np.float32)
    cnt = np.zeros((n, 2), np.uint32)
    rc = lib().or_trace_seeded(self._h, _ptr(self.tris, C.c_float), _ptr(rays, C.c_float), n,
                               cull, skip_bits, stride, leaf_min, _ptr(c, C.c_int32),
                               _ptr(fc, C.c_int32), _ptr(fn, C.c_int32), _ptr(fb, C.c_float),
                               len(fc), _ptr(t, C.c_float), _ptr(hid, C.c_int32),
                               _ptr(uv, C.c_float), _ptr(cnt, C.c_uint32))
    if rc != 0:
        raise ValueError(f"or_trace_seeded failed ({rc})")
    return dict(t=t, id=hid, uv=uv, counts=cnt)


def _set_cellform(self, form: int = 0):
    """Cell form of the culling tests: 0 = Alg. 1 as written (default),
    1 = the fused multiply-add form, mirroring the GPU option."""
    lib().or_bvh_set_cellform(self._h, int(form))
    return self


def _set_ideal(self, ideal: bool = True):
    """Culling tests use the exact ray mask (Sec. 4.1's ideal culling)."""
    lib().or_bvh_set_ideal(self._h, int(bool(ideal)))
    return self


def _wide(self):
    """4-wide view: dict(n[k], parent[k,4], child[k,4], next[k,4])."""
    k = int(lib().or_bvh_wide(self._h))
    n = np.zeros(max(k, 1), np.int32)
    p = np.zeros((max(k, 1), 4), np.int64)
    c = np.zeros((max(k, 1), 4), np.int32)
    nx = np.zeros((max(k, 1), 4), np.int64)
    lib().or_bvh_wide_export(self._h, _ptr(n, C.c_int32), _ptr(p, C.c_int64),
                             _ptr(c, C.c_int32), _ptr(nx, C.c_int64))
    return dict(n=n[:k], parent=p[:k], child=c[:k], next=nx[:k])


def _set_ray2r(self, on: bool = True):
    """Culling tests look up the R_ray = 2R table (Sec. 4.2) instead of the
    R table."""
    if on:
        self._lut2r = raylut2r(self.R)
        lib().or_bvh_set_raylut2r(self._h, _ptr(self._lut2r, C.c_uint32))
    else:
        lib().or_bvh_set_raylut2r(self._h, None)
        self._lut2r = None
    return self


def _refit(self, tris):
    """Moved triangles (same count, input order): slot boxes refit over the
    same topology.  Masks are rebuilt by build_masks, compression indices
    by reencode."""
    t = _f32(tris).reshape(-1, 9)
    if t.shape[0] != self.ntri:
        raise ValueError("refit needs the same number of triangles")
    self.tris = t
    lib().or_bvh_refit(self._h, _ptr(self.tris, C.c_float))
    return self


def _reencode(self):
    """Alg. 3 for every slot against the compression LUT already chosen."""
    if lib().or_bvh_reencode(self._h) != 0:
        raise ValueError("or_bvh_reencode needs masks and a compression LUT")
    return self


OracleBVH.refit = _refit
OracleBVH.reencode = _reencode
OracleBVH.set_ray2r = _set_ray2r
OracleBVH.wide = _wide
OracleBVH.set_ideal = _set_ideal
OracleBVH.set_cellform = _set_cellform
OracleBVH.frontier = _frontier
OracleBVH.trace_seeded = _trace_seeded


def scene_eps(tris, eps_rel: float = 2.0 ** -16) -> float:
    t = _f32(tris).reshape(-1, 9)
    return float(lib().or_scene_eps(_ptr(t, C.c_float), t.shape[0], eps_rel))


def brute(tris, rays, mode: int = 0):
    """Closest (any) hit over all triangles; returns (t, id, second_t)."""
    t9 = _f32(tris).reshape(-1, 9)
    r8 = _f32(rays).reshape(-1, 8)
    n = r8.shape[0]
    ht = np.zeros(n, np.float32)
    hid = np.zeros(n, np.int32)
    t2 = np.zeros(n, np.float32)
    lib().or_brute(_ptr(t9, C.c_float), t9.shape[0], _ptr(r8, C.c_float), n, mode,
                   _ptr(ht, C.c_float), _ptr(hid, C.c_int32), _ptr(t2, C.c_float))
    return ht, hid, t2


def ray_tri(ray8, tri9, tcur=np.inf):
    r, t = _f32(ray8).reshape(8), _f32(tri9).reshape(9)
    tt, u, v = C.c_float(), C.c_float(), C.c_float()
    ok = lib().or_ray_tri(_ptr(r, C.c_float), _ptr(t, C.c_float), float(tcur),
                          C.byref(tt), C.byref(u), C.byref(v))
    return (bool(ok), tt.value, u.value, v.value)


def slab(ray8, box6, tcur=np.inf):
    r, b = _f32(ray8).reshape(8), _f32(box6).reshape(6)
    tn, tf = C.c_float(), C.c_float()
    ok = lib().or_slab(_ptr(r, C.c_float), _ptr(b, C.c_float), float(tcur),
                       C.byref(tn), C.byref(tf))
    return bool(ok), tn.value, tf.value


def cell(p: float, lo: float, hi: float, R: int) -> int:
    return int(lib().or_cell(float(p), float(lo), float(hi), R))


def cell_t(t: float, o: float, d: float, lo: float, hi: float, R: int) -> int:
    """Alg. 1 cell by the fused form (an option of the traversal)."""
    return int(lib().or_cell_t(t, o, d, lo, hi, R))


def cell_at(t: float, o: float, d: float, lo: float, hi: float, R: int) -> int:
    """Alg. 1 cell as written: p = o + t d, then floor(R/extent (p - lo))."""
    return int(lib().or_cell_at(t, o, d, lo, hi, R))


def cell2_t(t: float, o: float, d: float, lo: float, hi: float, R: int) -> int:
    """2R-grid cell from the fused form (option)."""
    return int(lib().or_cell2_at(t, o, d, lo, hi, R, 1))


def cell2_at(t: float, o: float, d: float, lo: float, hi: float, R: int, form: int = 0) -> int:
    """2R-grid cell: twice the Alg. 1 coordinate (form 0, default) or the
    fused one (form 1), rounded down, clamped to [0, 2R-1]."""
    return int(lib().or_cell2_at(t, o, d, lo, hi, R, form))


# -------------------------------------------------------------- bounce rays --

def pcg_hash(v: int) -> int:
    return int(lib().or_pcg_hash(v & 0xFFFFFFFF))


def bounce(ray8, t: float, tri9, seed: int, rid: int, bounce_idx: int):
    """One diffuse bounce ray (float32[8]) or None for a degenerate triangle."""
    r, tr = _f32(ray8).reshape(8), _f32(tri9).reshape(9)
    out = np.zeros(8, np.float32)
    ok = lib().or_bounce(_ptr(r, C.c_float), float(t), _ptr(tr, C.c_float), seed & 0xFFFFFFFF,
                         rid & 0xFFFFFFFF, bounce_idx, _ptr(out, C.c_float))
    return out if ok else None


def bounce_wave(rays, hit_t, hit_id, tris, seed: int, bounce_idx: int, path=None):
    """Bounce rays for every hit of a wave, in ray order.  The random stream of
    a ray is keyed by its path id (the primary ray it descends from), so it
    does not depend on the order of a wave.  Returns (rays, path ids)."""
    path = np.arange(len(hit_id)) if path is None else np.asarray(path)
    out, par = [], []
    for i in np.nonzero(hit_id >= 0)[0]:
        b = bounce(rays[i], float(hit_t[i]), tris[hit_id[i]], seed, int(path[i]), bounce_idx)
        if b is not None:
            out.append(b)
            par.append(int(path[i]))
    if not out:
        return np.zeros((0, 8), np.float32), np.zeros(0, np.int64)
    return np.stack(out), np.asarray(par, np.int64)
