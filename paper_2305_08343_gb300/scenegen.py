"""Seeded synthetic inputs: hair / soup scenes and camera / random rays.

A module of its own: it wraps ``csrc/gen/scenegen.c`` (built into a small
stand-alone library) and holds none of the method's arithmetic, so both the
GPU path's tests and the CPU oracle draw byte-identical inputs from it.

Arrays returned:
  triangles float32[n, 9] (v0, v1, v2), rays float32[n, 8] (o, tmin, d, tmax).
"""
from __future__ import annotations

import ctypes as C
import threading

import numpy as np

from . import _build

_lock = threading.Lock()
_lib = None


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(_build.build_scenegen())
            P = C.POINTER
            L.sg_hair_count.restype = C.c_int64
            L.sg_hair_count.argtypes = [C.c_int64, C.c_int, C.c_int]
            L.sg_hair.restype = None
            L.sg_hair.argtypes = [C.c_uint64, C.c_int64, C.c_int, C.c_int, C.c_int64,
                                  C.c_int64, P(C.c_float)]
            L.sg_soup.restype = None
            L.sg_soup.argtypes = [C.c_uint64, C.c_int64, C.c_int64, P(C.c_float)]
            L.sg_rays_pinhole.restype = None
            L.sg_rays_pinhole.argtypes = [C.c_int, C.c_int, C.c_uint64, P(C.c_float),
                                          P(C.c_int32)]
            L.sg_rays_random.restype = None
            L.sg_rays_random.argtypes = [C.c_uint64, C.c_int64, C.c_int64, P(C.c_float)]
            L.sg_uniform.restype = C.c_double
            L.sg_uniform.argtypes = [C.c_uint64, C.c_uint64, C.c_int]
            L.sg_sincos.restype = None
            L.sg_sincos.argtypes = [C.c_double, P(C.c_double), P(C.c_double)]
            L.sg_exp.restype = C.c_double
            L.sg_exp.argtypes = [C.c_double]
            _lib = L
        return _lib


def _fp(a):
    return a.ctypes.data_as(C.POINTER(C.c_float))


def _split(n: int, fn, parts: int = 8):
    """Runs fn(begin, end) over [0, n) in `parts` threads (the C code releases
    the GIL through ctypes)."""
    if n < 65536:
        fn(0, n)
        return
    bounds = np.linspace(0, n, parts + 1).astype(np.int64)
    ts = [threading.Thread(target=fn, args=(int(bounds[i]), int(bounds[i + 1])))
          for i in range(parts)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()


def hair(strands: int, segs: int = 16, ground: bool = False, seed: int = 1) -> np.ndarray:
    L = lib()
    n = L.sg_hair_count(strands, segs, int(ground))
    out = np.zeros((n, 9), np.float32)
    p = _fp(out)
    _split(strands, lambda a, b: L.sg_hair(seed, strands, segs, int(ground), a, b, p))
    if ground:
        L.sg_hair(seed, strands, segs, 1, strands, strands, p)
    return out


def soup(n: int, seed: int = 3) -> np.ndarray:
    L = lib()
    out = np.zeros((n, 9), np.float32)
    p = _fp(out)
    _split(n, lambda a, b: L.sg_soup(seed, a, b, p))
    return out


def pinhole(W: int, H: int, jitter_seed: int = 0, with_pixels: bool = False):
    L = lib()
    rays = np.zeros((W * H, 8), np.float32)
    pix = np.zeros(W * H, np.int32)
    L.sg_rays_pinhole(W, H, jitter_seed, _fp(rays), pix.ctypes.data_as(C.POINTER(C.c_int32)))
    return (rays, pix) if with_pixels else rays


def random_rays(n: int, seed: int = 3) -> np.ndarray:
    L = lib()
    out = np.zeros((n, 8), np.float32)
    p = _fp(out)
    _split(n, lambda a, b: L.sg_rays_random(seed, a, b, p))
    return out


def uniform(seed: int, stream: int, k: int) -> float:
    return float(lib().sg_uniform(seed, stream, k))


def sincos(x: float):
    s, c = C.c_double(), C.c_double()
    lib().sg_sincos(x, C.byref(s), C.byref(c))
    return s.value, c.value


def exp(x: float) -> float:
    return float(lib().sg_exp(x))


# Named workloads (sizes of the synthetic stand-ins for the paper's scenes).
def workload(name: str):
    """Returns (triangles, rays) of a named synthetic workload."""
    if name == "hair65k":      # 2,048 strands x 16 segments x 2 = 65,536 tris
        return hair(2048, 16, False, seed=1), pinhole(256, 256)
    if name == "hair1m":       # 1,048,576 tris + ground quad, 1920x1080 primary
        return hair(32768, 16, True, seed=2), pinhole(1920, 1080)
    if name == "soup4m":       # 2^22 soup triangles, 2^23 random rays
        return soup(1 << 22, seed=3), random_rays(1 << 23, seed=3)
    if name == "hair12m":      # 378,125 strands x 16 x 2 = 12.1M tris, 1920x1080
        return hair(378125, 16, False, seed=4), pinhole(1920, 1080)
    raise KeyError(name)
