"""ctypes binding of libsubcull (include/subcull.h), same names as the C-ABI.

Argument marshalling only: every step of the path runs in the native
library (host builders in C++, traversal in CUDA for sm_103a).  PyTorch is
used for device memory and streams.  If the library cannot be built or
loaded this module raises; there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import _build

SC_ABI_VERSION = 2  # include/subcull.h; the library must report the same
SC_OK = 0
SC_ERR_ARG, SC_ERR_CUDA, SC_ERR_NOMEM, SC_ERR_TIMEOUT = -1, -2, -3, -4
SC_ERR_STACK, SC_ERR_UNSUPPORTED, SC_ERR_STATE, SC_ERR_IO = -5, -6, -7, -8
SC_SCENE_HAIR, SC_SCENE_SOUP = 0, 1
SC_RAYS_PINHOLE, SC_RAYS_RANDOM = 0, 1
SC_LAYOUT_PLAIN, SC_LAYOUT_MASKED, SC_LAYOUT_MASKED_COMPACT = 0, 1, 2
SC_LAYOUT_PLAIN4, SC_LAYOUT_MASKED4 = 3, 4
SC_LAYOUT_MASKED_RAY2R = 5
SC_CLOSEST, SC_ANY = 0, 1
SC_LUT_AUTO, SC_LUT_GLOBAL, SC_LUT_SHARED, SC_LUT_BITTABLE, SC_LUT_RAY2R = 0, 1, 2, 3, 4
SC_LUT_FACTORED_L1 = 5
STATUS_NAMES = {0: "SC_OK", -1: "SC_ERR_ARG", -2: "SC_ERR_CUDA", -3: "SC_ERR_NOMEM",
                -4: "SC_ERR_TIMEOUT", -5: "SC_ERR_STACK", -6: "SC_ERR_UNSUPPORTED",
                -7: "SC_ERR_STATE", -8: "SC_ERR_IO"}


class SubcullError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class sc_scene_params(C.Structure):
    _fields_ = [("count", C.c_int64), ("segments", C.c_int), ("ground", C.c_int)]


class sc_ray_params(C.Structure):
    _fields_ = [("width", C.c_int), ("height", C.c_int), ("count", C.c_int64),
                ("jitter_seed", C.c_uint64)]


class sc_build_opts(C.Structure):
    _fields_ = [("max_leaf", C.c_int), ("bins", C.c_int), ("L", C.c_int),
                ("lut_size", C.c_int), ("chunk_bits", C.c_int), ("eps_rel", C.c_double),
                ("threads", C.c_int), ("skip_bits", C.c_int), ("test_stride", C.c_int),
                ("leaf_min_tris", C.c_int), ("gpu_masks", C.c_int), ("gpu_bvh", C.c_int)]


class sc_bvh_info(C.Structure):
    _fields_ = [("num_tris", C.c_int64), ("num_nodes", C.c_int64), ("max_depth", C.c_int),
                ("grid_res", C.c_int), ("compress", C.c_int), ("L", C.c_int),
                ("clut_entries", C.c_int), ("eps", C.c_double), ("root_box", C.c_float * 6),
                ("ms_bvh", C.c_double), ("ms_masks", C.c_double), ("ms_compress", C.c_double)]


class sc_wave_out(C.Structure):
    _fields_ = [("hits", C.c_void_p), ("path", C.c_void_p), ("counts", C.c_void_p),
                ("rays", C.c_void_p)]


SC_MAX_BOUNCES = 4


class sc_trace_opts(C.Structure):
    _fields_ = [("block", C.c_int), ("blocks_per_sm", C.c_int), ("lut_mode", C.c_int),
                ("refill", C.c_int), ("stack", C.c_int), ("wave_chunk", C.c_int64),
                ("wait_timeout_ns", C.c_int64), ("variant", C.c_int)]


SC_VARIANT_FUSED_CELLS = 1
SC_VARIANT_PAIR = 2
SC_VARIANT_SPEC = 4
SC_VARIANT_TOS = 8
SC_VARIANT_SORT = 16
SC_VARIANT_DEFER = 32
SC_VARIANT_LAZY = 64
SC_VARIANT_SSTACK = 128
SC_VARIANT_TABLE_L1 = 256
SC_VARIANT_OCC9 = 1024
SC_VARIANT_OCC10 = 2048
SC_VARIANT_HSLOT = 4096


class sc_tune_result(C.Structure):
    _fields_ = [("block", C.c_int), ("stack", C.c_int), ("refill", C.c_int),
                ("wave_chunk", C.c_int64), ("ms", C.c_float), ("variant", C.c_int)]


_lock = threading.Lock()
_lib = None


def lib():
    """Loads (building if needed) libsubcull.so."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        L = C.CDLL(_build.build_product())
        P, vp = C.POINTER, C.c_void_p
        i64, u64, f32p, i32p, u32p, u8p = (C.c_int64, C.c_uint64, P(C.c_float), P(C.c_int32),
                                           P(C.c_uint32), P(C.c_uint8))
        sigs = {
            "sc_last_error": (C.c_char_p, []),
            "sc_abi_version": (C.c_int, []),
            "sc_scene_generate": (C.c_int, [C.c_int, P(sc_scene_params), u64, f32p, i64, P(i64)]),
            "sc_rays_generate": (C.c_int, [C.c_int, P(sc_ray_params), u64, f32p, i32p, i64,
                                           P(i64)]),
            "sc_build_opts_default": (None, [P(sc_build_opts)]),
            "sc_bvh_build": (C.c_int, [f32p, i64, C.c_int, C.c_int, P(sc_build_opts), P(vp)]),
            "sc_bvh_destroy": (None, [vp]),
            "sc_bvh_get_info": (C.c_int, [vp, P(sc_bvh_info)]),
            "sc_bvh_export": (C.c_int, [vp, i32p, i32p, i32p, f32p, i32p, u32p, u32p, u8p]),
            "sc_raylut": (C.c_int, [C.c_int, u32p]),
            "sc_raylut2r": (C.c_int, [C.c_int, u32p]),
            "sc_bvh_refit": (C.c_int, [vp, f32p, i64, P(sc_refit_info)]),
            "sc_l2_probe_blocks": (C.c_int, []),
            "sc_l2_read": (C.c_int, [vp, C.c_size_t, C.c_int, vp, vp]),
            "sc_bvh_save": (C.c_int, [vp, C.c_char_p]),
            "sc_bvh_load": (C.c_int, [C.c_char_p, P(vp)]),
            "sc_bvh_device_bytes": (C.c_int, [vp, C.c_int, P(C.c_size_t)]),
            "sc_bvh_upload": (C.c_int, [vp, C.c_int, vp, C.c_size_t, vp, P(vp)]),
            "sc_dbvh_destroy": (None, [vp]),
            "sc_trace_workspace_bytes": (C.c_size_t, []),
            "sc_trace": (C.c_int, [vp, vp, i64, vp, vp, C.c_int, C.c_int, P(sc_trace_opts), vp,
                                   C.c_size_t, vp]),
            "sc_trace_host": (C.c_int, [vp, vp, i64, vp, vp, C.c_int, C.c_int,
                                        P(sc_trace_opts), vp, vp, vp, vp, C.c_size_t, vp]),
            "sc_status_poll": (C.c_int, [vp, vp]),
            "sc_trace_noalloc": (C.c_int, [vp, vp, i64, vp, vp, C.c_int, C.c_int,
                                           P(sc_trace_opts), vp]),
            "sc_trace_waves_workspace_bytes": (C.c_size_t, [i64, P(sc_trace_opts)]),
            "sc_autotune_waves": (C.c_int, [vp, vp, i64, C.c_int, C.c_uint32, C.c_int,
                                            P(sc_wave_out), P(sc_trace_opts), vp, C.c_size_t,
                                            C.c_int, vp, C.c_size_t, P(sc_trace_opts),
                                            P(sc_tune_result), C.c_int, P(C.c_int), vp]),
            "sc_trace_waves": (C.c_int, [vp, vp, i64, C.c_int, C.c_uint32, C.c_int,
                                         P(sc_wave_out), P(sc_trace_opts), vp, C.c_size_t, vp]),
            "sc_waves_poll": (C.c_int, [vp, C.c_int, u32p, vp]),
            "sc_trace_waves_host": (C.c_int, [vp, vp, i64, C.c_int, C.c_uint32, C.c_int,
                                              P(sc_wave_out), P(sc_trace_opts), vp,
                                              P(sc_wave_out), vp, C.c_size_t, u32p, vp]),
            "sc_bvh_frontier": (C.c_int, [vp, C.c_int, vp, C.c_int, P(C.c_int), u8p]),
            "sc_trace_seeded": (C.c_int, [vp, vp, i64, vp, vp, C.c_int, vp, vp, C.c_int,
                                          P(sc_trace_opts), vp, C.c_size_t, vp]),
            "sc_mlp_num_params": (C.c_int, []),
            "sc_mlp_to_bf16": (C.c_int, [vp, vp, vp]),
            "sc_mlp_forward": (C.c_int, [vp, vp, i64, vp, vp, vp, C.c_float, vp]),
            "sc_mlp_train_workspace_bytes": (C.c_size_t, [i64]),
            "sc_mlp_forward_tc": (C.c_int, [vp, vp, i64, vp, vp, vp, C.c_float, vp, vp]),
            "sc_mlp_grad": (C.c_int, [vp, vp, vp, i64, vp, vp, vp, vp, C.c_size_t, vp]),
            "sc_mlp_grad_tc": (C.c_int, [vp, vp, vp, i64, vp, vp, vp, vp, C.c_size_t, vp, vp]),
            "sc_mlp_adam": (C.c_int, [vp, vp, vp, vp, vp, C.c_int, C.c_float, C.c_float,
                                      C.c_float, C.c_float, vp]),
            "sc_mlp_labels": (C.c_int, [vp, vp, i64, vp, vp, vp, vp, i64, vp]),
            "sc_mlp_gather": (C.c_int, [vp, vp, i64, C.c_uint64, i64, i64, vp, vp, vp]),
        }
        for name, (res, args) in sigs.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        got = L.sc_abi_version()
        if got != SC_ABI_VERSION:
            raise RuntimeError(f"libsubcull reports ABI version {got}, this binding is written "
                               f"for {SC_ABI_VERSION}: rebuild the library")
        _lib = L
        return L


def _check(code: int):
    if code != SC_OK:
        msg = lib().sc_last_error()
        raise SubcullError(code, msg.decode() if msg else "")


def _ptr(a: np.ndarray, t):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.POINTER(t))


# ------------------------------------------------------------------ inputs --

def sc_scene_generate(kind: int, count: int, segments: int = 16, ground: int = 0,
                      seed: int = 1) -> np.ndarray:
    p = sc_scene_params(count, segments, ground)
    n = C.c_int64()
    _check(lib().sc_scene_generate(kind, C.byref(p), seed, None, 0, C.byref(n)))
    out = np.empty((n.value, 9), np.float32)
    _check(lib().sc_scene_generate(kind, C.byref(p), seed, _ptr(out, C.c_float), n.value,
                                   C.byref(n)))
    return out


def sc_rays_generate(kind: int, width: int = 0, height: int = 0, count: int = 0,
                     jitter_seed: int = 0, seed: int = 0, with_pixels: bool = False):
    p = sc_ray_params(width, height, count, jitter_seed)
    n = C.c_int64()
    _check(lib().sc_rays_generate(kind, C.byref(p), seed, None, None, 0, C.byref(n)))
    out = np.empty((n.value, 8), np.float32)
    pix = np.empty(n.value, np.int32)
    _check(lib().sc_rays_generate(kind, C.byref(p), seed, _ptr(out, C.c_float),
                                  _ptr(pix, C.c_int32), n.value, C.byref(n)))
    return (out, pix) if with_pixels else out


# ------------------------------------------------------------------- build --

def sc_build_opts_default() -> sc_build_opts:
    o = sc_build_opts()
    lib().sc_build_opts_default(C.byref(o))
    return o


class Bvh:
    """Host BVH handle (sc_bvh*)."""

    def __init__(self, handle, ntri):
        self._h = handle
        self.ntri = ntri

    def __del__(self):
        if getattr(self, "_h", None):
            lib().sc_bvh_destroy(self._h)
            self._h = None

    @property
    def handle(self):
        return self._h

    def info(self) -> sc_bvh_info:
        i = sc_bvh_info()
        _check(lib().sc_bvh_get_info(self._h, C.byref(i)))
        return i

    def export(self):
        """Host arrays: dict(root, child, count, box, perm, masks?, clut?, cidx?)."""
        i = self.info()
        nn = i.num_nodes
        W = (i.grid_res ** 3 + 31) // 32 if i.grid_res else 0
        root = np.zeros(2, np.int32)
        child = np.zeros((max(nn, 1), 2), np.int32)
        count = np.zeros((max(nn, 1), 2), np.int32)
        box = np.zeros((max(nn, 1), 2, 6), np.float32)
        perm = np.zeros(max(i.num_tris, 1), np.int32)
        masks = np.zeros((max(nn, 1), 2, max(W, 1)), np.uint32) if W else None
        clut = np.zeros((max(i.clut_entries, 1), max(W, 1)), np.uint32) if i.compress else None
        cidx = np.zeros((max(nn, 1), 2), np.uint8) if i.compress else None
        _check(lib().sc_bvh_export(
            self._h, _ptr(root, C.c_int32), _ptr(child, C.c_int32), _ptr(count, C.c_int32),
            _ptr(box, C.c_float), _ptr(perm, C.c_int32),
            _ptr(masks, C.c_uint32) if masks is not None else None,
            _ptr(clut, C.c_uint32) if clut is not None else None,
            _ptr(cidx, C.c_uint8) if cidx is not None else None))
        out = dict(root=root, child=child[:nn], count=count[:nn], box=box[:nn],
                   perm=perm[: i.num_tris])
        if masks is not None:
            out["masks"] = masks[:nn]
        if clut is not None:
            out["clut"] = clut[: i.clut_entries]
            out["cidx"] = cidx[:nn]
        return out


def sc_bvh_build(tris: np.ndarray, grid_res: int = 6, compress: int = 0,
                 opts: sc_build_opts | None = None, **kw) -> Bvh:
    t = np.ascontiguousarray(tris, dtype=np.float32).reshape(-1, 9)
    o = opts if opts is not None else sc_build_opts_default()
    for k, v in kw.items():
        setattr(o, k, v)
    h = C.c_void_p()
    _check(lib().sc_bvh_build(_ptr(t, C.c_float) if len(t) else None, t.shape[0], grid_res,
                              compress, C.byref(o), C.byref(h)))
    return Bvh(h, t.shape[0])


class sc_refit_info(C.Structure):
    _fields_ = [("moved_tris", C.c_int64), ("dirty_nodes", C.c_int64), ("ms_boxes", C.c_double),
                ("ms_masks", C.c_double), ("ms_compress", C.c_double)]


def sc_bvh_refit(bvh: Bvh, tris: np.ndarray) -> sc_refit_info:
    """Moves the BVH's triangles to `tris` (same count, input order): boxes,
    masks and compression indices above moved triangles are computed again."""
    t = np.ascontiguousarray(tris, dtype=np.float32).reshape(-1, 9)
    info = sc_refit_info()
    _check(lib().sc_bvh_refit(bvh.handle, _ptr(t, C.c_float) if len(t) else None, t.shape[0],
                              C.byref(info)))
    return info


def sc_l2_probe_blocks() -> int:
    return int(lib().sc_l2_probe_blocks())


def sc_l2_read(buf, reps: int, sink, stream=None):
    """Reads the device tensor `buf` reps times through L2 (see the header);
    sink: contiguous device int64 / uint64 tensor of >= sc_l2_probe_blocks()
    entries (each block writes one)."""
    import torch
    if (not sink.is_cuda or not sink.is_contiguous()
            or sink.dtype not in (torch.int64, getattr(torch, "uint64", torch.int64))
            or sink.numel() < sc_l2_probe_blocks()):
        raise ValueError("sink must be a contiguous CUDA int64 tensor of at least "
                         f"{sc_l2_probe_blocks()} entries")
    _check(lib().sc_l2_read(C.c_void_p(buf.data_ptr()), buf.numel() * buf.element_size(), reps,
                            C.c_void_p(sink.data_ptr()), _stream_ptr(stream)))


def sc_bvh_save(bvh: Bvh, path: str):
    _check(lib().sc_bvh_save(bvh.handle, os.fsencode(path)))


def sc_bvh_load(path: str) -> Bvh:
    h = C.c_void_p()
    _check(lib().sc_bvh_load(os.fsencode(path), C.byref(h)))
    b = Bvh(h, 0)
    b.ntri = b.info().num_tris
    return b


def sc_raylut(R: int) -> np.ndarray:
    R3 = R ** 3
    out = np.zeros((R3 * R3, (R3 + 31) // 32), np.uint32)
    _check(lib().sc_raylut(R, _ptr(out, C.c_uint32)))
    return out


def sc_raylut2r(R: int) -> np.ndarray:
    R23 = (2 * R) ** 3
    out = np.zeros((R23 * R23, (R ** 3 + 31) // 32), np.uint32)
    _check(lib().sc_raylut2r(R, _ptr(out, C.c_uint32)))
    return out


def sc_bvh_device_bytes(bvh: Bvh, layout: int) -> int:
    n = C.c_size_t()
    _check(lib().sc_bvh_device_bytes(bvh.handle, layout, C.byref(n)))
    return n.value


def sc_trace_workspace_bytes() -> int:
    return int(lib().sc_trace_workspace_bytes())


# ------------------------------------------------------------ device side --

def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


class DeviceBVH:
    """A BVH image in a torch-owned device buffer plus its sc_dbvh view."""

    def __init__(self, bvh: Bvh, layout: int, device="cuda", stream=None):
        import torch
        nbytes = sc_bvh_device_bytes(bvh, layout)
        self.buf = torch.empty(nbytes, dtype=torch.uint8, device=device)
        self.layout = layout
        self.nbytes = nbytes
        h = C.c_void_p()
        _check(lib().sc_bvh_upload(bvh.handle, layout, C.c_void_p(self.buf.data_ptr()), nbytes,
                                   _stream_ptr(stream), C.byref(h)))
        self._h = h

    def __del__(self):
        if getattr(self, "_h", None):
            lib().sc_dbvh_destroy(self._h)
            self._h = None

    @property
    def handle(self):
        return self._h


def sc_bvh_upload(bvh: Bvh, layout: int, stream=None) -> DeviceBVH:
    return DeviceBVH(bvh, layout, stream=stream)


def _opts(block=0, blocks_per_sm=0, lut_mode=SC_LUT_AUTO, refill=0, stack=0, wave_chunk=0,
          wait_timeout_ns=0, variant=0):
    return sc_trace_opts(block, blocks_per_sm, lut_mode, refill, stack, wave_chunk,
                         wait_timeout_ns, variant)


def sc_trace(dbvh: DeviceBVH, rays, hits, counts, mode: int, cull: int, work,
             opts: sc_trace_opts | None = None, stream=None):
    """All tensors on the device: rays float32[n,8], hits float32[n,4] (16 B
    per hit: t, id bits, u, v), counts int32[n,2] or None, work uint8[>=256]."""
    n = rays.shape[0]
    o = opts or _opts()
    _check(lib().sc_trace(dbvh.handle, C.c_void_p(rays.data_ptr()), n,
                          C.c_void_p(hits.data_ptr()),
                          C.c_void_p(counts.data_ptr()) if counts is not None else None,
                          mode, cull, C.byref(o), C.c_void_p(work.data_ptr()), work.numel(),
                          _stream_ptr(stream)))


def sc_trace_host(dbvh: DeviceBVH, h_rays, h_hits, h_counts, mode: int, cull: int,
                  d_rays, d_hits, d_counts, work, opts=None, stream=None):
    """Host tensors (pinned) in, host tensors out; device scratch given."""
    n = h_rays.shape[0]
    o = opts or _opts()
    _check(lib().sc_trace_host(dbvh.handle, C.c_void_p(h_rays.data_ptr()), n,
                               C.c_void_p(h_hits.data_ptr()),
                               C.c_void_p(h_counts.data_ptr()) if h_counts is not None else None,
                               mode, cull, C.byref(o), C.c_void_p(d_rays.data_ptr()),
                               C.c_void_p(d_hits.data_ptr()),
                               C.c_void_p(d_counts.data_ptr()) if d_counts is not None else None,
                               C.c_void_p(work.data_ptr()), work.numel(), _stream_ptr(stream)))


def sc_trace_noalloc(dbvh: DeviceBVH, rays, hits, counts, mode: int, cull: int,
                     opts: sc_trace_opts | None = None, stream=None):
    """sc_trace without a workspace (static device scratch); blocks until the
    trace has finished and raises on a device-side error."""
    n = rays.shape[0]
    o = opts or _opts()
    _check(lib().sc_trace_noalloc(dbvh.handle, C.c_void_p(rays.data_ptr()), n,
                                  C.c_void_p(hits.data_ptr()),
                                  C.c_void_p(counts.data_ptr()) if counts is not None else None,
                                  mode, cull, C.byref(o), _stream_ptr(stream)))


def sc_status_poll(work, stream=None):
    _check(lib().sc_status_poll(C.c_void_p(work.data_ptr()), _stream_ptr(stream)))


# --------------------------------------------------------------- helpers --

def trace(dbvh: DeviceBVH, rays, mode: int = SC_CLOSEST, cull: int = 1, with_counts=True,
          opts=None, stream=None):
    """Convenience: allocates outputs and workspace with torch, traces, and
    returns (hits float32[n,4], counts int32[n,2] | None)."""
    import torch
    n = rays.shape[0]
    dev = rays.device
    hits = torch.empty((n, 4), dtype=torch.float32, device=dev)
    counts = torch.empty((n, 2), dtype=torch.int32, device=dev) if with_counts else None
    work = torch.empty(sc_trace_workspace_bytes(), dtype=torch.uint8, device=dev)
    sc_trace(dbvh, rays, hits, counts, mode, cull, work, opts, stream)
    sc_status_poll(work, stream)
    return hits, counts


def split_hits(hits):
    """(t, id, u, v) numpy views of a float32[n,4] hit array."""
    h = hits.cpu().numpy() if hasattr(hits, "cpu") else np.asarray(hits)
    h = np.ascontiguousarray(h, dtype=np.float32)
    return h[:, 0], h[:, 1].view(np.int32), h[:, 2], h[:, 3]


# ------------------------------------------------------------------ waves --

def sc_trace_waves_workspace_bytes(n0: int, opts: sc_trace_opts | None = None) -> int:
    return int(lib().sc_trace_waves_workspace_bytes(n0, C.byref(opts) if opts else None))


def _wave_arr(outs, bounces: int):
    arr = (sc_wave_out * (bounces + 1))()
    for w, o in enumerate(outs):
        h, pth, cnt = o[0], o[1], o[2]
        ry = o[3] if len(o) > 3 else None
        arr[w].hits = h.data_ptr()
        arr[w].path = pth.data_ptr() if pth is not None else None
        arr[w].counts = cnt.data_ptr() if cnt is not None else None
        arr[w].rays = ry.data_ptr() if ry is not None else None
    return arr


def sc_trace_waves(dbvh: DeviceBVH, rays, bounces: int, seed: int, cull: int, outs, ws,
                   opts: sc_trace_opts | None = None, stream=None):
    """outs: list of bounces+1 (hits float32[n0,4], path int32[n0] | None,
    counts int32[n0,2] | None[, rays float32[n0,8] | None]) device tensors;
    ws: uint8 device tensor."""
    n0 = rays.shape[0]
    arr = _wave_arr(outs, bounces)
    o = opts or _opts()
    _check(lib().sc_trace_waves(dbvh.handle, C.c_void_p(rays.data_ptr()), n0, bounces,
                                seed & 0xFFFFFFFF, cull, arr, C.byref(o),
                                C.c_void_p(ws.data_ptr()), ws.numel(), _stream_ptr(stream)))


def sc_trace_waves_host(dbvh: DeviceBVH, h_rays, bounces: int, seed: int, cull: int, h_outs,
                        d_rays, d_outs, ws, opts: sc_trace_opts | None = None, stream=None):
    """End to end through the C-ABI: h_rays (host float32[n0, 8] tensor,
    ideally pinned) in, the wave pipeline, each wave's entries out to h_outs
    (host tensors laid out like sc_trace_waves' outs); d_rays / d_outs are
    the device buffers.  Returns the wave sizes (sizes[0] = n0)."""
    n0 = h_rays.shape[0]
    ha, da = _wave_arr(h_outs, bounces), _wave_arr(d_outs, bounces)
    o = opts or _opts()
    sizes = np.zeros(bounces + 1, np.uint32)
    _check(lib().sc_trace_waves_host(dbvh.handle, C.c_void_p(h_rays.data_ptr()), n0, bounces,
                                     seed & 0xFFFFFFFF, cull, ha, C.byref(o),
                                     C.c_void_p(d_rays.data_ptr()), da,
                                     C.c_void_p(ws.data_ptr()), ws.numel(),
                                     _ptr(sizes, C.c_uint32), _stream_ptr(stream)))
    sizes[0] = n0
    return sizes


def sc_waves_poll(ws, bounces: int, stream=None):
    sizes = np.zeros(bounces + 1, np.uint32)
    _check(lib().sc_waves_poll(C.c_void_p(ws.data_ptr()), bounces, _ptr(sizes, C.c_uint32),
                               _stream_ptr(stream)))
    return sizes


class WaveBuffers:
    """Device outputs and workspace for sc_trace_waves (torch-owned)."""

    def __init__(self, n0: int, bounces: int, with_counts: bool = True, device="cuda",
                 with_rays: bool = False):
        import torch
        self.n0, self.bounces = n0, bounces
        self.hits = [torch.empty((n0, 4), dtype=torch.float32, device=device)
                     for _ in range(bounces + 1)]
        self.path = [torch.empty(n0, dtype=torch.int32, device=device) for _ in range(bounces + 1)]
        self.counts = [torch.empty((n0, 2), dtype=torch.int32, device=device) if with_counts
                       else None for _ in range(bounces + 1)]
        self.rays = [torch.empty((n0, 8), dtype=torch.float32, device=device) if with_rays
                     else None for _ in range(bounces + 1)]
        nb = sc_trace_waves_workspace_bytes(n0)  # largest chunk: fits every wave_chunk
        # 256-byte aligned view into a slightly larger buffer
        self._raw = torch.empty(nb + 256, dtype=torch.uint8, device=device)
        off = (-self._raw.data_ptr()) % 256
        self.ws = self._raw[off:off + nb]

    def outs(self):
        return list(zip(self.hits, self.path, self.counts, self.rays))


def trace_waves(dbvh: DeviceBVH, rays, bounces: int, seed: int, cull: int, buffers=None,
                opts=None, stream=None):
    """Runs the wave pipeline; returns (buffers, wave sizes)."""
    b = buffers or WaveBuffers(rays.shape[0], bounces, device=rays.device)
    sc_trace_waves(dbvh, rays, bounces, seed, cull, b.outs(), b.ws, opts, stream)
    sizes = sc_waves_poll(b.ws, bounces, stream)
    sizes[0] = rays.shape[0]
    return b, sizes


def sc_autotune_waves(dbvh: DeviceBVH, rays, bounces: int, seed: int, cull: int, buffers,
                      base: sc_trace_opts | None = None, reps: int = 3, flush=None, stream=None):
    """Times the wave pipeline over block / stack / refill / wave-chunk
    candidates (and the shared-memory stack ring where the image has kernel
    variants); returns (best opts, list of (block, stack, refill, chunk,
    variant, ms))."""
    n0 = rays.shape[0]
    arr = _wave_arr(buffers.outs(), bounces)
    best = sc_trace_opts()
    cap = 256
    res = (sc_tune_result * cap)()
    nres = C.c_int()
    b = base or _opts()
    _check(lib().sc_autotune_waves(dbvh.handle, C.c_void_p(rays.data_ptr()), n0, bounces,
                                   seed & 0xFFFFFFFF, cull, arr, C.byref(b),
                                   C.c_void_p(buffers.ws.data_ptr()), buffers.ws.numel(), reps,
                                   C.c_void_p(flush.data_ptr()) if flush is not None else None,
                                   flush.numel() if flush is not None else 0,
                                   C.byref(best), res, cap, C.byref(nres), _stream_ptr(stream)))
    rows = [(r.block, r.stack, r.refill, r.wave_chunk, r.variant, r.ms)
            for r in res[: min(nres.value, cap)]]
    return best, rows


# --------------------------------------------------------- learned proposal --

class sc_frontier_entry(C.Structure):
    _fields_ = [("lo", C.c_float * 3), ("hi", C.c_float * 3), ("slot", C.c_uint32),
                ("reserved", C.c_uint32)]


def sc_bvh_frontier(bvh: Bvh, depth: int = 8):
    """Frontier entries as float32[k][8] (lo.xyz, hi.xyz, slot word bits, 0)
    and the class of each triangle id (uint8[num_tris])."""
    cap = 1 << depth
    ent = np.zeros((cap, 8), np.float32)
    ntri = bvh.info().num_tris
    cls = np.zeros(max(ntri, 1), np.uint8)
    n = C.c_int()
    _check(lib().sc_bvh_frontier(bvh.handle, depth, ent.ctypes.data_as(C.c_void_p), cap,
                                 C.byref(n), _ptr(cls, C.c_uint8)))
    return ent[: n.value].copy(), cls[:ntri].copy()


def sc_trace_seeded(dbvh: DeviceBVH, rays, cls, frontier, hits, counts, cull: int, work,
                    opts: sc_trace_opts | None = None, stream=None):
    """rays float32[n,8], cls int32[n], frontier float32[k,8] entries
    (device); hits float32[n,4]; counts int32[n,2] or None; work: uint8."""
    o = opts or _opts()
    _check(lib().sc_trace_seeded(dbvh.handle, C.c_void_p(rays.data_ptr()), rays.shape[0],
                                 C.c_void_p(cls.data_ptr()), C.c_void_p(frontier.data_ptr()),
                                 frontier.shape[0], C.c_void_p(hits.data_ptr()),
                                 C.c_void_p(counts.data_ptr()) if counts is not None else None,
                                 cull, C.byref(o), C.c_void_p(work.data_ptr()), work.numel(),
                                 _stream_ptr(stream)))


def sc_mlp_num_params() -> int:
    return int(lib().sc_mlp_num_params())


def sc_mlp_to_bf16(w, wb, stream=None):
    _check(lib().sc_mlp_to_bf16(C.c_void_p(w.data_ptr()), C.c_void_p(wb.data_ptr()),
                                _stream_ptr(stream)))


def sc_mlp_forward(wb, rays, box, cls, logits=None, min_prob: float = 0.0, stream=None):
    _check(lib().sc_mlp_forward(C.c_void_p(wb.data_ptr()), C.c_void_p(rays.data_ptr()),
                                rays.shape[0], C.c_void_p(box.data_ptr()),
                                C.c_void_p(cls.data_ptr()),
                                C.c_void_p(logits.data_ptr()) if logits is not None else None,
                                min_prob, _stream_ptr(stream)))


def sc_mlp_forward_tc(wb, rays, box, cls, status, logits=None, min_prob: float = 0.0,
                      stream=None):
    """Tensor-core forward (tcgen05); status: device int32[1] (0 = ok)."""
    _check(lib().sc_mlp_forward_tc(C.c_void_p(wb.data_ptr()), C.c_void_p(rays.data_ptr()),
                                   rays.shape[0], C.c_void_p(box.data_ptr()),
                                   C.c_void_p(cls.data_ptr()),
                                   C.c_void_p(logits.data_ptr()) if logits is not None else None,
                                   min_prob, C.c_void_p(status.data_ptr()), _stream_ptr(stream)))


def sc_mlp_train_workspace_bytes(batch: int) -> int:
    return int(lib().sc_mlp_train_workspace_bytes(batch))


def sc_mlp_grad(wb, rays, labels, box, grad, loss, ws, stream=None):
    _check(lib().sc_mlp_grad(C.c_void_p(wb.data_ptr()), C.c_void_p(rays.data_ptr()),
                             C.c_void_p(labels.data_ptr()), rays.shape[0],
                             C.c_void_p(box.data_ptr()), C.c_void_p(grad.data_ptr()),
                             C.c_void_p(loss.data_ptr()), C.c_void_p(ws.data_ptr()), ws.numel(),
                             _stream_ptr(stream)))


def sc_mlp_grad_tc(wb, rays, labels, box, grad, loss, ws, status, stream=None):
    """sc_mlp_grad with the contractions on the tensor cores; status: device
    int32 tensor zeroed by the caller, ORed non-zero if a tensor-core wait
    ran out."""
    _check(lib().sc_mlp_grad_tc(C.c_void_p(wb.data_ptr()), C.c_void_p(rays.data_ptr()),
                                C.c_void_p(labels.data_ptr()), rays.shape[0],
                                C.c_void_p(box.data_ptr()), C.c_void_p(grad.data_ptr()),
                                C.c_void_p(loss.data_ptr()), C.c_void_p(ws.data_ptr()),
                                ws.numel(), C.c_void_p(status.data_ptr()), _stream_ptr(stream)))


def sc_mlp_adam(w, wb, grad, m, v, step: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8,
                stream=None):
    _check(lib().sc_mlp_adam(C.c_void_p(w.data_ptr()), C.c_void_p(wb.data_ptr()),
                             C.c_void_p(grad.data_ptr()), C.c_void_p(m.data_ptr()),
                             C.c_void_p(v.data_ptr()), step, lr, beta1, beta2, eps,
                             _stream_ptr(stream)))


def sc_mlp_gather(rays, labels, key: int, start: int, batch: int, out_rays, out_labels,
                  stream=None):
    """Rows perm(start .. start+batch-1) of (rays, labels) under the
    permutation of [0, n) chosen by key (see the header)."""
    _check(lib().sc_mlp_gather(C.c_void_p(rays.data_ptr()), C.c_void_p(labels.data_ptr()),
                               rays.shape[0], int(key) & 0xFFFFFFFFFFFFFFFF, start, batch,
                               C.c_void_p(out_rays.data_ptr()), C.c_void_p(out_labels.data_ptr()),
                               _stream_ptr(stream)))


def sc_mlp_labels(rays, hits, class_of_tri, out_rays, out_labels, count, stream=None):
    _check(lib().sc_mlp_labels(C.c_void_p(rays.data_ptr()), C.c_void_p(hits.data_ptr()),
                               rays.shape[0], C.c_void_p(class_of_tri.data_ptr()),
                               C.c_void_p(out_rays.data_ptr()),
                               C.c_void_p(out_labels.data_ptr()), C.c_void_p(count.data_ptr()),
                               out_labels.shape[0], _stream_ptr(stream)))
