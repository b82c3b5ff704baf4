"""GB300-native HMLFC: random-access decoding of hierarchical
motion-compensated light-field streams fused with two-plane rendering.

This module is a thin ctypes binding of ``libhmlfc.so`` (C ABI declared in
``include/hmlfc.h``): it marshals arguments -- device buffers are torch
tensors, the CUDA stream is torch's current stream -- and every step of the
decode and render runs in the library's CUDA kernels.  There is no CPU
fallback: if the library cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os
from pathlib import Path

import numpy as np

from .build import LIB, build  # noqa: F401

# Identifies the render kernel's code; profile figures recorded for another
# version are not reused.
KERNEL_VERSION = "render-cached-v16"
ENCODER_VERSION = "encode-planes-v4"

OK, E_INVALID_ARG, E_CORRUPT, E_OOM, E_CUDA, E_TIMEOUT, E_UNSUPPORTED = 0, -1, -2, -3, -4, -5, -6
MC_OFF, MC_QPEL, MC_ZERO, MC_INTEGER = 0, 1, 2, 3


class HmlfcError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"hmlfc error {code}: {msg}")
        self.code = code


class View(C.Structure):
    _fields_ = [("lf", C.c_int32), ("width", C.c_int32), ("height", C.c_int32),
                ("H_uv", C.c_float * 9), ("H_st", C.c_float * 9), ("reserved", C.c_int32),
                ("out_offset", C.c_int64)]


assert C.sizeof(View) == 96


class StreamInfo(C.Structure):
    _fields_ = [(n, C.c_int32) for n in ("nu", "nv", "width", "height", "levels", "block", "search",
                                          "qstep", "mc", "n_roots", "chroma")] + \
               [(n, C.c_int64) for n in ("n_nc", "n_blocks", "n_sig", "n_ref_tiles", "stream_bytes",
                                         "device_bytes")]


class EncodeParams(C.Structure):
    _fields_ = [(n, C.c_int32) for n in ("levels", "block", "search", "qstep", "t_ref", "t_pred", "mc",
                                          "threads", "chroma")]


_lib = None


class EncodeStats(C.Structure):
    _fields_ = [("blocks", C.c_uint64), ("sig_blocks", C.c_uint64), ("blocks_searched", C.c_uint64),
                ("int_terms", C.c_uint64), ("frac_terms", C.c_uint64)]


def lib() -> C.CDLL:
    """Load libhmlfc.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = Path(os.environ.get("HMLFC_LIB", str(LIB)))
    if not path.exists() or path == LIB:
        build()
    L = C.CDLL(str(path))
    P, I, I64, SZ = C.c_void_p, C.c_int, C.c_int64, C.c_size_t
    L.hmlfc_last_error.restype = C.c_char_p
    L.hmlfc_load_stream.argtypes = [P, SZ, I, P, C.POINTER(P)]
    L.hmlfc_free_stream.argtypes = [P]
    L.hmlfc_free_stream.restype = None
    L.hmlfc_stream_info.argtypes = [P, C.POINTER(StreamInfo)]
    L.hmlfc_decode_pixels.argtypes = [P, P, I64, P, P]
    L.hmlfc_decode_pixels_lod.argtypes = [P, P, I64, I, P, P]
    L.hmlfc_render_views_lod.argtypes = [P, I, P, I, I, P, P]
    L.hmlfc_render_views_host.argtypes = [P, I, P, I, P, P]
    L.hmlfc_touched_bytes_union_lod.argtypes = [P, I, P, I, I, P, P]
    L.hmlfc_check_status.argtypes = [P, P]
    L.hmlfc_render_views.argtypes = [P, I, P, I, P, P]
    L.hmlfc_render_views_relaxed.argtypes = [P, I, P, P, P, I, P, P]
    L.hmlfc_render_views_relaxed_ex.argtypes = [P, I, P, P, P, I, C.c_uint32, P, P]
    L.hmlfc_render_backward.argtypes = [P, I, P, I, P, P, P, P]
    L.hmlfc_dequant.argtypes = [P, P, P, P]
    L.hmlfc_encode.argtypes = [P, I, I, I, I, C.POINTER(EncodeParams), C.POINTER(P), C.POINTER(SZ)]
    L.hmlfc_encode_device.argtypes = [P, I, I, I, I, C.POINTER(EncodeParams), P, C.POINTER(P), C.POINTER(SZ),
                                      C.POINTER(EncodeStats)]
    L.hmlfc_set_encode_events.argtypes = [P, I]
    L.hmlfc_requantize.argtypes = [P, P, P, C.POINTER(P), C.POINTER(SZ)]
    L.hmlfc_free_host.argtypes = [P]
    L.hmlfc_free_host.restype = None
    L.hmlfc_touched_bytes.argtypes = [P, I, P, I, P]
    L.hmlfc_touched_bytes_union.argtypes = [P, I, P, I, P, P]
    L.hmlfc_set_render_path.argtypes = [I]
    L.hmlfc_set_block_cache_bytes.argtypes = [SZ]
    L.hmlfc_set_phase_events.argtypes = [P]
    L.hmlfc_render_batch.argtypes = [P, I, P, I, P, P]
    L.hmlfc_set_batch_tuning.argtypes = [I, I, I, SZ]
    _lib = L
    return L


def _check(rc: int):
    if rc != OK:
        raise HmlfcError(rc, lib().hmlfc_last_error().decode(errors="replace"))


def _stream_handle(cuda_stream):
    """Raw cudaStream_t of a torch stream (None -> torch's current stream)."""
    import torch
    if cuda_stream is None:
        cuda_stream = torch.cuda.current_stream()
    return C.c_void_p(int(cuda_stream.cuda_stream))


def _ptr(t) -> C.c_void_p:
    return C.c_void_p(int(t.data_ptr()))


def _views_array(views) -> "C.Array":
    """Accept a numpy record array of 96-byte views (see synthlf.VIEW_DTYPE)
    or a sequence of View structures."""
    if isinstance(views, np.ndarray):
        arr = np.ascontiguousarray(views)
        assert arr.dtype.itemsize == 96
        buf = (View * len(arr)).from_buffer_copy(arr.tobytes())
        return buf
    buf = (View * len(views))()
    for k, v in enumerate(views):
        buf[k] = v
    return buf


class Stream:
    """A compressed light field resident on the GPU (Sec. 4.8.2)."""

    def __init__(self, data: bytes, device: int = 0, cuda_stream=None):
        h = C.c_void_p()
        raw = bytes(data)
        _check(lib().hmlfc_load_stream(raw, len(raw), int(device), _stream_handle(cuda_stream), C.byref(h)))
        self._h = h
        self.device = device
        inf = StreamInfo()
        _check(lib().hmlfc_stream_info(self._h, C.byref(inf)))
        self.info = {f: getattr(inf, f) for f, _ in StreamInfo._fields_}

    @property
    def handle(self) -> C.c_void_p:
        if self._h is None:
            raise HmlfcError(E_INVALID_ARG, "stream already freed")
        return self._h

    def free(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            _lib.hmlfc_free_stream(self._h)
        self._h = None

    __del__ = free

    def decode_pixels(self, coords, out=None, cuda_stream=None, level: int = 0):
        """coords: int32 CUDA tensor [n, 4] = (i, j, x, y) -> uint8 [n, 3];
        level > 0: progressive decode down to that level only."""
        import torch
        assert coords.dtype == torch.int32 and coords.is_cuda and coords.is_contiguous()
        n = coords.shape[0]
        if out is None:
            out = torch.empty((n, 3), dtype=torch.uint8, device=coords.device)
        if level:
            _check(lib().hmlfc_decode_pixels_lod(self.handle, _ptr(coords), n, level, _ptr(out),
                                                 _stream_handle(cuda_stream)))
        else:
            _check(lib().hmlfc_decode_pixels(self.handle, _ptr(coords), n, _ptr(out), _stream_handle(cuda_stream)))
        return out

    def check_status(self, cuda_stream=None):
        _check(lib().hmlfc_check_status(self.handle, _stream_handle(cuda_stream)))

    def dequant(self, cuda_stream=None):
        """Dequantised coefficients [n_nc, H, W] and roots [n_roots, 3, H, W] (float32 CUDA)."""
        import torch
        i = self.info
        dev = torch.device("cuda", self.device)
        co = torch.empty((i["n_nc"], i["height"], i["width"]), dtype=torch.float32, device=dev)
        ro = torch.empty((i["n_roots"], 3, i["height"], i["width"]), dtype=torch.float32, device=dev)
        _check(lib().hmlfc_dequant(self.handle, _ptr(co), _ptr(ro), _stream_handle(cuda_stream)))
        return co, ro


def _streams_array(streams):
    arr = (C.c_void_p * len(streams))()
    for k, s in enumerate(streams):
        arr[k] = s.handle
    return arr


def out_size(views) -> int:
    """Elements of the output buffer the views need (max of offset + size)."""
    if isinstance(views, np.ndarray):
        if len(views) == 0:
            return 0
        return int(np.max(views["out_offset"] + views["width"].astype(np.int64) * views["height"] * 3))
    return max((v.out_offset + v.width * v.height * 3 for v in views), default=0)


MAX_VIEWS_PER_LAUNCH = 128       # views of one launch of the render kernels


def launches_per_render(views) -> int:
    """Kernels one hmlfc_render_views call launches on the cached path: per
    stream, the footprint marking and the blend once per launch chunk of its
    views, the slot assignment and the block decode once."""
    lfs = np.asarray(views["lf"])
    sizes = np.asarray(views["width"]).astype(np.int64) * np.asarray(views["height"])
    n = 0
    for lf in np.unique(lfs[sizes > 0]):
        chunks = -(-int(np.sum((lfs == lf) & (sizes > 0))) // MAX_VIEWS_PER_LAUNCH)
        n += 2 * chunks + 2
    return n


def render_views(streams, views, out=None, cuda_stream=None, level: int = 0):
    """Fused decode + render of novel views (float32 [sum H*W*3] CUDA tensor);
    level > 0 renders from the progressive decode at that level."""
    import torch
    va = _views_array(views)
    if out is None:
        out = torch.empty(out_size(views), dtype=torch.float32, device=torch.device("cuda", streams[0].device))
    if level:
        _check(lib().hmlfc_render_views_lod(_streams_array(streams), len(streams), va, len(va), level, _ptr(out),
                                            _stream_handle(cuda_stream)))
    else:
        _check(lib().hmlfc_render_views(_streams_array(streams), len(streams), va, len(va), _ptr(out),
                                        _stream_handle(cuda_stream)))
    return out


def render_views_host(streams, views, out=None, cuda_stream=None):
    """render_views into host memory (a page-locked float32 CPU tensor of
    out_size(views) floats): decode once, blend in groups of views, each group
    copied back while the next blends.  Asynchronous: out holds the views once
    the stream has synchronised."""
    import torch
    va = _views_array(views)
    if out is None:
        out = torch.empty(out_size(views), dtype=torch.float32, pin_memory=True)
    if out.is_cuda or out.dtype != torch.float32 or not out.is_contiguous() or out.numel() < out_size(views):
        raise ValueError("out must be a contiguous float32 host tensor of out_size(views) floats")
    _check(lib().hmlfc_render_views_host(_streams_array(streams), len(streams), va, len(va), _ptr(out),
                                         _stream_handle(cuda_stream)))
    return out


def render_batch(streams, views, out=None, cuda_stream=None):
    """Batched form: every view of every stream in one pass (persistent
    kernels, graph-capturable); same output as render_views."""
    import torch
    va = _views_array(views)
    if out is None:
        out = torch.empty(out_size(views), dtype=torch.float32, device=torch.device("cuda", streams[0].device))
    _check(lib().hmlfc_render_batch(_streams_array(streams), len(streams), va, len(va), _ptr(out),
                                    _stream_handle(cuda_stream)))
    return out


def set_batch_tuning(tile_shape: int = 0, group: int = 4, ctas_per_sm: int = 8, cache_bytes: int = 0):
    _check(lib().hmlfc_set_batch_tuning(int(tile_shape), int(group), int(ctas_per_sm), int(cache_bytes)))


RELAX_BIAS = 1


def render_views_relaxed(streams, coeffs, roots, views, out=None, cuda_stream=None, bias: bool = False):
    """The relaxed render; with bias, each rounding it drops carries its
    expected value (HMLFC_RELAX_BIAS)."""
    import torch
    va = _views_array(views)
    if out is None:
        out = torch.empty(out_size(views), dtype=torch.float32, device=torch.device("cuda", streams[0].device))
    cp = (C.c_void_p * len(streams))(*[int(t.data_ptr()) for t in coeffs])
    rp = (C.c_void_p * len(streams))(*[int(t.data_ptr()) for t in roots])
    _check(lib().hmlfc_render_views_relaxed_ex(_streams_array(streams), len(streams), cp, rp, va, len(va),
                                               RELAX_BIAS if bias else 0, _ptr(out), _stream_handle(cuda_stream)))
    return out


def render_backward(streams, views, grad_out, grad_coeffs, grad_roots, cuda_stream=None):
    """Accumulates the adjoint of the relaxed render into the given buffers."""
    va = _views_array(views)
    gc = (C.c_void_p * len(streams))(*[int(t.data_ptr()) for t in grad_coeffs])
    gr = (C.c_void_p * len(streams))(*[int(t.data_ptr()) for t in grad_roots])
    _check(lib().hmlfc_render_backward(_streams_array(streams), len(streams), va, len(va), _ptr(grad_out), gc, gr,
                                       _stream_handle(cuda_stream)))


RENDER_CACHED, RENDER_DIRECT, RENDER_TILE = 0, 1, 2


def set_render_path(path: int):
    """0: decoded-block cache per call (default); 1: per-ray decode; 2: per-tile staging."""
    _check(lib().hmlfc_set_render_path(int(path)))


def set_phase_events(events):
    """Record four torch.cuda.Events at the cached render's phase boundaries
    (before mark, before decode, before blend, end); None stops."""
    if events is None:
        _check(lib().hmlfc_set_phase_events(None))
        return
    for e in events:
        e.record()            # torch creates the CUDA event at its first record
    arr = (C.c_void_p * 4)(*[int(e.cuda_event) for e in events])
    _check(lib().hmlfc_set_phase_events(arr))


def set_encode_events(events):
    """torch.cuda.Event list (2 per level, top level first) recorded around
    the block-search passes of encode_device; None turns it off."""
    if not events:
        _check(lib().hmlfc_set_encode_events(None, 0))
        return
    for e in events:
        e.record()            # torch creates the CUDA event at its first record
    arr = (C.c_void_p * len(events))(*[int(e.cuda_event) for e in events])
    _check(lib().hmlfc_set_encode_events(arr, len(events)))


DEFAULT_CACHE_BYTES = 8 << 30     # the library's default scratch budget of one cached render call


def set_block_cache_bytes(n: int):
    """Scratch budget of one cached render call (index + decoded camera
    images of W * H * 4 bytes each); cameras beyond it decode per ray, and a
    budget below one image uses the per-tile path."""
    _check(lib().hmlfc_set_block_cache_bytes(int(n)))


def encode(lf: np.ndarray, levels: int, block: int, search: int, qstep: int, t_ref: int = 0, t_pred: int = 0,
           mc: int = MC_QPEL, threads: int = 0, sub: int = 0) -> bytes:
    """Encode uint8 [nu][nv][H][W][3] into an HMLFC stream (host threads);
    sub = 1: chroma sub-sampled 4:2:0 (Sec. 4.5)."""
    lf = np.ascontiguousarray(lf, np.uint8)
    nu, nv, H, W, _ = lf.shape
    prm = EncodeParams(levels, block, search, qstep, t_ref, t_pred, mc, threads, sub)
    out = C.c_void_p()
    n = C.c_size_t()
    _check(lib().hmlfc_encode(lf.ctypes.data_as(C.c_void_p), nu, nv, W, H, C.byref(prm), C.byref(out), C.byref(n)))
    data = C.string_at(out, n.value)
    lib().hmlfc_free_host(out)
    return data


def encode_device(lf, levels: int, block: int, search: int, qstep: int, t_ref: int = 0, t_pred: int = 0,
                  mc: int = MC_QPEL, cuda_stream=None, stats: dict | None = None) -> bytes:
    """Encode on the GPU; the same stream as encode().  lf: uint8
    [nu][nv][H][W][3], a CUDA tensor (used in place) or a host array (copied
    to the device first).  A dict passed as stats receives the work counts."""
    import torch
    if not isinstance(lf, torch.Tensor):
        lf = torch.from_numpy(np.ascontiguousarray(lf, np.uint8))
    if not lf.is_cuda:
        lf = lf.cuda()
    if lf.dtype != torch.uint8 or lf.dim() != 5 or lf.shape[4] != 3:
        raise ValueError("lf must be uint8 [nu][nv][H][W][3]")
    lf = lf.contiguous()
    nu, nv, H, W, _ = lf.shape
    prm = EncodeParams(levels, block, search, qstep, t_ref, t_pred, mc, 0, 0)
    out = C.c_void_p()
    n = C.c_size_t()
    st = EncodeStats()
    _check(lib().hmlfc_encode_device(_ptr(lf), nu, nv, W, H, C.byref(prm), _stream_handle(cuda_stream),
                                     C.byref(out), C.byref(n), C.byref(st)))
    if stats is not None:
        stats.update({k: int(getattr(st, k)) for k, _ in EncodeStats._fields_})
    data = C.string_at(out, n.value)
    lib().hmlfc_free_host(out)
    return data


def requantize(stream: Stream, coeff: np.ndarray, root: np.ndarray) -> bytes:
    co = np.ascontiguousarray(coeff, np.float32)
    ro = np.ascontiguousarray(root, np.float32)
    out = C.c_void_p()
    n = C.c_size_t()
    _check(lib().hmlfc_requantize(stream.handle, co.ctypes.data_as(C.c_void_p), ro.ctypes.data_as(C.c_void_p),
                                  C.byref(out), C.byref(n)))
    data = C.string_at(out, n.value)
    lib().hmlfc_free_host(out)
    return data


def touched_bytes_union(streams, views, with_blocks: bool = False, level: int = 0):
    """Compulsory bytes of a whole call: distinct items counted once; with
    with_blocks also the number of distinct (camera, block) pairs reached
    ((node, block) pairs at a progressive level > 0)."""
    va = _views_array(views)
    out = C.c_double()
    nb = C.c_double()
    _check(lib().hmlfc_touched_bytes_union_lod(_streams_array(streams), len(streams), va, len(va), level,
                                               C.byref(out), C.byref(nb)))
    return (out.value, nb.value) if with_blocks else out.value


def touched_bytes(streams, views) -> np.ndarray:
    va = _views_array(views)
    out = np.zeros(len(va), np.float64)
    _check(lib().hmlfc_touched_bytes(_streams_array(streams), len(streams), va, len(va),
                                     out.ctypes.data_as(C.c_void_p)))
    return out
