"""Plain CPU oracle of HMLFC (arXiv 1902.09396) -- TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library shares no code
with it: the C source ``hmlfc_oracle.c`` has its own stream writer, reader,
decoder and renderer, and is compiled into its own shared object here with
gcc.  Each wrapper below states which section of the paper it follows; the C
file gives the step-by-step reading.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass
from pathlib import Path

import numpy as np

_DIR = Path(__file__).resolve().parent
_SRC = _DIR / "hmlfc_oracle.c"
_OUT = _DIR / "_build" / "liboracle.so"

E_OK, E_ARG, E_CORRUPT, E_OOM, E_RANGE = 0, -1, -2, -3, -4


def build(force: bool = False) -> Path:
    """Compile the oracle with gcc (plain C11 + OpenMP)."""
    if not force and _OUT.exists() and _OUT.stat().st_mtime >= _SRC.stat().st_mtime:
        return _OUT
    _OUT.parent.mkdir(parents=True, exist_ok=True)
    tmp = _OUT.with_suffix(f".{os.getpid()}.tmp")
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-Wall",
           "-o", str(tmp), str(_SRC), "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _OUT)
    return _OUT


_lib = None


def load(path) -> C.CDLL:
    """Load an oracle shared object (the default build, or a test variant)."""
    L = C.CDLL(str(path))
    _bind(L)
    return L


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = load(_OUT)
    return _lib


class using:
    """Context manager: route this module's wrappers to another build of the
    oracle (used by the tests that plant mistakes in a copy of the source)."""

    def __init__(self, path):
        self.path = path

    def __enter__(self):
        global _lib
        self.prev = _lib
        _lib = load(self.path)
        return _lib

    def __exit__(self, *exc):
        global _lib
        _lib = self.prev


def build_variant(src_text: str, out_path) -> Path:
    """Compile C source text (e.g. a mutated copy of the oracle) to out_path."""
    out_path = Path(out_path)
    out_path.parent.mkdir(parents=True, exist_ok=True)
    src = out_path.with_suffix(".c")
    src.write_text(src_text)
    subprocess.run(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-w",
                    "-o", str(out_path), str(src), "-lm"], check=True)
    return out_path


def source_text() -> str:
    return _SRC.read_text()


def _bind(L):
    """Declare the C signatures on a loaded oracle object."""
    P, I, I64, SZ = C.c_void_p, C.c_int, C.c_int64, C.c_size_t
    L.orc_encode.argtypes = [P, P, C.POINTER(C.c_void_p), C.POINTER(SZ), P, P]
    L.orc_free.argtypes = [P]
    L.orc_open.argtypes = [P, SZ, C.POINTER(C.c_void_p)]
    L.orc_close.argtypes = [P]
    L.orc_stream_info.argtypes = [P, P]
    L.orc_decode_samples.argtypes = [P, P, I64, P, P]
    L.orc_decode_samples_lod.argtypes = [P, P, I64, I, P, P]
    L.orc_render_pixels_lod.argtypes = [P, P, I, P, I64, I, P]
    L.orc_touched_bytes_lod.argtypes = [P, P, I, I, P]
    L.orc_decode_all.argtypes = [P, P, P]
    L.orc_block_info.argtypes = [P, I64, I, P]
    L.orc_dequant.argtypes = [P, P, P]
    L.orc_render_dense.argtypes = [P, I, I, I, I, P, I, P]
    L.orc_render_pixels.argtypes = [P, P, I, P, I64, P]
    L.orc_relax_render.argtypes = [P, P, P, P, I, P]
    L.orc_relax_render_ex.argtypes = [P, P, P, P, I, I, P]
    L.orc_mc_rounding_bias.argtypes = [I, I]
    L.orc_mc_rounding_bias.restype = C.c_double
    L.orc_relax_adjoint.argtypes = [P, P, I, P, P, P]
    L.orc_touched_bytes.argtypes = [P, P, I, P]
    L.orc_rgb_to_ycocg.argtypes = [I, I, I, P, P, P]
    L.orc_ycocg_to_rgb.argtypes = [I, I, I, P, P, P]
    L.orc_quantise.argtypes = [I, I]
    L.orc_pred_qpel.argtypes = [P, I, I, I, I, I, I]
    L.orc_bise_choose.argtypes = [C.c_uint32, P, P]
    L.orc_bise_bits.argtypes = [I, I, C.c_uint64]
    L.orc_bise_bits.restype = C.c_uint64
    L.orc_bise_pack.argtypes = [P, I, I, P, C.c_uint64]
    L.orc_bise_get.argtypes = [P, I, I, C.c_uint64]
    L.orc_bise_get.restype = C.c_int64
    L.orc_bise_unpack.argtypes = [P, I, I, P, C.c_uint64]
    L.orc_set_threads.argtypes = [I]
    L.orc_mc_search_block.argtypes = [P, P, I, I, I, I, I, I, P]


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _check(rc: int, what: str):
    if rc != E_OK:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def get_threads() -> int:
    return int(lib().orc_get_threads())


# --------------------------------------------------------------------------
# small pieces, exposed for the pins
# --------------------------------------------------------------------------

def rgb_to_ycocg(r: int, g: int, b: int):
    """Sec. 4.5: forward YCoCg-R lifting."""
    y, co, cg = C.c_int(), C.c_int(), C.c_int()
    lib().orc_rgb_to_ycocg(r, g, b, C.byref(y), C.byref(co), C.byref(cg))
    return y.value, co.value, cg.value


def ycocg_to_rgb(y: int, co: int, cg: int):
    """Sec. 4.5: inverse YCoCg-R lifting."""
    r, g, b = C.c_int(), C.c_int(), C.c_int()
    lib().orc_ycocg_to_rgb(y, co, cg, C.byref(r), C.byref(g), C.byref(b))
    return r.value, g.value, b.value


def mc_search_block(S: np.ndarray, R: np.ndarray, block: int, k: int, search: int, refine: bool):
    """Phase-shifted search of block k (Sec. 4.4): (mvx, mvy, sign, cost)."""
    S = np.ascontiguousarray(S, np.int32)
    R = np.ascontiguousarray(R, np.int16)
    h, w = S.shape
    out = np.zeros(4, np.int64)
    _check(lib().orc_mc_search_block(_p(S), _p(R), w, h, block, k, search, int(refine), _p(out)), "search")
    return tuple(int(x) for x in out)


def quantise(r: int, q: int) -> int:
    return int(lib().orc_quantise(int(r), int(q)))


def pred_qpel(plane: np.ndarray, x: int, y: int, mvx: int, mvy: int) -> int:
    """Quarter-pel motion-compensated prediction of pixel (x, y) from an int16
    reference plane (Sec. 4.4, sub-pel per Sec. 6)."""
    plane = np.ascontiguousarray(plane, np.int16)
    h, w = plane.shape
    return int(lib().orc_pred_qpel(_p(plane), w, h, x, y, mvx, mvy))


def bise_choose(rng: int):
    """Sec. 4.6: smallest N in {2^b, 3*2^b, 5*2^b} >= rng -> (mode, b)."""
    m, b = C.c_int(), C.c_int()
    lib().orc_bise_choose(C.c_uint32(rng), C.byref(m), C.byref(b))
    return m.value, b.value


def bise_bits(mode: int, b: int, n: int) -> int:
    return int(lib().orc_bise_bits(mode, b, n))


def bise_pack(values, mode: int, b: int) -> np.ndarray:
    v = np.ascontiguousarray(values, np.uint32)
    words = (bise_bits(mode, b, len(v)) + 31) // 32
    buf = np.zeros(max(words, 1) + 1, np.uint32)
    lib().orc_bise_pack(_p(buf), mode, b, _p(v), len(v))
    return buf[:words]


def bise_get(buf: np.ndarray, mode: int, b: int, i: int) -> int:
    buf = np.ascontiguousarray(np.concatenate([buf, np.zeros(2, np.uint32)]), np.uint32)
    return int(lib().orc_bise_get(_p(buf), mode, b, i))


def bise_unpack(buf: np.ndarray, mode: int, b: int, n: int) -> np.ndarray:
    buf = np.ascontiguousarray(np.concatenate([buf, np.zeros(2, np.uint32)]), np.uint32)
    out = np.zeros(n, np.uint32)
    _check(lib().orc_bise_unpack(_p(buf), mode, b, _p(out), n), "bise_unpack")
    return out


# --------------------------------------------------------------------------
# encoder
# --------------------------------------------------------------------------

class _Params(C.Structure):
    _fields_ = [(n, C.c_int32) for n in
                ("nu", "nv", "W", "H", "L", "B", "Ws", "q", "t_ref", "t_pred", "mc", "sub")]


MC_OFF, MC_QPEL, MC_ZERO, MC_INTEGER = 0, 1, 2, 3


@dataclass
class EncodeResult:
    stream: bytes
    S: np.ndarray | None = None       # [n_nc][H][W] SRV before motion compensation
    Rhat: np.ndarray | None = None    # [n_nc][H][W] dequantised reference SRVs


def encode(lf: np.ndarray, levels: int, block: int, search: int, qstep: int,
           t_ref: int = 0, t_pred: int = 0, mc: int = MC_QPEL, debug: bool = False, sub: int = 0) -> EncodeResult:
    """HMLFC encoder (Sec. 4.3-4.7): hierarchy, closed-loop phase-shifted MC,
    quantiser + two block thresholds, BISE, breadth-first stream.  sub = 1:
    chroma sub-sampled 4:2:0 (Sec. 4.5; Co, Cg coded at half resolution)."""
    lf = np.ascontiguousarray(lf, np.uint8)
    nu, nv, H, W, _ = lf.shape
    prm = _Params(nu, nv, W, H, levels, block, search, qstep, t_ref, t_pred, mc, sub)
    out = C.c_void_p()
    n = C.c_size_t()
    S = R = None
    if debug:
        n_nc = 3 * sum(((nu + (1 << l) - 1) >> l) * ((nv + (1 << l) - 1) >> l) for l in range(levels))
        S = np.zeros((n_nc, H, W), np.int32)
        R = np.zeros((n_nc, H, W), np.int32)
    rc = lib().orc_encode(C.byref(prm), _p(lf), C.byref(out), C.byref(n),
                          _p(S) if debug else None, _p(R) if debug else None)
    _check(rc, "encode")
    data = C.string_at(out, n.value)
    lib().orc_free(out)
    return EncodeResult(data, S, R)


# --------------------------------------------------------------------------
# decoder / renderer
# --------------------------------------------------------------------------

def _views(views) -> np.ndarray:
    arr = np.ascontiguousarray(views)
    assert arr.dtype.itemsize == 96, "views must use the 96-byte view record"
    return arr


def _out_len(views) -> int:
    v = _views(views)
    return int(max((int(r["out_offset"]) + int(r["width"]) * int(r["height"]) * 3) for r in v)) if len(v) else 0


class Stream:
    """A parsed stream (Sec. 4.7) with the decoding entry points (Sec. 4.8)."""

    def __init__(self, data: bytes):
        self._buf = np.frombuffer(data, np.uint8).copy()
        h = C.c_void_p()
        _check(lib().orc_open(_p(self._buf), len(self._buf), C.byref(h)), "open")
        self._h = h
        info = np.zeros(17, np.int32)
        lib().orc_stream_info(self._h, _p(info))
        (self.nu, self.nv, self.W, self.H, self.L, self.B, self.Ws, self.q, self.mc,
         self.n_nc, self.nblocks, self.n_sig, self.n_rec_words, self.n_mv, self.n_roots,
         self.nbytes, self.sub) = (int(x) for x in info)

    def close(self):
        if getattr(self, "_h", None):
            lib().orc_close(self._h)
            self._h = None

    __del__ = close

    # -- decoding -----------------------------------------------------------
    def decode_samples(self, coords: np.ndarray, with_ycocg: bool = False, level: int = 0):
        """Random-access decoding (Sec. 4.8.1) of samples (i, j, x, y) -> RGB8;
        level > 0: progressive decoding down to that level."""
        c = np.ascontiguousarray(coords, np.int32).reshape(-1, 4)
        rgb = np.zeros((len(c), 3), np.uint8)
        ycc = np.zeros((len(c), 3), np.int32) if with_ycocg else None
        _check(lib().orc_decode_samples_lod(self._h, _p(c), len(c), level, _p(rgb), _p(ycc) if with_ycocg else None),
               "decode_samples")
        return (rgb, ycc) if with_ycocg else rgb

    def decode_all(self, with_ycocg: bool = False):
        """Full top-down reconstruction -> uint8 [nu][nv][H][W][3]."""
        out = np.zeros((self.nu, self.nv, self.H, self.W, 3), np.uint8)
        ycc = np.zeros((self.nu, self.nv, 3, self.H, self.W), np.int32) if with_ycocg else None
        _check(lib().orc_decode_all(self._h, _p(out), _p(ycc) if with_ycocg else None), "decode_all")
        return (out, ycc) if with_ycocg else out

    def block_info(self, nc: int, k: int):
        """(significant, mvx, mvy, sign) of block k of node-channel nc."""
        o = np.zeros(4, np.int32)
        _check(lib().orc_block_info(self._h, nc, k, _p(o)), "block_info")
        return tuple(int(x) for x in o)

    def dequant(self):
        """Dequantised coefficients [n_nc][H][W] and roots [n_roots][3][H][W] (float64)."""
        co = np.zeros((self.n_nc, self.H, self.W), np.float64)
        ro = np.zeros((self.n_roots, 3, self.H, self.W), np.float64)
        _check(lib().orc_dequant(self._h, _p(co), _p(ro)), "dequant")
        return co, ro

    # -- rendering ----------------------------------------------------------
    def render_pixels(self, views, pix: np.ndarray, level: int = 0) -> np.ndarray:
        """FP64 render of selected (view, px, py) by random-access decoding
        (down to `level`)."""
        v = _views(views)
        p = np.ascontiguousarray(pix, np.int32).reshape(-1, 3)
        out = np.zeros((len(p), 3), np.float64)
        _check(lib().orc_render_pixels_lod(self._h, _p(v), len(v), _p(p), len(p), level, _p(out)), "render_pixels")
        return out

    def relax_render(self, coeff: np.ndarray, roots: np.ndarray, views, bias: bool = False) -> np.ndarray:
        """The relaxed render; with bias, every dropped rounding carries its
        expected value (orc_mc_rounding_bias per predictor, -1/4 per >> 1)."""
        v = _views(views)
        co = np.ascontiguousarray(coeff, np.float64)
        ro = np.ascontiguousarray(roots, np.float64)
        out = np.zeros(_out_len(v), np.float64)
        _check(lib().orc_relax_render_ex(self._h, _p(co), _p(ro), _p(v), len(v), int(bool(bias)), _p(out)),
               "relax_render")
        return out

    def relax_adjoint(self, views, grad_out: np.ndarray):
        v = _views(views)
        g = np.ascontiguousarray(grad_out, np.float64)
        gc = np.zeros((self.n_nc, self.H, self.W), np.float64)
        gr = np.zeros((self.n_roots, 3, self.H, self.W), np.float64)
        _check(lib().orc_relax_adjoint(self._h, _p(v), len(v), _p(g), _p(gc), _p(gr)), "relax_adjoint")
        return gc, gr

    def touched_bytes(self, views, level: int = 0) -> np.ndarray:
        v = _views(views)
        out = np.zeros(len(v), np.float64)
        _check(lib().orc_touched_bytes_lod(self._h, _p(v), len(v), level, _p(out)), "touched_bytes")
        return out


def render_dense(lf: np.ndarray, views) -> np.ndarray:
    """FP64 quadrilinear render (Sec. 2.1 two-plane rays) from a dense RGB8
    light field; returns the flat output buffer (views at their offsets)."""
    lf = np.ascontiguousarray(lf, np.uint8)
    nu, nv, H, W, _ = lf.shape
    v = _views(views)
    out = np.zeros(_out_len(v), np.float64)
    _check(lib().orc_render_dense(_p(lf), nu, nv, W, H, _p(v), len(v), _p(out)), "render_dense")
    return out


def psnr(a: np.ndarray, b: np.ndarray, peak: float = 255.0) -> float:
    """10 log10(peak^2 / MSE) over all samples."""
    d = a.astype(np.float64) - b.astype(np.float64)
    mse = float(np.mean(d * d))
    return float("inf") if mse == 0 else 10.0 * np.log10(peak * peak / mse)


def mc_rounding_bias(mvx: int, mvy: int) -> float:
    """Expected rounding of the integer predictor at quarter-pel motion
    (mvx, mvy) against its exact weighted sum (orc_mc_rounding_bias)."""
    return float(lib().orc_mc_rounding_bias(int(mvx), int(mvy)))
