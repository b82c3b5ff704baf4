"""Robustness of the host stream parser: seeded corruptions of a valid
stream (bit flips in every section, truncations, extensions) are either
rejected by validation (HMLFC_E_CORRUPT / UNSUPPORTED / INVALID_ARG) or, if
structurally valid, reach the device step -- which fails cleanly here, where
there is no GPU.  Nothing may crash: the loads run in a child process.
Runs on hosts without a CUDA device only (it never uploads a fuzzed stream)."""
import json
import subprocess
import sys
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parent.parent

CHILD = r"""
import ctypes as C, json, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
import paper_1902_09396_gb300 as H
good = open(sys.argv[2], "rb").read()
L = H.lib()
rng = np.random.default_rng(1234)
hdr = [int.from_bytes(good[4 * k:4 * k + 4], "little") for k in range(32)]
sections = [(hdr[21], hdr[22]), (hdr[22], hdr[23]), (hdr[23], hdr[24]), (hdr[24], hdr[25]), (hdr[25], hdr[26]),
            (0, 128)]
codes = {}
for t in range(400):
    b = bytearray(good)
    kind = t % 4
    if kind == 0:                                   # flips inside one section
        lo, hi = sections[int(rng.integers(len(sections)))]
        if hi <= lo:
            continue
        for _ in range(int(rng.integers(1, 6))):
            i = int(rng.integers(lo, hi))
            b[i] ^= 1 << int(rng.integers(8))
    elif kind == 1:                                 # a random 32-bit word anywhere
        i = int(rng.integers(0, len(b) // 4)) * 4
        b[i:i + 4] = int(rng.integers(0, 2**32)).to_bytes(4, "little")
    elif kind == 2:                                 # truncation
        b = b[:int(rng.integers(0, len(b)))]
    else:                                           # extension with junk
        b += bytes(rng.integers(0, 256, int(rng.integers(1, 64)), dtype=np.uint8))
    h = C.c_void_p()
    rc = L.hmlfc_load_stream(bytes(b), len(b), 0, None, C.byref(h))
    if rc == 0:
        L.hmlfc_free_stream(h)
    codes[rc] = codes.get(rc, 0) + 1
print(json.dumps({str(k): v for k, v in codes.items()}))
"""


def test_loader_survives_corrupt_streams(tmp_path, tiny_streams, tiny_cfg):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("fuzzed streams are only loaded on hosts without a CUDA device")
    import paper_1902_09396_gb300 as H
    H.build()
    src = tmp_path / "good.hmlf"
    src.write_bytes(tiny_streams[tiny_cfg.qstep].stream)
    r = subprocess.run([sys.executable, "-c", CHILD, str(ROOT), str(src)], capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    codes = {int(k): v for k, v in json.loads(r.stdout.strip().splitlines()[-1]).items()}
    allowed = {H.E_CORRUPT, H.E_UNSUPPORTED, H.E_INVALID_ARG, H.E_CUDA, H.E_OOM, H.OK}
    assert set(codes) <= allowed, codes
    assert codes.get(H.E_CORRUPT, 0) > 100          # most corruptions are caught by validation
