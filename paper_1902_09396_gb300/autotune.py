"""Autotuner of the batched render (hmlfc_render_batch).

Candidates: rays per tile (16x16, 32x8, 8x8), decode items per pass (1, 2,
4 -- how many (level-2 node, block) items a CTA builds descriptors for
before decoding them) and decode CTAs launched per SM (5: all resident,
10, 32).  Each candidate
renders the caller's own batch a few times under CUDA events; the fastest is
set and remembered per workload signature (stream shapes and the histogram of
view sizes) in a JSON file next to the built library.
"""
from __future__ import annotations

import hashlib
import json
import os
from pathlib import Path

import numpy as np

from . import render_batch, set_batch_tuning
from .build import OUT_DIR

CANDIDATES = [(t, g, c) for t in (0, 1, 2) for g in (1, 2, 4) for c in (5, 10, 32)]
CACHE_FILE = OUT_DIR / "autotune.json"


def signature(streams, views) -> str:
    shapes = [tuple(int(s.info[k]) for k in ("nu", "nv", "width", "height", "levels", "block")) for s in streams]
    arr = np.asarray(views)
    sizes = sorted(set(zip(arr["width"].tolist(), arr["height"].tolist())))
    hist = [(w, h, int(np.sum((arr["width"] == w) & (arr["height"] == h)))) for w, h in sizes]
    return hashlib.sha1(json.dumps([shapes, hist]).encode()).hexdigest()[:16]


def _load(path: Path) -> dict:
    try:
        return json.loads(path.read_text())
    except Exception:
        return {}


def tune(streams, views, out, reps: int = 3, candidates=CANDIDATES, cache_file: Path | None = CACHE_FILE,
         force: bool = False) -> dict:
    """Pick and set the fastest candidate for this batch; returns
    {"tuning": (tile, group, ctas), "ms": best time, "table": {cand: ms}}."""
    import torch
    sig = signature(streams, views)
    cache = _load(cache_file) if cache_file else {}
    if not force and sig in cache:
        best = tuple(cache[sig]["tuning"])
        set_batch_tuning(*best)
        return cache[sig]
    table = {}
    for cand in candidates:
        set_batch_tuning(*cand)
        render_batch(streams, views, out)            # warm-up
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            render_batch(streams, views, out)
        e1.record()
        torch.cuda.synchronize()
        table[str(cand)] = e0.elapsed_time(e1) / reps
    best = min(candidates, key=lambda c: table[str(c)])
    set_batch_tuning(*best)
    res = {"tuning": list(best), "ms": table[str(best)], "table": table}
    if cache_file:
        cache[sig] = res
        try:
            cache_file.parent.mkdir(parents=True, exist_ok=True)
            tmp = cache_file.with_suffix(f".{os.getpid()}.tmp")
            tmp.write_text(json.dumps(cache, indent=1))
            os.replace(tmp, cache_file)
        except OSError:
            pass
    return res
