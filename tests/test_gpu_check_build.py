"""The bounds-checked build (HMLFC_CHECK): every kernel read of a stream
array is checked against the array's length, and a read outside it sets a
status bit that hmlfc_check_status reports.  The tiny and ragged parity
workloads -- full-resolution and 4:2:0 chroma, block sizes 16, 8, 5 and 4,
every render path, progressive levels, the batched, serving and relaxed
forms -- run in a child process on that build: results equal the oracle's
(samples bit for bit, views within 1e-3) and no check fires.  The checks
stand in for a memory checker, which this pool does not provide."""
import os
import subprocess
import sys
from pathlib import Path

import pytest

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

ROOT = Path(__file__).resolve().parent.parent

CHILD = r'''
import numpy as np, torch
import oracle as O, synthlf as S
import paper_1902_09396_gb300 as H
from paper_1902_09396_gb300.serve import ResidentCache
assert "_build_check" in str(H.lib()._name), H.lib()._name
tiny = S.CONFIGS["tiny"]
lf_t = S.make_lf(tiny.seed, tiny.nu, tiny.nv, tiny.width, tiny.height, tiny.n_planes, tiny.disp_max, tiny.texture)
lf_r = S.make_lf(11, 5, 3, 37, 29, 3, 4.0, "pink")
cases = [(lf_t, O.encode(lf_t, tiny.levels, tiny.block, tiny.search, tiny.qstep).stream, tiny.levels),
         (lf_t, O.encode(lf_t, tiny.levels, 16, tiny.search, 2, sub=1).stream, tiny.levels),
         (lf_r, O.encode(lf_r, 3, 8, 4, 2, t_ref=20, t_pred=30).stream, 3),
         (lf_r, O.encode(lf_r, 3, 8, 4, 2, sub=1).stream, 3),
         (lf_r, O.encode(lf_r, 2, 5, 3, 3, mc=O.MC_INTEGER).stream, 2),
         (lf_r, O.encode(lf_r, 2, 4, 2, 1, sub=1).stream, 2)]
for lf, data, L in cases:
    st, ost = H.Stream(data), O.Stream(data)
    nu, nv, Hh, W = lf.shape[:4]
    ii, jj, xx, yy = np.meshgrid(np.arange(nu), np.arange(nv), np.arange(W), np.arange(Hh), indexing="ij")
    co = np.stack([ii, jj, xx, yy], -1).reshape(-1, 4).astype(np.int32)
    dec = ost.decode_all()
    def status(what):
        torch.cuda.synchronize()
        try:
            st.check_status()
        except H.HmlfcError as e:
            raise AssertionError(f"{what}: {e}")
    for level in range(L + 1):
        got = st.decode_pixels(torch.from_numpy(co).cuda(), level=level).cpu().numpy()
        want = dec[co[:, 0], co[:, 1], co[:, 3], co[:, 2]] if level == 0 else ost.decode_samples(co, level=level)
        assert np.array_equal(got, want), ("decode", level)
        status(f"decode_pixels level {level}")
    geo = S.lf_geometry(nu, nv, W, Hh)
    views = S.views_to_array(S.random_views(71, geo, 4, [(48, 40), (17, 9)]))
    ref = O.render_dense(dec, views)
    outs = []
    for path in (0, 1, 2):
        H.set_render_path(path)
        outs.append(H.render_views([st], views).cpu().numpy())
        status(f"render path {path}")
    H.set_render_path(0)
    H.set_block_cache_bytes(3 * W * Hh * 4)
    outs.append(H.render_views([st], views).cpu().numpy())
    status("render with a few camera images")
    H.set_block_cache_bytes(H.DEFAULT_CACHE_BYTES)
    outs.append(H.render_batch([st], views).cpu().numpy())
    status("render_batch")
    for o in outs:
        assert np.max(np.abs(o.astype(np.float64) - ref)) <= 1e-3, "render"
    for level in range(1, L + 1):
        H.render_views([st], views, level=level)
        status(f"render level {level}")
    cache = ResidentCache(st, 1 << 20)
    out = torch.zeros(H.out_size(views), dtype=torch.float32, device="cuda")
    cache.render(views, out)
    assert np.array_equal(out.cpu().numpy(), outs[0]), "serve"
    status("serve")
    if not st.info["chroma"]:
        co_, ro_ = st.dequant()
        H.render_views_relaxed([st], [co_], [ro_], views)
        status("relaxed render")
print("check build ok")
'''


def test_parity_workloads_under_the_bounds_checked_build():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1902_09396_gb300.build import build
    lib = build(check=True)
    env = dict(os.environ, HMLFC_LIB=str(lib), PYTHONPATH=str(ROOT))
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=str(ROOT), env=env, capture_output=True, text=True,
                       timeout=1800)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "check build ok" in r.stdout
