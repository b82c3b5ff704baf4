"""Differentiable form: gradients of a rendered-view loss with respect to the
dequantised residual coefficients and the root images, through the library's
adjoint kernel and the autograd wrapper.

- The gradient equals the FP64 oracle's transpose of the relaxed render, at
  the differentiable form's size (9x9 grid of 256x256 views, 3 levels,
  32 random 256x256 views).
- It equals FP64 central finite differences of the oracle's relaxed render
  on 1000 sampled coefficients (reduced field: the loss is quadratic, so the
  differences are exact up to rounding).
- A few Adam steps lower the loss, and the re-quantised stream decodes.
"""
import numpy as np
import pytest

import oracle as O
import synthlf as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.fixture(scope="module")
def diff_setup():
    c = S.CONFIGS["diff"]
    lf = S.make_lf(c.seed, c.nu, c.nv, c.width, c.height, c.n_planes, c.disp_max, c.texture)
    data = O.encode(lf, c.levels, c.block, c.search, c.qstep).stream
    geo = S.lf_geometry(c.nu, c.nv, c.width, c.height)
    views = S.views_to_array(S.random_views(c.seed, geo, 32, [(256, 256)]))
    return c, lf, data, views


def test_gradient_matches_oracle_adjoint(torch_cuda, diff_setup):
    torch = torch_cuda
    import paper_1902_09396_gb300 as H
    from paper_1902_09396_gb300.torch_ops import relaxed_render
    c, lf, data, views = diff_setup
    st = H.Stream(data)
    coeff, root = st.dequant()
    coeff.requires_grad_(True)
    root.requires_grad_(True)
    rng = np.random.default_rng(7)
    n = H.out_size(views)
    target = torch.tensor(rng.random(n), dtype=torch.float32, device="cuda")
    out = relaxed_render(coeff, root, st, views)
    loss = torch.sum((out - target) ** 2)
    loss.backward()
    g_out = (2.0 * (out.detach() - target)).double().cpu().numpy()
    ost = O.Stream(data)
    wc, wr = ost.relax_adjoint(views, g_out)
    scale = max(np.max(np.abs(wc)), np.max(np.abs(wr)))
    assert np.max(np.abs(coeff.grad.cpu().numpy() - wc)) <= 2e-5 * scale
    assert np.max(np.abs(root.grad.cpu().numpy() - wr)) <= 2e-5 * scale
    assert np.count_nonzero(wc) > 0.05 * wc.size


def test_gradient_finite_differences(torch_cuda):
    """FP64 finite differences of the oracle's relaxed render, 1000
    coefficients (and 50 root pixels) sampled where the gradient is non-zero
    and elsewhere."""
    torch = torch_cuda
    import paper_1902_09396_gb300 as H
    from paper_1902_09396_gb300.torch_ops import relaxed_render
    lf = S.make_lf(17, 5, 5, 64, 64, 3, 4.0, "pink")
    data = O.encode(lf, 3, 8, 4, 4).stream
    geo = S.lf_geometry(5, 5, 64, 64)
    views = S.views_to_array(S.random_views(18, geo, 4, [(48, 48)]))
    st = H.Stream(data)
    ost = O.Stream(data)
    coeff, root = st.dequant()
    coeff.requires_grad_(True)
    root.requires_grad_(True)
    rng = np.random.default_rng(19)
    target = rng.random(H.out_size(views))
    out = relaxed_render(coeff, root, st, views)
    loss = torch.sum((out.double() - torch.tensor(target, device="cuda")) ** 2)
    loss.backward()
    gc = coeff.grad.cpu().numpy()
    gr = root.grad.cpu().numpy()
    co0, ro0 = ost.dequant()
    base_out = ost.relax_render(co0, ro0, views)
    hot = np.argwhere(gc != 0)
    pick = np.concatenate([hot[rng.choice(len(hot), 900, replace=False)],
                           np.stack([rng.integers(0, s, 100) for s in gc.shape], -1)])
    h = 1.0

    def L(o):
        return float(np.sum((o - target) ** 2))

    scale = np.max(np.abs(gc))
    for nc, y, x in pick:
        cp = co0.copy()
        cp[nc, y, x] += h
        cm = co0.copy()
        cm[nc, y, x] -= h
        fd = (L(ost.relax_render(cp, ro0, views)) - L(ost.relax_render(cm, ro0, views))) / (2 * h)
        assert abs(fd - gc[nc, y, x]) <= 1e-4 * scale + 1e-6 * abs(fd)
    for r in np.argwhere(gr != 0)[rng.choice(np.count_nonzero(gr), 50, replace=False)]:
        rp = ro0.copy()
        rp[tuple(r)] += h
        rm = ro0.copy()
        rm[tuple(r)] -= h
        fd = (L(ost.relax_render(co0, rp, views)) - L(ost.relax_render(co0, rm, views))) / (2 * h)
        assert abs(fd - gr[tuple(r)]) <= 1e-4 * max(scale, np.max(np.abs(gr))) + 1e-6 * abs(fd)
    assert np.isfinite(L(base_out))


def test_adam_refinement_and_requantisation(torch_cuda, tiny_streams, tiny_cfg, tiny_lf):
    """A few Adam steps towards views of the uncompressed field lower the
    loss; the refined coefficients re-quantise to a stream that loads and
    decodes (same motion vectors, same quantiser step)."""
    torch = torch_cuda
    import paper_1902_09396_gb300 as H
    from paper_1902_09396_gb300.torch_ops import refine, requantized_stream
    c = tiny_cfg
    st = H.Stream(tiny_streams[c.qstep].stream)
    lossless = H.Stream(H.encode(tiny_lf, c.levels, c.block, c.search, 1))
    geo = S.lf_geometry(c.nu, c.nv, c.width, c.height)
    views = S.views_to_array(S.random_views(44, geo, 6, [(64, 64)]))
    target = H.render_views([lossless], views)
    co, ro, losses = refine(st, views, target, steps=25)
    assert losses[-1] < losses[0]
    new = H.Stream(requantized_stream(st, co, ro))
    assert new.info["qstep"] == c.qstep and new.info["n_nc"] == st.info["n_nc"]
    out = H.render_views([new], views)
    torch.cuda.synchronize()
    assert torch.isfinite(out).all()
