"""GPU implicit-function-theorem backward vs the FP64 oracle's backward (each at its own
fit of the same pixels), the invariance identities, and the autograd wrapper."""
import numpy as np
import pytest
import torch

from paper_2106_02045_gb300 import fitspots, synth

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")
TIGHT = dict(max_iter=50, min_delta=0.0, min_step=1e-6)   # tight stop FP32 can reach


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _upstream(n, seed):
    g = torch.Generator().manual_seed(seed)
    return (torch.randn(n, 4, generator=g), torch.randn(n, generator=g),
            torch.randn(n, generator=g), torch.randn(n, generator=g))


def test_backward_matches_oracle_ift_on_iso16():
    """16x16 isotropic spots (the backward workload): per-spot relative error of the
    pixel gradient against the oracle's FP64 backward <= 1e-4 on determined spots."""
    import oracle
    n = 1024
    b = synth.make_workload("iso16", n)
    g = b.to(DEV)
    out = fitspots.fit_batch(g, **TIGHT)
    gp, ga, gb, gc = _upstream(n, 3)
    grad = fitspots.backward(g.images, g.offsets, g.dims, g.model, out, gp, ga, gb, gc)
    torch.cuda.synchronize()
    grad = grad.cpu().numpy()
    d = b.numpy()
    img = synth.as_numpy_images(b)
    ref = oracle.fit_spots(img, d["offsets"], d["dims"], d["init"], d["model"], max_iter=300,
                           min_delta=0.0, min_step=1e-13)
    errs = []
    for s in range(n):
        off = int(d["offsets"][s])
        gs = img[off:off + 256].astype(np.float64)
        up = np.concatenate([gp[s].numpy(), [ga[s], gb[s], gc[s]]]).astype(np.float64)
        ro = oracle.backward(0, 16, 16, gs, ref["params"][s], ref["alpha"][s], ref["beta"][s], up)
        assert ro is not None
        errs.append(np.linalg.norm(grad[off:off + 256] - ro) / np.linalg.norm(ro))
    errs = np.array(errs)
    st = out["state"].cpu().numpy()
    print(f"iso16 backward: median rel err {np.median(errs):.2e}, p99 {np.percentile(errs, 99):.2e}, "
          f"max {errs.max():.2e}; GPU states {np.unique(st, return_counts=True)}; "
          f"states of the worst: {st[np.argsort(errs)[-5:]]}")
    assert np.isin(st, fitspots.CONVERGED_STATES).mean() >= 0.999
    assert np.mean(errs <= 1e-4) >= 0.999
    assert np.median(errs) <= 1e-5


def test_backward_without_chi2_upstream_matches_oracle():
    """The gradient of (x0, y0, sigma, alpha, beta) alone (no upstream for the normalised
    chi^2, the second pixel pass then reads no pixels), against the oracle's FP64 backward
    with a zero chi^2 upstream, on 1,024 iso16 spots and on uint16 ell32 spots."""
    import oracle
    for name, n in (("iso16", 1024), ("ell32", 400)):
        b = synth.make_workload(name, n)
        g = b.to(DEV)
        out = fitspots.fit_batch(g, **TIGHT)
        gp, ga, gb, _ = _upstream(n, 17)
        grad = fitspots.backward(g.images, g.offsets, g.dims, g.model, out, gp, ga, gb, None)
        torch.cuda.synchronize()
        grad = grad.cpu().numpy()
        d = b.numpy()
        img = synth.as_numpy_images(b)
        ref = oracle.fit_spots(img, d["offsets"], d["dims"], d["init"], d["model"], max_iter=300,
                               min_delta=0.0, min_step=1e-13)
        from tests.parity import determined
        det = determined(b, ref) if name == "ell32" else np.ones(n, bool)
        errs = []
        for s in np.nonzero(det)[0]:
            off = int(d["offsets"][s])
            W, H = int(d["dims"][s, 0]), int(d["dims"][s, 1])
            gs = img[off:off + W * H].astype(np.float64)
            up = np.concatenate([gp[s].numpy(), [ga[s], gb[s], 0.0]]).astype(np.float64)
            ro = oracle.backward(int(d["model"][s]), W, H, gs, ref["params"][s], ref["alpha"][s],
                                 ref["beta"][s], up)
            assert ro is not None
            errs.append(np.linalg.norm(grad[off:off + W * H] - ro) / np.linalg.norm(ro))
        errs = np.array(errs)
        print(f"{name} backward without chi2 upstream: {len(errs)} spots, median "
              f"{np.median(errs):.2e}, max {errs.max():.2e}")
        assert np.mean(errs <= 1e-4) >= 0.999 and np.median(errs) <= 1e-5


def test_backward_matches_finite_differences_1024_iso16():
    """The backward workload's stated check: the GPU pixel gradient (forward and backward
    kernels, tight FP32 stop) of the first 1,024 16x16 isotropic spots against central
    finite differences of polished FP64 oracle refits over every pixel, per spot
    ||grad - fd|| / ||fd|| <= 1e-4."""
    from tests.backward_fd import fd_vjp, polished, rel_err
    n = 1024
    b = synth.make_workload("iso16", n)
    g = b.to(DEV)
    out = fitspots.fit_batch(g, **TIGHT)
    gp, ga, gb, gc = _upstream(n, 13)
    grad = fitspots.backward(g.images, g.offsets, g.dims, g.model, out, gp, ga, gb, gc)
    torch.cuda.synchronize()
    grad = grad.cpu().numpy().astype(np.float64).reshape(n, 256)
    d = b.numpy()
    img = synth.as_numpy_images(b).astype(np.float64)
    ref = polished(img, d["offsets"], d["dims"], d["init"], d["model"])
    up = torch.cat([gp, ga[:, None], gb[:, None], gc[:, None]], 1).double().numpy()
    fd, _ = fd_vjp(img, d["offsets"], d["dims"], d["model"], ref["params"], up)
    e = rel_err(grad, fd)
    st = out["state"].cpu().numpy()
    print(f"iso16 backward vs FD (1,024 spots): median {np.median(e):.2e}, "
          f"p99 {np.percentile(e, 99):.2e}, max {e.max():.2e}")
    assert np.isin(st, fitspots.CONVERGED_STATES).all()
    assert e.max() <= 1e-4


def _oracle_errors(b, out, up):
    """Per-spot relative error of the GPU pixel gradient against the oracle's FP64 backward
    at the oracle's own tight fit; also the determined mask of those fits."""
    import oracle
    from tests.parity import determined
    gp, ga, gb, gc = up
    grad = fitspots.backward(b.images.to(DEV), b.offsets.to(DEV), b.dims.to(DEV),
                             b.model.to(DEV), out, gp, ga, gb, gc)
    torch.cuda.synchronize()
    grad = grad.cpu().numpy()
    d = b.numpy()
    img = synth.as_numpy_images(b)
    ref = oracle.fit_spots(img, d["offsets"], d["dims"], d["init"], d["model"], max_iter=300,
                           min_delta=0.0, min_step=1e-13)
    det = determined(b, ref)
    errs = np.full(b.n, np.inf)
    for s in np.nonzero(det)[0]:
        off = int(d["offsets"][s])
        W, H = int(d["dims"][s, 0]), int(d["dims"][s, 1])
        gs = img[off:off + W * H].astype(np.float64)
        u = np.concatenate([gp[s].numpy(), [ga[s], gb[s], gc[s]]]).astype(np.float64)
        ro = oracle.backward(int(d["model"][s]), W, H, gs, ref["params"][s], ref["alpha"][s],
                             ref["beta"][s], u)
        if ro is not None:
            errs[s] = np.linalg.norm(grad[off:off + W * H] - ro) / np.linalg.norm(ro)
    return errs, det


def test_backward_full_size_iso16_sampled():
    """All 262,144 iso16 spots, forward and backward in the launches the benchmark times;
    the pixel gradients of a random sample of 512 spots against the oracle's FP64 backward
    at its own polished fit."""
    import oracle
    b = synth.make_workload("iso16", None, device=DEV)
    assert b.n == 262_144
    fo = fitspots.fit_batch(b, **TIGHT)
    gen = torch.Generator(device=DEV).manual_seed(7)
    up = [torch.randn(b.n, 4, generator=gen, device=DEV)] + \
         [torch.randn(b.n, generator=gen, device=DEV) for _ in range(3)]
    grad = fitspots.backward(b.images, b.offsets, b.dims, b.model, fo, *up)
    torch.cuda.synchronize()
    rng = np.random.default_rng(11)
    idx = np.sort(rng.choice(b.n, 512, replace=False))
    sub = b.subset(idx).to("cpu")
    d = sub.numpy()
    img = synth.as_numpy_images(sub)
    ref = oracle.fit_spots(img, d["offsets"], d["dims"], d["init"], d["model"], max_iter=300,
                           min_delta=0.0, min_step=1e-13)
    offs = b.offsets.cpu().numpy()
    grad = grad.cpu().numpy()
    st = fo["state"].cpu().numpy()
    ups = [u.cpu().numpy() for u in up]
    errs = []
    for j, s in enumerate(idx):
        o = int(offs[s])
        g_gpu = grad[o:o + 256].astype(np.float64)
        gs = img[int(d["offsets"][j]):int(d["offsets"][j]) + 256].astype(np.float64)
        u = np.concatenate([ups[0][s], [ups[1][s], ups[2][s], ups[3][s]]]).astype(np.float64)
        ro = oracle.backward(0, 16, 16, gs, ref["params"][j], ref["alpha"][j], ref["beta"][j], u)
        assert ro is not None
        errs.append(np.linalg.norm(g_gpu - ro) / np.linalg.norm(ro))
    errs = np.array(errs)
    print(f"iso16 full-size backward sample: median {np.median(errs):.2e}, "
          f"p99 {np.percentile(errs, 99):.2e}, max {errs.max():.2e}")
    assert np.isin(st, fitspots.CONVERGED_STATES).mean() >= 0.999
    assert np.mean(errs <= 1e-4) >= 0.99
    assert np.median(errs) <= 1e-5


def test_backward_matches_oracle_mixed_sizes():
    """Sizes 5..32 per side (row steps that do and do not divide the warp, odd heights,
    partial row groups) and both models: same per-spot bar as the 16x16 workload on the
    determined spots."""
    n = 1500
    b = synth.make_workload("mixed", n)
    out = fitspots.fit_batch(b.to(DEV), **TIGHT)
    errs, det = _oracle_errors(b, out, _upstream(n, 5))
    e = errs[det]
    print(f"mixed backward: {det.sum()} determined of {n}; median rel err {np.median(e):.2e}, "
          f"p99.9 {np.percentile(e, 99.9):.2e}, max {e.max():.2e}")
    assert det.sum() >= n // 3
    assert np.mean(e <= 1e-4) >= 0.999
    assert np.median(e) <= 1e-5


def test_backward_matches_oracle_uint16_ell32():
    """uint16 pixels, elliptic model, 32x32 (one row per step)."""
    n = 400
    b = synth.make_workload("ell32", n)
    out = fitspots.fit_batch(b.to(DEV), **TIGHT)
    errs, det = _oracle_errors(b, out, _upstream(n, 6))
    e = errs[det]
    print(f"ell32 backward: {det.sum()} determined of {n}; median rel err {np.median(e):.2e}, "
          f"p99.9 {np.percentile(e, 99.9):.2e}, max {e.max():.2e}")
    assert det.sum() >= 50
    assert np.mean(e <= 1e-4) >= 0.999
    assert np.median(e) <= 1e-5


def test_backward_identities_both_models():
    """Shift and scale invariance of the fit fix sum_i dq/dg_i and sum_i g_i dq/dg_i. They hold
    at the exact minimum, so the backward kernel is evaluated at the oracle's polished FP64
    fit of each spot (the forward kernel's FP32 stop can lie off the minimum by more than the
    identities' tolerance); this checks the backward alone."""
    import oracle
    for name in ("iso16", "ell32"):
        b = synth.make_workload(name, 256)   # ell32 stays uint16
        d = b.numpy()
        ref = oracle.fit_spots(synth.as_numpy_images(b), d["offsets"], d["dims"], d["init"],
                               d["model"], max_iter=300, min_delta=0.0, min_step=1e-13)
        b = b.to(DEV)
        out = {k: torch.as_tensor(ref[k], device=DEV).to(torch.float32)
               for k in ("params", "alpha", "beta", "chi2")}
        out["state"] = torch.as_tensor(ref["state"], device=DEV)
        conv = torch.isin(out["state"], torch.tensor(fitspots.CONVERGED_STATES, device=DEV,
                                                     dtype=torch.int32))
        # spots whose amplitude stands above the residual noise: a well-defined minimum
        conv &= out["alpha"] > 3.0 * torch.sqrt(out["chi2"].clamp_min(0.0))
        assert conv.sum() >= 100
        N = int(b.dims[0, 0] * b.dims[0, 1])
        gimg = b.images.to(torch.float32).view(b.n, N).double()
        for k, name_k in enumerate(("x0", "y0", "sx", "sy", "alpha", "beta", "chi2")):
            if name == "iso16" and k == 3:
                continue
            gp = torch.zeros(b.n, 4, device=DEV)
            ga = torch.zeros(b.n, device=DEV)
            gb = torch.zeros(b.n, device=DEV)
            gc = torch.zeros(b.n, device=DEV)
            if k < 4:
                gp[:, k] = 1.0
            elif k == 4:
                ga[:] = 1.0
            elif k == 5:
                gb[:] = 1.0
            else:
                gc[:] = 1.0
            grad = fitspots.backward(b.images, b.offsets, b.dims, b.model, out, gp, ga, gb, gc)
            G = grad.view(b.n, N).double()
            s1 = G.sum(1)[conv]
            sg = (G * gimg).sum(1)[conv]
            scale = G.abs().sum(1)[conv] + 1e-30
            sgscale = (G * gimg).abs().sum(1)[conv] + 1e-30
            if k < 4:
                exp1, expg = torch.zeros_like(s1), torch.zeros_like(sg)
            elif k == 4:
                exp1, expg = torch.zeros_like(s1), out["alpha"].double()[conv]
            elif k == 5:
                exp1, expg = torch.ones_like(s1), out["beta"].double()[conv]
            else:
                exp1, expg = torch.zeros_like(s1), 2 * out["chi2"].double()[conv]
            e1 = ((s1 - exp1).abs() / scale).max().item()
            eg = ((sg - expg).abs() / sgscale).max().item()
            print(f"{name} {name_k}: identity errors {e1:.1e} {eg:.1e}")
            assert e1 < 2e-4 and eg < 2e-4, (name, name_k, e1, eg)


def test_autograd_function_and_zero_paths():
    b = synth.make_workload("iso15", 200, device=DEV)
    images = b.images.clone().requires_grad_(True)
    init = b.init.clone().requires_grad_(True)
    params, alpha, beta, chi2, state, iters = fitspots.fit_differentiable(
        images, init, b.offsets, b.dims, b.model)
    w = torch.randn(params.shape, device=DEV)
    loss = (params * w).sum() + 0.5 * alpha.sum() - beta.sum() + chi2.sum()
    gi, gin = torch.autograd.grad(loss, (images, init))
    direct = fitspots.backward(b.images, b.offsets, b.dims, b.model,
                               dict(params=params.detach(), alpha=alpha.detach(),
                                    beta=beta.detach(), state=state),
                               w, torch.full_like(alpha, 0.5), torch.full_like(beta, -1.0),
                               torch.ones_like(chi2))
    assert torch.equal(gi, direct.view(gi.shape))
    assert torch.count_nonzero(gin) == 0
    # a spot stopped by the iteration budget is not at a minimum: zero gradient
    out = fitspots.fit_batch(b, max_iter=1)
    grad = fitspots.backward(b.images, b.offsets, b.dims, b.model, out,
                             torch.ones(b.n, 4, device=DEV))
    G = grad.view(b.n, -1)
    not_conv = out["state"] == 0
    assert not_conv.any()
    assert torch.count_nonzero(G[not_conv]) == 0
