"""Calls on a stream that is not the current one, with workspace and outputs allocated by
the binding: their memory belongs to the launch stream, so allocations the current stream
makes right after the call (here filled with zeros, which only corrupt results, never
address anything) cannot land on buffers the kernels still use."""
import pytest
import torch

from paper_2106_02045_gb300 import fitspots, synth

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _scribble():
    return [torch.zeros(1 << 22, dtype=torch.int32, device=DEV) for _ in range(16)]


def _same(a: torch.Tensor, b: torch.Tensor) -> bool:
    return torch.equal(torch.nan_to_num(a), torch.nan_to_num(b))


def test_side_stream_calls_own_their_temporaries():
    b = synth.make_workload("mixed", 40_000, device=DEV)
    u = synth.make_workload("ell32", 40_000, device=DEV)
    ref = fitspots.fit_batch(b)
    ref_u = fitspots.fit_uniform(u.images, 32, 32, synth.MODEL_ELLIPTIC, u.init)
    up = [torch.randn(b.n, 4, device=DEV), torch.randn(b.n, device=DEV)]
    ref_g = fitspots.backward(b.images, b.offsets, b.dims, b.model, ref, *up)
    ref_s = fitspots.start_values(b.images, b.offsets, b.dims)
    torch.cuda.synchronize()

    side = torch.cuda.Stream(DEV)
    side.wait_stream(torch.cuda.current_stream(DEV))
    out = fitspots.fit_batch(b, stream=side)
    junk = _scribble()
    out_u = fitspots.fit_uniform(u.images, 32, 32, synth.MODEL_ELLIPTIC, u.init, stream=side)
    junk += _scribble()
    side.synchronize()
    # upstream gradients given as float64 host tensors: converted on the launch stream
    g = fitspots.backward(b.images, b.offsets, b.dims, b.model, out,
                          up[0].double().cpu(), up[1].double().cpu(), stream=side)
    junk += _scribble()
    s0 = fitspots.start_values(b.images, b.offsets, b.dims, stream=side)
    junk += _scribble()
    torch.cuda.synchronize()
    del junk
    for k in ref:
        assert _same(ref[k], out[k]), k
        assert _same(ref_u[k], out_u[k]), k
    assert torch.allclose(ref_g, g, rtol=0, atol=0)
    assert _same(ref_s, s0)


def test_backward_rejects_malformed_inputs():
    b = synth.make_workload("iso15", 64, device=DEV)
    out = fitspots.fit_batch(b)
    with pytest.raises(fitspots.FitSpotsError):
        fitspots.backward(b.images.double(), b.offsets, b.dims, b.model, out)
    with pytest.raises(fitspots.FitSpotsError):
        fitspots.backward(b.images, b.offsets.int(), b.dims, b.model, out)
    with pytest.raises(fitspots.FitSpotsError):
        fitspots.backward(b.images, b.offsets, b.dims, b.model, dict(out, alpha=out["alpha"][:-1]))
    with pytest.raises(fitspots.FitSpotsError):
        fitspots.backward(b.images, b.offsets, b.dims, b.model, out,
                          grad_images=torch.zeros(3, device=DEV))
