"""Start values on the device (``fit_spots_start``) against the oracle's rules: the same
integer decisions (pixels above the one-sigma level, the 3x3 neighbourhood argmax) on
integer-valued pixels, centroids to FP32 rounding."""
import numpy as np
import pytest
import torch

from oracle import start as st
from paper_2106_02045_gb300 import fitspots, synth

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _compare(b, rule):
    g = b.to(DEV)
    out = fitspots.start_values(g.images, g.offsets, g.dims, rule).cpu().numpy()
    ref = st.start_values(synth.as_numpy_images(b), b.offsets.numpy(), b.dims.numpy(), rule)
    assert np.isfinite(out).all()
    assert np.allclose(out[:, 2:], ref[:, 2:], rtol=1e-6, atol=0)      # same M
    if rule == st.PAPER:
        assert np.array_equal(out[:, :2], ref[:, :2])
    else:
        assert np.abs(out[:, :2] - ref[:, :2]).max() <= 1e-4


@pytest.mark.parametrize("rule", [st.CENTROID, st.PAPER])
@pytest.mark.parametrize("name,n", [("iso15", 3000), ("ell32", 1000), ("mixed", 3000)])
def test_start_values_match_oracle(name, n, rule):
    _compare(synth.make_workload(name, n), rule)


def test_start_values_paper_protocol_and_degenerate_rois():
    _compare(synth.make_paper(2000, 9, 1000.0, 100.0, seed=3), st.PAPER)
    imgs = torch.full((3 * 64,), 7.0)
    imgs[64 + 9] = 900.0
    offs = torch.tensor([0, 64, 128], dtype=torch.int64)
    dims = torch.tensor([[8, 8], [8, 8], [40, 1]], dtype=torch.int32)
    out = fitspots.start_values(imgs.to(DEV), offs.to(DEV), dims.to(DEV)).cpu().numpy()
    assert np.allclose(out[0], [3.5, 3.5, np.sqrt(1 / np.pi), np.sqrt(1 / np.pi)])   # flat
    assert np.allclose(out[1, :2], [1.0, 1.0])                                       # one pixel
    assert np.isnan(out[2]).all()                                                    # W > 32


def test_device_start_values_feed_the_fit():
    """Fits from device start values agree with fits from the host rule's start values."""
    b = synth.make_workload("ell32", 4000, device=DEV)
    init = fitspots.start_values(b.images, b.offsets, b.dims)
    a = fitspots.fit_uniform(b.images, 32, 32, 1, b.init)
    c = fitspots.fit_uniform(b.images, 32, 32, 1, init)
    conv = torch.isin(a["state"], torch.tensor(fitspots.CONVERGED_STATES, device=DEV))
    same = (a["params"] - c["params"]).abs().max(dim=1).values < 1e-3
    assert float((same | ~conv).float().mean()) >= 0.99
