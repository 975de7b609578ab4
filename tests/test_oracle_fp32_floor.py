"""How well can any fit that evaluates the model in 32-bit floats agree with the FP64
oracle? The oracle's third build rounds the profile f_i and its derivatives (Eq. 10, 11) to
the nearest FP32 value and keeps everything after them in FP64. Compared with the FP64
build on the same spots, by the GPU parity tests' own metrics:

* on determined spots (well-posed, centre standard error <= 0.1 px, width standard error
  <= 10 %) the two builds agree completely;
* on all spots the share of converged fits inside the 1e-3 px / 1e-4 relative bar stays
  below 0.999: on flat chi^2 surfaces (widths near the ROI size, dim or negative
  amplitudes) the projected Jacobian of the implicit-amplitude model is a small difference
  of large terms, and one rounding of the model values moves the min_delta stop point
  beyond the bar.

So the all-spot bar of 0.999 is out of reach for an implementation whose model values are
FP32 (the paper's own, Sec. "Implementation", included); these measured figures are the
floor beside which the GPU parity tests set their all-spot bars. (The oracle is also robust
to the other perturbations tried: start values moved by 16 FP32 ulps, or the normal
equations rounded to FP32, keep 99.94 % or more inside the bar.)
"""
import numpy as np
import pytest

from paper_2106_02045_gb300 import synth
from tests.parity import compare, determined


@pytest.mark.parametrize("name", ["ell32", "mixed"])
def test_fp32_model_values_alone_move_flat_fits_beyond_the_bar(oracle_mod, name):
    b = synth.make_workload(name, 20000)
    d = b.numpy()
    img = synth.as_numpy_images(b)
    ref = oracle_mod.fit_spots(img, d["offsets"], d["dims"], d["init"], d["model"])
    r32 = oracle_mod.fit_spots(img, d["offsets"], d["dims"], d["init"], d["model"],
                               fp32_profile=True)
    det = determined(b, ref)
    m = compare(r32, ref, d["dims"], det)
    print(f"{name}: FP32 model values vs FP64: class {m['class_agree']:.5f}, converged within "
          f"the bar {m['bar_converged']:.5f}; determined ({m['n_well_posed']}) class "
          f"{m['class_agree_wp']:.5f}, bar {m['bar_wp']:.5f}")
    assert m["class_agree_wp"] == 1.0 and m["bar_wp"] >= 0.999
    assert m["class_agree"] >= 0.999
    assert m["bar_converged"] < 0.999


def test_fits_do_not_move_with_fp32_ulp_changes_of_the_start(oracle_mod):
    """The contrast: moving every start value by 16 FP32 ulps (random directions) leaves all
    converged ell32 fits inside the bar, so the end points are not fragile to the path as
    such; what moves them is the precision of the model values (the test above)."""
    b = synth.make_workload("ell32", 20000)
    d = b.numpy()
    img = synth.as_numpy_images(b)
    ref = oracle_mod.fit_spots(img, d["offsets"], d["dims"], d["init"], d["model"])
    rng = np.random.default_rng(1)
    init = d["init"].copy()
    for _ in range(16):
        init = np.nextafter(init, np.where(rng.random(init.shape) < 0.5, -np.inf, np.inf)
                            ).astype(np.float32)
    alt = oracle_mod.fit_spots(img, d["offsets"], d["dims"], init, d["model"])
    m = compare(alt, ref, d["dims"], determined(b, ref))
    print(f"ell32, start values moved by 16 ulps: class {m['class_agree']:.5f}, converged "
          f"within the bar {m['bar_converged']:.5f}")
    assert m["class_agree"] >= 0.9999 and m["bar_converged"] >= 0.9999
