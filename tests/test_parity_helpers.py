"""The comparison helpers behind every GPU parity test, checked on the host with known
answers: identical results agree fully, and each kind of disagreement is counted."""
import numpy as np

from paper_2106_02045_gb300 import synth
from tests.parity import XY_TOL, compare, determined, run_oracle


def _fixture():
    b = synth.make_workload("iso15", 300)
    ref = run_oracle(b)
    out = {k: (v.astype(np.float32) if v.dtype == np.float64 else v.copy()) for k, v in ref.items()}
    return b, ref, out


def test_identical_results_agree_fully():
    b, ref, out = _fixture()
    det = determined(b, ref)
    assert det.sum() > 200
    m = compare(out, ref, b.dims.numpy(), det)
    assert m["class_agree"] == m["state_agree"] == 1.0
    assert m["bar_converged"] == m["bar_wp"] == m["class_agree_wp"] == 1.0
    assert m["n_well_posed"] == det.sum()


def test_each_disagreement_is_counted():
    b, ref, out = _fixture()
    det = determined(b, ref)
    dims = b.dims.numpy()
    s = int(np.nonzero(det)[0][0])
    nd = int(det.sum())
    both = np.isin(ref["state"], (1, 2, 3, 4))
    # a centre off by twice the tolerance
    o = {k: v.copy() for k, v in out.items()}
    o["params"][s, 0] += 2 * XY_TOL
    m = compare(o, ref, dims, det)
    assert m["bar_wp"] == (nd - 1) / nd and m["class_agree"] == 1.0
    assert np.isclose(m["max_dxy_wp"], 2 * XY_TOL, rtol=1e-3)
    # a relative error of 2e-4 in alpha, then a NaN width
    for key, idx, val in (("alpha", (s,), out["alpha"][s] * (1 + 2e-4)),
                          ("params", (s, 2), np.nan)):
        o = {k: v.copy() for k, v in out.items()}
        o[key][idx] = val
        assert compare(o, ref, dims, det)["bar_wp"] == (nd - 1) / nd
    # a converged spot reported as not converged: class disagreement, out of the bar
    o = {k: v.copy() for k, v in out.items()}
    o["state"][s] = 0
    m = compare(o, ref, dims, det)
    assert m["class_agree"] == 1 - 1 / len(det) and m["class_agree_wp"] == 1 - 1 / nd
    assert m["bar_wp"] == 1.0 and m["bar_converged"] == 1.0 and both.sum() > 0
    # a different converged code is not a class disagreement
    o = {k: v.copy() for k, v in out.items()}
    o["state"][s] = 2 if ref["state"][s] != 2 else 1
    m = compare(o, ref, dims, det)
    assert m["class_agree"] == 1.0 and m["state_agree"] == 1 - 1 / len(det)
