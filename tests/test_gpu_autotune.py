"""Configuration autotuner: picks a usable configuration per class (the fastest it timed),
caches and reloads the choice, and leaves the fits of fit_spots (whose single launch runs the
generic kernel whatever the table says) at the parity bar against the FP64 oracle. The tuned
table itself drives fit_spots_per_class and fit_spots_uniform; the bench times it there."""
import numpy as np
import pytest
import torch

from paper_2106_02045_gb300 import autotune, fitspots, synth
from parity import compare, determined, run_oracle

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def test_autotune_choices_and_parity(tmp_path):
    classes = [0, 5, 10, 15]
    cache = tmp_path / "tune.json"
    res = autotune.autotune(classes=classes, n=1024, reps=1, device=DEV, cache=cache)
    try:
        for c in classes:
            assert fitspots.config_fits(c, res[c]["config"])
            assert fitspots.get_config(c) == res[c]["config"]
            assert res[c]["ms"] == min(res[c]["tried"].values())
        autotune.defaults()
        assert autotune.load(cache, device=DEV) == {c: res[c]["config"] for c in classes}
        # parity of a mixed batch through fit_spots with the tuned table in place
        b = synth.make_workload("mixed", 2000)
        out = fitspots.fit_batch(b.to(DEV))
        torch.cuda.synchronize()
        ref = run_oracle(b)
        rep = compare({k: v.cpu().numpy() for k, v in out.items()}, ref, b.dims.numpy(),
                      determined(b, ref))
        print("autotuned mixed:", rep)
        assert rep["class_agree_wp"] >= 0.999 and rep["bar_wp"] >= 0.999
    finally:
        autotune.defaults()
