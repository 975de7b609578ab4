"""fit_spots_noalloc: the entry point for callers that cannot allocate device memory.

It keeps its schedule in an array compiled into the library instead of a workspace the
caller allocates. This test calls it through the C ABI twice in a row, on two different
batches (so the second call starts from the first call's leftovers), and checks each
result against fit_spots with a caller workspace: the same kernels on the same inputs, so
the results must agree bit for bit. The file name sorts last so that a run stopping at the first failure has
run every other test before this one.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")


def _lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2106_02045_gb300 import fitspots
    lib = fitspots.library()
    vp, i, i64, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    lib.fit_spots_noalloc.argtypes = [vp, i, i64, vp, vp, vp, vp, i64, i, d, d, d,
                                      vp, vp, vp, vp, vp, vp, vp, vp]
    lib.fit_spots_noalloc.restype = i
    lib.fit_spots_noalloc_max_spots.argtypes = []
    lib.fit_spots_noalloc_max_spots.restype = i64
    return lib


def _noalloc(lib, b):
    from paper_2106_02045_gb300 import fitspots
    o = fitspots.alloc_outputs(b.n, DEV)
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    rc = lib.fit_spots_noalloc(p(b.images), 1, b.images.numel(), p(b.offsets), p(b.dims),
                               p(b.init), p(b.model), b.n, 20, 0.0, 1e-6, 1e-4,
                               p(o["params"]), p(o["alpha"]), p(o["beta"]), p(o["chi2"]),
                               p(o["state"]), p(o["iters"]), p(o["evals"]),
                               ctypes.c_void_p(torch.cuda.current_stream(DEV).cuda_stream))
    assert rc == 0, rc
    return o


def test_noalloc_matches_workspace_entry_point_on_two_calls():
    from paper_2106_02045_gb300 import fitspots, synth
    lib = _lib()
    assert lib.fit_spots_noalloc_max_spots() == 1 << 20
    batches = [synth.make_workload("mixed", 6000, device=DEV),
               synth.make_mixed(2500, seed=synth.SEED_BASE + 77, device=DEV)]
    for b in batches:
        got = _noalloc(lib, b)
        ref = fitspots.fit_batch(b)
        torch.cuda.synchronize()
        # the same kernels on the same inputs with the same schedule: identical bits
        for k in ref:
            assert torch.equal(got[k].view(torch.int32), ref[k].view(torch.int32)), k


def test_noalloc_rejects_batches_above_its_limit():
    lib = _lib()
    fake = ctypes.c_void_p(0x1000)
    n = lib.fit_spots_noalloc_max_spots() + 1
    rc = lib.fit_spots_noalloc(fake, 1, 10, fake, fake, fake, fake, n, 20, 0.0, 1e-6, 1e-4,
                               fake, fake, fake, fake, fake, fake, None, None)
    assert rc == -2
