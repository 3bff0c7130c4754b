"""pt_deposit_noalloc: the deposition for callers that cannot allocate device
memory (a solver whose device memory belongs to its own pool, a time loop that
must not allocate).  Called through the C ABI and checked against pt_deposit
on two calls in a row; sizes beyond its fixed scratch are refused.

This file is collected last on purpose, so that a run stopping at the first
failure has already run every other test."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2211_05458_gb300 import pt
from paper_2211_05458_gb300 import workloads as W
from tests import helpers as H

pytestmark = pytest.mark.gpu


def _noalloc(ctx, parts, mode, S):
    p = parts.struct()
    rc = pt.lib().pt_deposit_noalloc(ctx.h, ctypes.byref(p), int(mode),
                                     ctypes.c_void_p(S.data_ptr()))
    return rc


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("mode", [pt.DEPOSIT_SEGMENTED, pt.DEPOSIT_ATOMIC])
def test_noalloc_deposit_matches_pt_deposit_twice(precision, mode):
    wl = W.curved_channel((6, 5, 4), 2, 7, P=3000, nsteps=1, seed=4, mass_loading=0.3)
    rng = np.random.default_rng(4)
    wl.v = wl.v + torch.as_tensor(rng.normal(size=(3000, 3)) * 0.3)
    ctx = H.gpu_context(wl, precision)
    parts = H.gpu_particles(wl, ctx)
    ref = ctx.deposit(parts, mode).clone()
    scale = float(ref.abs().max())
    assert scale > 0
    for _ in range(2):
        S = torch.full_like(ref, 7.0)  # stale contents must be overwritten
        assert _noalloc(ctx, parts, mode, S) == pt.PT_OK
        torch.cuda.synchronize()
        assert float((S - ref).abs().max()) <= 1e-5 * scale


def test_noalloc_deposit_refuses_sizes_beyond_its_scratch():
    wl = W.curved_channel((3, 3, 3), 2, 3, P=10, nsteps=1)
    ctx = H.gpu_context(wl, "fp32")
    n = (1 << 20) + 1
    big = pt.ParticleSet(torch.zeros((3, n), dtype=torch.float64, device="cuda"),
                         torch.zeros((3, n), dtype=torch.float32, device="cuda"),
                         torch.ones(n, dtype=torch.float32, device="cuda"),
                         torch.zeros(n, dtype=torch.int32, device="cuda"))
    S = torch.zeros((wl.mesh.nelem, 4, 64), dtype=torch.float32, device="cuda")
    assert _noalloc(ctx, big, pt.DEPOSIT_SEGMENTED, S) == pt.PT_ERR_ARG
    assert b"1048576" in pt.lib().pt_last_error(ctx.h)
