"""pt_deposit_noalloc: the deposition for callers that cannot allocate device
memory (a solver whose device memory belongs to its own pool, a time loop that
must not allocate).  Called through the C ABI and checked against pt_deposit
on two calls in a row and against the FP64 oracle; sizes beyond its fixed
scratch are refused; an empty particle set gives a zero source.

This file is collected last on purpose, so that a run stopping at the first
failure has already run every other test."""
import ctypes

import numpy as np

import oracle
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
        if mode == pt.DEPOSIT_SEGMENTED and precision == "fp32":
            # same factors and summation order as the two-pass pt_deposit
            assert torch.equal(S, ref)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("mode", [pt.DEPOSIT_SEGMENTED, pt.DEPOSIT_ATOMIC,
                                  pt.DEPOSIT_SEGMENTED | pt.DEPOSIT_NEAREST])
def test_noalloc_deposit_matches_oracle(precision, mode):
    wl = W.curved_channel((6, 5, 4), 2, 7, P=3000, nsteps=1, seed=6, mass_loading=0.3)
    rng = np.random.default_rng(6)
    wl.v = wl.v + torch.as_tensor(rng.normal(size=(3000, 3)) * 0.3)
    ctx = H.gpu_context(wl, precision)
    parts = H.gpu_particles(wl, ctx)
    n3 = (wl.N + 1) ** 3
    S = torch.zeros((wl.mesh.nelem, 4, n3), dtype=torch.float32, device="cuda")
    assert _noalloc(ctx, parts, mode, S) == pt.PT_OK
    torch.cuda.synchronize()
    orc = H.make_oracle(wl)
    args = (H.oracle_params(wl), H.np64(wl.x), H.np64(wl.v), H.np64(wl.d),
            H.np64(wl.elem).astype(np.int32))
    if mode & pt.DEPOSIT_NEAREST:
        # particles within 1e-8 of a midpoint between two nodes may go to either
        xn = oracle.nodes(wl.node_type, wl.N + 1)
        mids = 0.5 * (xn[1:] + xn[:-1])
        x, el = args[1], args[4]
        for i in range(len(el)):
            ok, xi, _ = orc.newton(int(el[i]), x[i])
            assert not ok or np.min(np.abs(xi[:, None] - mids[None, :])) >= 1e-8
        So = orc.deposit_nearest(*args)
    else:
        So = orc.deposit(*args)
    Sg = S.double().cpu().numpy()
    assert np.max(np.abs(Sg - So)) <= 1e-5 * np.abs(So).max()
    es, eo = Sg.sum(axis=2), So.sum(axis=2)
    assert np.max(np.abs(es - eo) / np.abs(eo).max(axis=0, keepdims=True)) < 1e-5


@pytest.mark.parametrize("mode", [pt.DEPOSIT_SEGMENTED, pt.DEPOSIT_ATOMIC])
def test_noalloc_deposit_of_no_particles_is_zero(mode):
    wl = W.curved_channel((3, 3, 3), 2, 3, P=10, nsteps=1)
    ctx = H.gpu_context(wl, "fp32")
    empty = pt.ParticleSet(torch.zeros((3, 0), dtype=torch.float64, device="cuda"),
                           torch.zeros((3, 0), dtype=torch.float32, device="cuda"),
                           torch.zeros(0, dtype=torch.float32, device="cuda"),
                           torch.zeros(0, dtype=torch.int32, device="cuda"))
    S = torch.full((wl.mesh.nelem, 4, 64), 3.0, dtype=torch.float32, device="cuda")
    assert _noalloc(ctx, empty, mode, S) == pt.PT_OK
    torch.cuda.synchronize()
    assert float(S.abs().max()) == 0.0


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
    # more elements than the scratch's element counters: 51^3 = 132651 > 131072
    wl = W.tgv_box(51, 1, P=100, nsteps=1, seed=1, precision="fp32")
    ctx = H.gpu_context(wl, "fp32")
    parts = H.gpu_particles(wl, ctx)
    S = torch.zeros((wl.mesh.nelem, 4, 8), dtype=torch.float32, device="cuda")
    for mode in (pt.DEPOSIT_SEGMENTED, pt.DEPOSIT_ATOMIC):
        assert _noalloc(ctx, parts, mode, S) == pt.PT_ERR_ARG
        assert b"131072" in pt.lib().pt_last_error(ctx.h)
