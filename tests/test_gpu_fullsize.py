"""Full-size workloads on the GPU, checked on sampled particles that the oracle
recomputes one by one from the same initial state (particles are independent
during a push, so a sample is an exact sub-problem).  Launch configuration as
in bench.py: element re-binning every 10 steps, 128-thread blocks."""
import math

import numpy as np
import pytest
import torch

from paper_2211_05458_gb300 import pt
from paper_2211_05458_gb300 import workloads as W
from tests import helpers as H

pytestmark = pytest.mark.gpu

FP32_BAND = dict(band_ref=2e-4)


def _sample(n, k, seed=0):
    return np.sort(np.random.default_rng(seed).choice(n, size=k, replace=False))


def _check_sample(wl, parts, idx, tol, band_ref, band_x, nsteps):
    g_all = H.gpu_result(parts)
    g = {k: v[idx] for k, v in g_all.items()}
    o = H.run_oracle(wl, idx, nsteps=nsteps, band_ref=band_ref, band_x=band_x)
    return H.compare(g, o, tol)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_curved_channel_32cubed_1e6_particles_200_steps(precision):
    wl = W.curved_channel((32, 32, 32), 2, 5, P=1_000_000, nsteps=200, device="cuda")
    h = 2.0 / 32
    band = (1e-10, 1e-10) if precision == "fp64" else (2e-4, 1e-4 * h)
    ctx = H.gpu_context(wl, precision, rebin_every=10, band_ref=band[0], band_x=band[1])
    parts = H.gpu_particles(wl, ctx)
    st = ctx.push(parts, 200, wl.dt)
    assert st["newton_fail"] == 0 and st["lost"] == 0 and st["cross_cap"] == 0
    assert st["particle_steps"] == 200 * 1_000_000
    wl.U, wl.x, wl.v, wl.d, wl.elem = wl.U.cpu(), wl.x.cpu(), wl.v.cpu(), wl.d.cpu(), wl.elem.cpu()
    idx = _sample(1_000_000, 300)
    _check_sample(wl, parts, idx, 1e-12 if precision == "fp64" else 2e-5, *band, 200)


def test_learned_channel_64cubed_1e7_particles():
    wl = W.curved_channel((64, 64, 64), 3, 5, P=10_000_000, nsteps=20, device="cuda",
                          precision="fp32")
    h = 2.0 / 64
    ctx = H.gpu_context(wl, "fp32", rebin_every=10, band_ref=2e-4, band_x=1e-4 * h)
    inp, tgt = ctx.mlp_make_pairs(2_000_000, seed=1000)
    losses = ctx.mlp_train(inp, tgt, epochs=20, batch=4096, lr=1e-3, seed=0)
    assert losses[-1] < losses[0]
    del inp, tgt
    ctx.set_config(guess=pt.GUESS_MLP)
    parts = H.gpu_particles(wl, ctx)
    for _ in range(2):
        st = ctx.push(parts, 10, wl.dt)
    assert st["newton_fail"] == 0 and st["lost"] == 0
    wl.U, wl.x, wl.v, wl.d, wl.elem = wl.U.cpu(), wl.x.cpu(), wl.v.cpu(), wl.d.cpu(), wl.elem.cpu()
    idx = _sample(10_000_000, 150, seed=1)
    _check_sample(wl, parts, idx, 2e-5, 2e-4, 1e-4 * h, 20)


def test_two_way_channel_128x64x64_2e7_particles_deposit_sampled_elements():
    dims = (128, 64, 64)
    wl = W.curved_channel(dims, 2, 7, P=20_000_000, nsteps=1, device="cuda", mass_loading=0.3)
    rng = np.random.default_rng(5)
    # particles released at the fluid velocity carry no drag: give them a slip
    # velocity so that every source is well above the FP32 rounding of u - v
    gen = torch.Generator(device="cuda").manual_seed(5)
    wl.v = wl.v + 0.3 * torch.randn(wl.v.shape, generator=gen, device="cuda", dtype=wl.v.dtype)
    ctx = H.gpu_context(wl, "fp32")
    parts = H.gpu_particles(wl, ctx)
    S_seg = ctx.deposit(parts, pt.DEPOSIT_SEGMENTED).clone()
    S_at = ctx.deposit(parts, pt.DEPOSIT_ATOMIC)
    # total momentum source equals minus the total drag force: both modes agree
    tot_seg = S_seg[:, :3].double().sum(dim=(0, 2))
    tot_at = S_at[:, :3].double().sum(dim=(0, 2))
    assert torch.all((tot_seg - tot_at).abs() <= 1e-6 * S_seg[:, :3].double().abs().sum(dim=(0, 2)))
    # oracle on the particles of sampled elements
    el = wl.elem.cpu().numpy()
    sel = rng.choice(wl.mesh.nelem, size=40, replace=False)
    mask = np.isin(el, sel)
    idx = np.flatnonzero(mask)
    wl.U = wl.U.cpu()
    orc = H.make_oracle(wl)
    So = orc.deposit(H.oracle_params(wl), H.np64(wl.x.cpu())[idx], H.np64(wl.v.cpu())[idx],
                     H.np64(wl.d.cpu())[idx], el[idx].astype(np.int32))
    Sg = S_seg.double().cpu().numpy()
    for e in sel:
        es, eo = Sg[e].sum(axis=1), So[e].sum(axis=1)
        assert np.all(np.abs(es - eo) <= 1e-5 * np.abs(eo).max() + 1e-30)
        assert np.max(np.abs(Sg[e] - So[e])) <= 1e-5 * np.abs(So[e]).max() + 1e-30


def test_two_way_channel_push_sampled():
    dims = (128, 64, 64)
    wl = W.curved_channel(dims, 2, 7, P=20_000_000, nsteps=10, device="cuda", mass_loading=0.3)
    h = 2.0 / 64
    ctx = H.gpu_context(wl, "fp32", rebin_every=10, band_ref=2e-4, band_x=1e-4 * h)
    parts = H.gpu_particles(wl, ctx)
    st = ctx.push(parts, 10, wl.dt)
    assert st["particle_steps"] == 10 * 20_000_000
    wl.U, wl.x, wl.v, wl.d, wl.elem = wl.U.cpu(), wl.x.cpu(), wl.v.cpu(), wl.d.cpu(), wl.elem.cpu()
    idx = _sample(20_000_000, 100, seed=3)
    _check_sample(wl, parts, idx, 2e-5, 2e-4, 1e-4 * h, 10)


def test_batched_boxes_128_sampled():
    boxes = W.batched_boxes(nbox=128, seed=1, nsteps=50, device="cuda")
    ctxs = [H.gpu_context(wl, "fp32") for wl in boxes]
    parts = [H.gpu_particles(wl, c) for wl, c in zip(boxes, ctxs)]
    for _ in range(2):  # tuning call, then graph replay: 100 steps in all
        st = pt.push_batch(ctxs, parts, 50, 1e-3)
    tot = sum(p.n for p in parts)
    assert sum(s["particle_steps"] for s in st) == 50 * tot
    assert all(s["newton_fail"] == 0 and s["lost"] == 0 for s in st)
    rng = np.random.default_rng(11)
    for b in rng.choice(128, size=6, replace=False):
        wl = boxes[b]
        wl.U, wl.x, wl.v, wl.d, wl.elem = wl.U.cpu(), wl.x.cpu(), wl.v.cpu(), wl.d.cpu(), wl.elem.cpu()
        n = wl.x.shape[0]
        idx = _sample(n, min(n, 40), seed=int(b))
        h = 1.0 / wl.mesh.dims[0]
        _check_sample(wl, parts[b], idx, 2e-5, 2e-4, 1e-4 * h, 100)
