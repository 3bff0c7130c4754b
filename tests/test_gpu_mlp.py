"""Learned Newton start: GPU training kernels against the FP64 oracle network
(forward values, loss gradients), features, and what the trained network gains
over the trilinear start at equal 1e-12 convergence of the inverse map."""
import numpy as np
import pytest
import torch

import oracle
from paper_2211_05458_gb300 import pt
from paper_2211_05458_gb300 import workloads as W
from tests import helpers as H

pytestmark = pytest.mark.gpu

NORM_ID = np.concatenate([np.zeros(51), np.ones(51), np.ones(3)]).astype(np.float32)


def _ctx(dims=(8, 8, 8), precision="fp32"):
    wl = W.curved_channel(dims, 3, 4, P=2000, nsteps=10, dt=2e-3)
    return wl, H.gpu_context(wl, precision)


def test_forward_matches_oracle_network():
    wl, ctx = _ctx((3, 3, 3))
    rng = np.random.default_rng(1)
    theta = (rng.normal(size=oracle.mlp_nparams()) * 0.15).astype(np.float32)
    ctx.mlp_set(theta, NORM_ID)
    inp = rng.normal(size=(300, 51)).astype(np.float32)
    got = ctx.mlp_forward(torch.as_tensor(inp).cuda()).cpu().numpy()
    want = oracle.mlp_forward(theta.astype(np.float64), inp.astype(np.float64))
    assert np.max(np.abs(got - want)) <= 1e-5 * max(1.0, np.abs(want).max())


def test_loss_gradient_matches_oracle_backprop():
    wl, ctx = _ctx((3, 3, 3))
    rng = np.random.default_rng(2)
    theta = (rng.normal(size=oracle.mlp_nparams()) * 0.15).astype(np.float32)
    ctx.mlp_set(theta, NORM_ID)
    inp = rng.normal(size=(257, 51)).astype(np.float32)
    tgt = rng.normal(size=(257, 3)).astype(np.float32)
    loss, g = ctx.mlp_grad(torch.as_tensor(inp).cuda(), torch.as_tensor(tgt).cuda())
    lo, go = oracle.mlp_loss_grad(theta.astype(np.float64), inp.astype(np.float64),
                                  tgt.astype(np.float64))
    g = g.cpu().numpy()
    assert abs(loss - lo) <= 1e-5 * abs(lo)
    assert np.max(np.abs(g - go)) <= 1e-4 * np.abs(go).max()


def test_features_match_oracle():
    wl, ctx = _ctx((4, 4, 4))
    x = wl.x.T.contiguous().cuda()
    f = ctx.mlp_features(x, wl.elem.cuda()).cpu().numpy()
    orc = oracle.Oracle(wl.mesh.as_dict())
    for i in range(0, wl.x.shape[0], 37):
        fo = orc.mlp_features(int(wl.elem[i]), H.np64(wl.x[i]))
        assert np.allclose(f[i, :3], fo[:3], atol=2e-6)
        assert np.allclose(f[i, 3:], fo[3:], atol=1e-6, rtol=1e-5)


def test_trained_start_beats_trilinear_and_converges_to_1e12():
    wl, ctx = _ctx((8, 8, 8))
    wl.mesh = W.channel_mesh((8, 8, 8), 3, amp=0.25)  # strongly curved: the guess matters
    ctx = H.gpu_context(wl, "fp32")
    inp, tgt = ctx.mlp_make_pairs(200_000, seed=5)
    losses = ctx.mlp_train(inp, tgt, epochs=12, batch=1024, lr=3e-3, seed=3)
    print("losses", losses)
    assert losses[-1] < 0.7 * losses[0]
    # held-out points
    x, el = W.seed_particles(wl.mesh, 20_000, seed=77, margin=0.0)
    xd, ed = x.T.contiguous().cuda(), el.cuda()
    c64 = H.gpu_context(wl, "fp64")
    xi_ref, _, st = c64.locate(xd, ed)
    assert int((st != 0).sum()) == 0
    theta, norm = ctx.mlp_get()
    feats = ctx.mlp_features(xd, ed)
    mean, sd, osc = norm[:51].cuda(), norm[51:102].cuda(), norm[102:].cuda()
    out = ctx.mlp_forward(((feats - mean) / sd).contiguous())
    xi_tri = feats[:, :3].double()
    xi_mlp = xi_tri + (out * osc).double()
    e_tri = (xi_tri - xi_ref.T).abs().max(dim=1).values
    e_mlp = (xi_mlp - xi_ref.T).abs().max(dim=1).values
    print("mean |xi0 - xi*|: trilinear", float(e_tri.mean()), "learned", float(e_mlp.mean()))
    assert float(e_mlp.mean()) < 0.5 * float(e_tri.mean())
    # the push-side BF16 network, through locate: same 1e-12 answer, fewer iterations
    ctx.set_config(guess=pt.GUESS_TRILINEAR)
    xi_t, it_t, st_t = ctx.locate(xd, ed)
    ctx.set_config(guess=pt.GUESS_MLP)
    xi_m, it_m, st_m = ctx.locate(xd, ed)
    assert int((st_t != 0).sum()) == 0 and int((st_m != 0).sum()) == 0
    assert float((xi_m - xi_ref).abs().max()) < 2e-12
    assert float((xi_t - xi_ref).abs().max()) < 2e-12
    print("mean iterations: trilinear", float(it_t.float().mean()), "learned",
          float(it_m.float().mean()))
    assert float(it_m.float().mean()) < float(it_t.float().mean())


def test_push_with_learned_start_matches_oracle():
    wl = W.curved_channel((6, 6, 6), 3, 5, P=400, nsteps=30, dt=2e-3)
    rng = np.random.default_rng(0)
    wl.v = wl.v * 4.0 + torch.as_tensor(rng.normal(size=(400, 3)) * 1.5)
    h = 2.0 / 6
    ctx = H.gpu_context(wl, "fp32", band_ref=2e-4, band_x=1e-4 * h)
    inp, tgt = ctx.mlp_make_pairs(100_000, seed=9)
    ctx.mlp_train(inp, tgt, epochs=3, batch=1024, lr=2e-3, seed=1)
    ctx.set_config(guess=pt.GUESS_MLP)
    parts = H.gpu_particles(wl, ctx)
    st = ctx.push(parts, wl.nsteps, wl.dt)
    g = H.gpu_result(parts)
    o = H.run_oracle(wl, band_ref=2e-4, band_x=1e-4 * h)
    res = H.compare(g, o, 2e-5)
    assert res["checked"] > 300 and st["crossings"] > 50


@pytest.mark.parametrize("engine", [1, 0])
def test_learned_start_inference_matches_oracle_network(engine):
    """The push-side BF16 network (engine 1: tcgen05 tensor-core kernel of the
    staged schedule; 0: warp-level mma.sync of the resident one) against the
    FP64 oracle network on the same weights: the start xi_tri + correction,
    on a strongly curved mesh where the correction is large, for a particle
    count that is not a multiple of the 128-particle tile."""
    wl = W.curved_channel((8, 8, 8), 3, 4, P=100, nsteps=1, dt=2e-3)
    wl.mesh = W.channel_mesh((8, 8, 8), 3, amp=0.25)
    ctx = H.gpu_context(wl, "fp32")
    inp, tgt = ctx.mlp_make_pairs(100_000, seed=5)
    ctx.mlp_train(inp, tgt, epochs=4, batch=1024, lr=3e-3, seed=3)
    theta, norm = ctx.mlp_get()
    x, el = W.seed_particles(wl.mesh, 4001, seed=78, margin=0.0)
    xd, ed = x.T.contiguous().cuda(), el.cuda()
    g = ctx.mlp_start(xd, ed, engine).T.double().cpu().numpy()
    orc = oracle.Oracle(wl.mesh.as_dict())
    th = theta.double().numpy()
    nm = norm.double().numpy()
    mean, sd, osc = nm[:51], nm[51:102], nm[102:]
    feats = np.array([orc.mlp_features(int(el[i]), H.np64(x[i])) for i in range(len(el))])
    out = oracle.mlp_forward(th, (feats - mean) / sd) * osc
    ref = feats[:, :3] + out
    scale = np.sqrt(np.mean(out ** 2))
    err = np.abs(g - ref)
    print("engine", engine, "correction rms", scale, "max err", err.max(), "mean", err.mean())
    assert scale > 1e-4
    # BF16 operands through four layers (~3 significant digits per product)
    assert err.max() <= 0.05 * scale and err.mean() <= 0.01 * scale
