"""Extra force models of Sec. 2.2 on the GPU against the FP64 oracle: the
Haider-Levenspiel drag law and the Saffman lift with Mei's correction, in the
push (FP64 1e-12, FP32 2e-5) and in the two-way source (1e-5)."""
import numpy as np
import pytest
import torch

from paper_2211_05458_gb300 import pt
from paper_2211_05458_gb300 import workloads as W
from tests import helpers as H

pytestmark = pytest.mark.gpu


def _shear_channel(seed=0, P=400, nsteps=30):
    wl = W.curved_channel((6, 5, 4), 2, 5, P=P, nsteps=nsteps, dt=2e-3, st=(0.5, 50.0), seed=seed)
    # a strong, uniform shear on top of the channel flow: lift well above rounding
    rng = np.random.default_rng(seed)
    A = rng.normal(size=(3, 3)) * 3.0
    wl.U = W.fluid_linear(wl.mesh, wl.N, A, (0.4, 0.0, 0.1), (0.02, -0.01, 0.03))
    wl.v = wl.v + torch.as_tensor(rng.normal(size=tuple(wl.v.shape)) * 0.5)
    return wl


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
@pytest.mark.parametrize("law", [1, 2])
def test_push_with_lift_matches_oracle(precision, tol, law):
    wl = _shear_channel(seed=law)
    wl.drag_law = law
    band = (1e-10, 1e-10) if precision == "fp64" else (2e-4, 1e-4 * 2.0 / 5)
    cfg = dict(lift=1, sphericity=0.8)
    ctx = H.gpu_context(wl, precision, band_ref=band[0], band_x=band[1], **cfg)
    parts = H.gpu_particles(wl, ctx)
    st = ctx.push(parts, wl.nsteps, wl.dt)
    g = H.gpu_result(parts)
    o = H.run_oracle(wl, band_ref=band[0], band_x=band[1], **cfg)
    res = H.compare(g, o, tol)
    assert res["checked"] >= 350
    # the lift is not negligible: without it the oracle ends elsewhere
    o0 = H.run_oracle(wl, band_ref=band[0], band_x=band[1], sphericity=0.8)
    assert np.max(np.abs(o0["x"] - o["x"])) > 10 * max(tol, 2e-5)


@pytest.mark.parametrize("mode", [pt.DEPOSIT_ATOMIC, pt.DEPOSIT_SEGMENTED,
                                  pt.DEPOSIT_ATOMIC | pt.DEPOSIT_NEAREST])
def test_deposit_with_lift_and_haider_levenspiel_matches_oracle(mode):
    wl = _shear_channel(seed=5, P=3000, nsteps=1)
    wl.drag_law = 2
    cfg = dict(lift=1, sphericity=0.7)
    ctx = H.gpu_context(wl, "fp32", **cfg)
    parts = H.gpu_particles(wl, ctx)
    S = ctx.deposit(parts, mode).double().cpu().numpy()
    orc = H.make_oracle(wl)
    p = H.oracle_params(wl, **cfg)
    args = (H.np64(wl.x), H.np64(wl.v), H.np64(wl.d), H.np64(wl.elem).astype(np.int32))
    So = orc.deposit_nearest(p, *args) if mode & pt.DEPOSIT_NEAREST else orc.deposit(p, *args)
    assert np.max(np.abs(S - So)) <= 1e-5 * np.abs(So).max()
    es, eo = S.sum(axis=2), So.sum(axis=2)
    assert np.max(np.abs(es - eo) / np.abs(eo).max(axis=0, keepdims=True)) < 1e-5
    # lift present: the oracle source without it differs beyond the tolerance
    p0 = H.oracle_params(wl, sphericity=0.7)
    S0 = orc.deposit_nearest(p0, *args) if mode & pt.DEPOSIT_NEAREST else orc.deposit(p0, *args)
    assert np.max(np.abs(S0 - So)) > 5e-5 * np.abs(So).max()


def test_bad_force_config_is_rejected():
    wl = _shear_channel(P=10, nsteps=1)
    with pytest.raises(pt.PtError):
        H.gpu_context(wl, "fp32", lift=2)
    wl.drag_law = 2
    with pytest.raises(pt.PtError):
        H.gpu_context(wl, "fp32", sphericity=0.0)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
def test_push_with_gravity_and_buoyancy_matches_oracle(precision, tol):
    """Eq. theory:maxey: gravity on m_p - m_f (g (1 - rho/rho_p), rho interpolated);
    light particles so that the buoyancy is 10 % of the weight."""
    wl = W.curved_channel((6, 5, 4), 2, 5, P=400, nsteps=30, dt=2e-3, st=(0.5, 50.0), seed=9,
                          rho_p=12.0)
    band = (1e-10, 1e-10) if precision == "fp64" else (2e-4, 1e-4 * 2.0 / 5)
    cfg = dict(buoyancy=1, g=(0.0, -9.81, 0.0))
    ctx = H.gpu_context(wl, precision, band_ref=band[0], band_x=band[1], **cfg)
    parts = H.gpu_particles(wl, ctx)
    ctx.push(parts, wl.nsteps, wl.dt)
    o = H.run_oracle(wl, band_ref=band[0], band_x=band[1], **cfg)
    res = H.compare(H.gpu_result(parts), o, tol)
    assert res["checked"] >= 350
    o0 = H.run_oracle(wl, band_ref=band[0], band_x=band[1], g=(0.0, -9.81, 0.0))
    assert np.max(np.abs(o0["v"] - o["v"])) > 100 * max(tol, 2e-5)
