"""Two-way coupling source (Sec. 2.3, Eq. theory:source) with Lagrange weights:
FP32 atomics and the deterministic segmented reduction against the FP64 oracle
(1e-5 relative on per-element nodal sums), momentum conservation (1e-6) and
bitwise reproducibility of the segmented mode."""
import math

import numpy as np
import pytest
import torch

from paper_2211_05458_gb300 import pt
from paper_2211_05458_gb300 import workloads as W
import oracle
from tests import helpers as H

pytestmark = pytest.mark.gpu


def _state(dims=(6, 5, 4), ngeo=2, N=7, P=3000, seed=0):
    wl = W.curved_channel(dims, ngeo, N, P=P, nsteps=1, seed=seed, mass_loading=0.3)
    rng = np.random.default_rng(seed)
    wl.v = wl.v + torch.as_tensor(rng.normal(size=(P, 3)) * 0.3)  # slip -> non-zero drag
    return wl


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("mode", [pt.DEPOSIT_ATOMIC, pt.DEPOSIT_SEGMENTED])
def test_deposit_matches_oracle(precision, mode):
    wl = _state()
    ctx = H.gpu_context(wl, precision)
    parts = H.gpu_particles(wl, ctx)
    S = ctx.deposit(parts, mode).double().cpu().numpy()
    orc = H.make_oracle(wl)
    So = orc.deposit(H.oracle_params(wl), H.np64(wl.x), H.np64(wl.v), H.np64(wl.d),
                     H.np64(wl.elem).astype(np.int32))
    # per-element nodal sums of the four sources
    es, eo = S.sum(axis=2), So.sum(axis=2)
    scale = np.abs(eo).max(axis=0, keepdims=True)
    assert np.max(np.abs(es - eo) / scale) < 1e-5
    # nodal values
    assert np.max(np.abs(S - So)) < 1e-5 * np.abs(So).max()
    # total momentum: sum of the deposited source = -(sum of drag forces)
    tot_s, tot_o = S[:, :3].sum(axis=(0, 2)), So[:, :3].sum(axis=(0, 2))
    assert np.all(np.abs(tot_s - tot_o) <= 1e-6 * np.abs(So[:, :3]).sum(axis=(0, 2)))


def test_segmented_is_bitwise_reproducible_and_close_to_atomic():
    wl = _state(P=20_000)
    ctx = H.gpu_context(wl, "fp32")
    parts = H.gpu_particles(wl, ctx)
    a = ctx.deposit(parts, pt.DEPOSIT_SEGMENTED).clone()
    b = ctx.deposit(parts, pt.DEPOSIT_SEGMENTED).clone()
    assert torch.equal(a, b)
    c = ctx.deposit(parts, pt.DEPOSIT_ATOMIC)
    assert float((a - c).abs().max()) <= 1e-5 * float(a.abs().max())


def test_empty_elements_are_zero_and_frozen_particles_skipped():
    wl = _state(P=50)
    ctx = H.gpu_context(wl, "fp32")
    parts = H.gpu_particles(wl, ctx)
    parts.status[:] = pt.ST_LOST
    S = ctx.deposit(parts, pt.DEPOSIT_SEGMENTED)
    assert float(S.abs().max()) == 0.0
    S = ctx.deposit(parts, pt.DEPOSIT_ATOMIC)
    assert float(S.abs().max()) == 0.0


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("summation", [pt.DEPOSIT_ATOMIC, pt.DEPOSIT_SEGMENTED])
def test_nearest_node_projection_matches_oracle(precision, summation):
    """Sec. 2.3 projection P{a} = a / V_ijk at the nearest node.  Particles whose
    xi lies within 1e-8 of a midpoint between two nodes (where either node is
    a correct choice) are frozen on both sides."""
    wl = _state(dims=(5, 4, 4), ngeo=2, N=5, P=4000, seed=3)
    orc = H.make_oracle(wl)
    x, el = H.np64(wl.x), H.np64(wl.elem).astype(np.int32)
    xn = oracle.nodes(wl.node_type, wl.N + 1)
    mids = 0.5 * (xn[1:] + xn[:-1])
    status = np.zeros(len(el), np.uint32)
    for i in range(len(el)):
        ok, xi, _ = orc.newton(int(el[i]), x[i])
        if ok and np.min(np.abs(xi[:, None] - mids[None, :])) < 1e-8:
            status[i] = oracle.ST_LOST
    p = H.oracle_params(wl)
    So = orc.deposit_nearest(p, x, H.np64(wl.v), H.np64(wl.d), el, status)
    ctx = H.gpu_context(wl, precision)
    parts = H.gpu_particles(wl, ctx)
    parts.status.copy_(torch.as_tensor(status.astype(np.int32)))
    S = ctx.deposit(parts, summation | pt.DEPOSIT_NEAREST).double().cpu().numpy()
    # the same nodes are hit, with the same densities
    assert np.array_equal(S != 0, So != 0)
    assert np.max(np.abs(S - So)) <= 1e-5 * np.abs(So).max()
    # per-element sums of each source component
    es, eo = S.sum(axis=2), So.sum(axis=2)
    assert np.max(np.abs(es - eo) / np.abs(eo).max(axis=0, keepdims=True)) < 1e-5


def test_nearest_segmented_is_bitwise_reproducible():
    wl = _state(P=20_000)
    ctx = H.gpu_context(wl, "fp32")
    parts = H.gpu_particles(wl, ctx)
    mode = pt.DEPOSIT_SEGMENTED | pt.DEPOSIT_NEAREST
    a = ctx.deposit(parts, mode).clone()
    b = ctx.deposit(parts, mode).clone()
    assert torch.equal(a, b)
    c = ctx.deposit(parts, pt.DEPOSIT_NEAREST)
    assert float((a - c).abs().max()) <= 1e-5 * float(a.abs().max())


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_two_way_time_step_guard_counts_like_oracle(precision):
    """Sec. 2.3 restriction dt <= 2.75 tau_p, reported as PT_WARN_DT with the
    number of violating particles; the push itself still runs."""
    wl = _state(P=2000, seed=4)
    rng = np.random.default_rng(4)
    wl.d = torch.as_tensor(10 ** rng.uniform(-5.2, -4.9, 2000))  # dt / tau_p in [1, 5]
    ctx = H.gpu_context(wl, precision)
    parts = H.gpu_particles(wl, ctx)
    d_used = parts.d.double().cpu().numpy()  # as the kernel reads them (FP32 rounded in FP32 mode)
    dt = 1e-3
    tau = wl.rho_p * d_used ** 2 / (18 * wl.mu)
    assert np.min(np.abs(dt / (2.75 * tau) - 1)) > 1e-6  # no particle at the threshold
    expect = oracle.dt_violations(H.oracle_params(wl), d_used, dt)
    assert 0 < expect < 2000
    st = ctx.push(parts, 1, dt)
    assert st["dt_warn"] == expect
    errors = st["newton_fail"] + st["lost"] + st["cross_cap"]
    assert st["status_code"] == pt.PT_WARN_DT or errors > 0


@pytest.mark.parametrize("mode", [pt.DEPOSIT_SEGMENTED, pt.DEPOSIT_SEGMENTED | pt.DEPOSIT_NEAREST])
def test_segmented_with_large_segments_matches_oracle_and_is_reproducible(mode):
    """8 elements holding ~5000 particles each: every segment is longer than
    the shared-memory sort, so the index order is made in global memory."""
    wl = W.tgv_box(2, 3, P=40_000, nsteps=1, seed=3, precision="fp32")
    rng = np.random.default_rng(3)
    wl.v = torch.as_tensor(rng.normal(size=(40_000, 3)) * 0.3)  # slip: non-zero energy source
    ctx = H.gpu_context(wl, "fp32")
    parts = H.gpu_particles(wl, ctx)
    counts = np.bincount(H.np64(wl.elem).astype(np.int64), minlength=8)
    assert counts.min() > 4096
    a = ctx.deposit(parts, mode).clone()
    b = ctx.deposit(parts, mode).clone()
    assert torch.equal(a, b)
    orc = H.make_oracle(wl)
    args = (H.oracle_params(wl), H.np64(wl.x), H.np64(wl.v), H.np64(wl.d),
            H.np64(wl.elem).astype(np.int32))
    So = orc.deposit_nearest(*args) if mode & pt.DEPOSIT_NEAREST else orc.deposit(*args)
    S = a.double().cpu().numpy()
    assert np.max(np.abs(S - So)) <= 1e-5 * np.abs(So).max()
    # per-element sums of ~5000 sources that largely cancel: relative to the
    # sum of the nodal magnitudes (the sum's condition)
    es, eo = S.sum(axis=2), So.sum(axis=2)
    cond = np.abs(So).sum(axis=2).max(axis=0, keepdims=True)
    assert np.max(np.abs(es - eo) / cond) < 1e-5
