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
