"""Batched push of many independent boxes (boxes grouped by polynomial degree,
one persistent kernel per group and chunk with a tuned block size, captured in
a CUDA graph after the tuning call): identical to pushing every box alone, and
within the FP32-mode tolerance of the oracle."""
import numpy as np
import pytest
import torch

from paper_2211_05458_gb300 import pt
from paper_2211_05458_gb300 import workloads as W
from tests import helpers as H

pytestmark = pytest.mark.gpu


def _setup(nbox=6, seed=1):
    boxes = W.batched_boxes(nbox=nbox, seed=seed, side_range=(3, 5), P_range=(50, 300),
                            nsteps=20, dt=2e-3)
    for b, wl in enumerate(boxes):
        rng = np.random.default_rng(b)
        wl.v = torch.as_tensor(rng.normal(size=tuple(wl.x.shape)) * 2.0)
        wl.d = torch.full_like(wl.d, 3e-3)
    ctxs = [H.gpu_context(wl, "fp32") for wl in boxes]
    parts = [H.gpu_particles(wl, c) for wl, c in zip(boxes, ctxs)]
    return boxes, ctxs, parts


def test_batch_equals_individual_pushes_bitwise():
    boxes, ctxs, parts = _setup()
    parts[0].elem[0] = -1  # an owner out of range: lost in both, untouched otherwise
    ref = [p.clone() for p in parts]
    # 20 steps are two chunks: calls 1 and 2 try the three block sizes, call 3
    # captures the graph and replays it, call 4 replays it again
    for _ in range(4):
        st = pt.push_batch(ctxs, parts, 20, 2e-3)
    for c, p in zip(ctxs, ref):
        for _ in range(4):
            c.push(p, 20, 2e-3)
    torch.cuda.synchronize()
    for a, b in zip(parts, ref):
        for f in ("x", "v", "elem", "hits", "status"):
            assert torch.equal(getattr(a, f), getattr(b, f)), f
    assert sum(s["particle_steps"] for s in st) == 20 * (sum(p.n for p in parts) - 1)
    assert sum(s["crossings"] for s in st) > 100
    assert int(parts[0].status[0]) & pt.ST_LOST
    # one group per polynomial degree, each with a tuned block size
    tun = pt.batch_tuning(ctxs[0])
    print("batch tuning", tun)
    assert [g["N"] for g in tun] == sorted({wl.N for wl in boxes})
    assert all(g["block"] in (64, 96, 128) and min(g["ms_per_step"]) > 0 for g in tun)


def test_batch_matches_oracle_fp32():
    boxes, ctxs, parts = _setup(nbox=4, seed=2)
    pt.push_batch(ctxs, parts, 20, 2e-3)
    for wl, p in zip(boxes, parts):
        g = H.gpu_result(p)
        wl.nsteps, wl.dt = 20, 2e-3
        o = H.run_oracle(wl, band_ref=2e-4, band_x=1e-4 / 5)
        H.compare(g, o, 2e-5)


def test_batch_rejects_mixed_configurations():
    boxes, ctxs, parts = _setup(nbox=2)
    ctxs[1].set_config(guess=pt.GUESS_TRILINEAR)
    wl = W.curved_channel((3, 3, 3), 2, 3, P=10, nsteps=1)
    other = H.gpu_context(wl, "fp32")
    with pytest.raises(pt.PtError):
        pt.push_batch([ctxs[0], other], [parts[0], H.gpu_particles(wl, other)], 1, 1e-3)
