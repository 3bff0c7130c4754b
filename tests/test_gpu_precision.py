"""Per-result error of the FP32 mode against the FP64 oracle (the precision
split: FP32 interpolation, drag and RK update; the inverse map converged to
1e-12 with double-float final iterations).  For a fixed sample of (x, element)
with a slip velocity, the terms of one RK stage -- xi, rho and rho u at xi,
the particle's acceleration and the stage increments -- come from the push's
own code (pt_stage_terms) and from the oracle at the oracle's xi."""
import numpy as np
import pytest
import torch

from paper_2211_05458_gb300 import pt
from paper_2211_05458_gb300 import workloads as W
from tests import helpers as H

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,tol", [("fp32", 2e-5), ("fp64", 1e-12)])
def test_stage_terms_match_oracle(precision, tol):
    wl = W.curved_channel((10, 10, 10), 3, 5, P=20_000, nsteps=1, seed=5)
    ctx = H.gpu_context(wl, precision)
    orc = H.make_oracle(wl)
    err = H.stage_term_errors(wl, ctx, orc, 2000, seed=5)
    print("per-result errors:", precision, err)
    assert err["xi"] <= 2e-12
    for k in ("U", "acc", "dx", "dv"):
        assert err[k] <= tol, (k, err[k])
