"""Shared helpers of the parity tests: run the same seeded workload through the
oracle (CPU, FP64) and through libpt (GPU), and compare particle by particle."""
from __future__ import annotations

import math

import numpy as np
import torch

import oracle
from paper_2211_05458_gb300 import workloads as W


def np64(t):
    return t.detach().cpu().numpy().astype(np.float64) if torch.is_tensor(t) else np.asarray(t)


def oracle_params(wl: W.Workload, band_ref=1e-10, band_x=1e-10, **kw):
    return oracle.make_params(mu=wl.mu, rho_p=wl.rho_p, drag_law=wl.drag_law, band_ref=band_ref,
                              band_x=band_x, **kw)


def run_oracle(wl: W.Workload, idx=None, nsteps=None, band_ref=1e-10, band_x=1e-10, orc=None,
               **kw):
    """Oracle push of particles idx (all if None) from the workload's initial state."""
    orc = orc or make_oracle(wl)
    idx = np.arange(wl.x.shape[0]) if idx is None else np.asarray(idx)
    x = np64(wl.x)[idx]
    v = np64(wl.v)[idx]
    d = np64(wl.d)[idx]
    el = np64(wl.elem).astype(np.int32)[idx]
    p = oracle_params(wl, band_ref, band_x, **kw)
    return orc.push(p, x, v, d, el, nsteps=wl.nsteps if nsteps is None else nsteps, dt=wl.dt)


def make_oracle(wl: W.Workload):
    orc = oracle.Oracle(wl.mesh.as_dict())
    orc.set_fluid(wl.N, wl.node_type, np64(wl.U).reshape(-1))
    return orc


def gpu_context(wl: W.Workload, precision=None, **cfg):
    from paper_2211_05458_gb300 import pt
    prec = pt.FP64 if (precision or wl.precision) == "fp64" else pt.FP32
    ctx = pt.Context(wl.mesh, precision=prec, mu=wl.mu, rho_p=wl.rho_p, drag_law=wl.drag_law,
                     **cfg)
    U = wl.U.to("cuda", torch.float64 if prec == pt.FP64 else torch.float32).contiguous()
    ctx.set_fluid(wl.N, wl.node_type, U)
    return ctx


def gpu_particles(wl: W.Workload, ctx, idx=None):
    from paper_2211_05458_gb300 import pt
    sel = slice(None) if idx is None else torch.as_tensor(np.asarray(idx))
    return pt.ParticleSet.create(wl.x[sel], wl.v[sel], wl.d[sel], wl.elem[sel], ctx.precision,
                                 "cuda")


def gpu_result(parts):
    return dict(x=parts.x.T.cpu().numpy().astype(np.float64),
                v=parts.v.T.cpu().numpy().astype(np.float64),
                elem=parts.elem.cpu().numpy(), hits=parts.hits.cpu().numpy(),
                status=parts.status.cpu().numpy().astype(np.uint32))


def compare(gpu, orc, tol, xscale=1.0, vscale=1.0, min_checked=0.9):
    """Element ids and wall hits bit-exact, x and v within tol relative (to
    max(|ref|, scale)), outside the near-face band flagged by either side."""
    near = ((gpu["status"] | orc["status"]) & oracle.ST_NEAR_FACE) != 0
    frozen = ((gpu["status"] | orc["status"]) & oracle.ST_FROZEN) != 0
    ok = ~near & ~frozen
    n = len(ok)
    assert ok.sum() >= min_checked * n, f"only {ok.sum()} of {n} comparable"
    ge, oe = gpu["elem"][ok], orc["elem"][ok]
    bad = np.flatnonzero(ge != oe)
    assert bad.size == 0, f"{bad.size} element mismatches, e.g. {ge[bad[:5]]} vs {oe[bad[:5]]}"
    gh, oh = gpu["hits"][ok], orc["hits"][ok]
    assert np.array_equal(gh, oh), f"wall-hit mismatch {np.flatnonzero(gh != oh)[:5]}"
    ex = np.abs(gpu["x"][ok] - orc["x"][ok]) / np.maximum(np.abs(orc["x"][ok]), xscale)
    ev = np.abs(gpu["v"][ok] - orc["v"][ok]) / np.maximum(np.abs(orc["v"][ok]), vscale)
    assert ex.max() <= tol, f"position rel error {ex.max():.3e} > {tol:.1e}"
    assert ev.max() <= tol, f"velocity rel error {ev.max():.3e} > {tol:.1e}"
    # frozen states agree (a particle frozen on one side only is a failure)
    fz_g = (gpu["status"] & oracle.ST_FROZEN) != 0
    fz_o = (orc["status"] & oracle.ST_FROZEN) != 0
    bad = np.flatnonzero((fz_g != fz_o) & ~near)
    assert bad.size == 0, (f"frozen-state mismatch at {bad[:5]}: gpu status "
                           f"{gpu['status'][bad[:5]]}, oracle {orc['status'][bad[:5]]}")
    return dict(checked=int(ok.sum()), near=int(near.sum()), ex=float(ex.max()),
                ev=float(ev.max()))
