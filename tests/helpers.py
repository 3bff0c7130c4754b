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
    """Oracle push of particles idx (all if None) from the workload's initial state.
    The result also carries the oracle context and parameters (keys "_orc",
    "_params") so that compare() can locate final positions with them."""
    orc = orc or make_oracle(wl)
    idx = np.arange(wl.x.shape[0]) if idx is None else np.asarray(idx)
    x = np64(wl.x)[idx]
    v = np64(wl.v)[idx]
    d = np64(wl.d)[idx]
    el = np64(wl.elem).astype(np.int32)[idx]
    p = oracle_params(wl, band_ref, band_x, **kw)
    res = orc.push(p, x, v, d, el, nsteps=wl.nsteps if nsteps is None else nsteps, dt=wl.dt)
    res["_orc"], res["_params"] = orc, p
    return res


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


def _periods(orc_obj):
    """Period of the mesh along each axis (0 where it is not periodic): the
    largest |translation| of a periodic face."""
    sh = orc_obj._keep["shift"].reshape(-1, 3)
    bc = orc_obj._keep["bc"].reshape(-1)
    per = bc == 2
    return np.abs(sh[per]).max(axis=0) if per.any() else np.zeros(3)


def _xi_max(orc_obj, params, e, x):
    ok, xi, _ = orc_obj.newton(int(e), x, params)
    return float(np.max(np.abs(xi))) if ok else math.inf


def compare(gpu, orc, tol, xscale=1.0, vscale=1.0, min_checked=0.95, wall_tol=1e-4):
    """Particle-by-particle parity of a GPU push with the oracle.

    Strict set: every particle that is frozen on neither side, met the
    near-face band of no wall or open face on either side (PT_ST_NEAR_WALL) and
    whose final position lies outside the band of its owner's faces on both
    sides.  There element ids and wall hits are bit-exact and x, v agree within
    tol relative (to max(|ref|, scale)).  A near-face event on an internal or
    periodic face before the end does not leave the strict set: it can only
    move the stage at which the owner changes along the same straight segment.

    The rest is still checked:
      * ends near a face: the GPU's owner holds the GPU's position within the
        band; the owners are equal or the oracle's owner is among the brute-
        force owners of the GPU's position within 4 bands; hits equal; x (up to
        a period of the mesh) and v within tol;
      * near a wall or open face: the GPU's owner holds its position within
        the band; hits differ by at most one; x (up to a period) and v within
        wall_tol relative: a reflection taken one stage earlier or later
        mirrors the same path, and only the fluid's velocity component normal
        to the wall enters the drag of that one stage differently.
    Frozen states must agree outside these sets."""
    orc_obj, prm = orc.get("_orc"), orc.get("_params")
    assert orc_obj is not None, "compare() needs the oracle result of run_oracle()"
    band = float(prm.band_ref)
    stg = gpu["status"].astype(np.uint32)
    sto = orc["status"].astype(np.uint32)
    frozen = ((stg | sto) & oracle.ST_FROZEN) != 0
    nearwall = ((stg | sto) & oracle.ST_NEAR_WALL) != 0
    n = len(stg)
    ximax_g = np.full(n, math.inf)
    ximax_o = np.full(n, math.inf)
    for i in np.flatnonzero(~frozen):
        ximax_g[i] = _xi_max(orc_obj, prm, gpu["elem"][i], gpu["x"][i])
        ximax_o[i] = _xi_max(orc_obj, prm, orc["elem"][i], orc["x"][i])
    endnear = ~frozen & ((ximax_g > 1.0 - band) | (ximax_o > 1.0 - band))
    strict = ~frozen & ~nearwall & ~endnear
    assert strict.sum() >= min_checked * n, (
        f"only {strict.sum()} of {n} in the strict check ({nearwall.sum()} near a wall, "
        f"{endnear.sum()} ending near a face, {frozen.sum()} frozen)")
    ok = strict
    ge, oe = gpu["elem"][ok], orc["elem"][ok]
    bad = np.flatnonzero(ge != oe)
    assert bad.size == 0, f"{bad.size} element mismatches, e.g. {ge[bad[:5]]} vs {oe[bad[:5]]}"
    gh, oh = gpu["hits"][ok], orc["hits"][ok]
    assert np.array_equal(gh, oh), f"wall-hit mismatch {np.flatnonzero(gh != oh)[:5]}"
    ex = np.abs(gpu["x"][ok] - orc["x"][ok]) / np.maximum(np.abs(orc["x"][ok]), xscale)
    ev = np.abs(gpu["v"][ok] - orc["v"][ok]) / np.maximum(np.abs(orc["v"][ok]), vscale)
    assert ex.size == 0 or ex.max() <= tol, f"position rel error {ex.max():.3e} > {tol:.1e}"
    assert ev.size == 0 or ev.max() <= tol, f"velocity rel error {ev.max():.3e} > {tol:.1e}"
    # the particles outside the strict set
    per = _periods(orc_obj)
    loose = ~frozen & ~strict
    ex_l = ev_l = 0.0
    for i in np.flatnonzero(loose):
        assert ximax_g[i] <= 1.0 + band, (
            f"particle {i}: GPU position outside its element {gpu['elem'][i]} "
            f"(max |xi| = {ximax_g[i]:.3e})")
        raw = gpu["x"][i] - orc["x"][i]
        dx = raw.copy()
        for r in range(3):
            if per[r] > 0:
                dx[r] -= per[r] * np.round(dx[r] / per[r])
        exi = np.max(np.abs(dx) / np.maximum(np.abs(orc["x"][i]), xscale))
        evi = np.max(np.abs(gpu["v"][i] - orc["v"][i]) / np.maximum(np.abs(orc["v"][i]), vscale))
        lim = wall_tol if nearwall[i] else tol
        assert exi <= lim and evi <= lim, (
            f"particle {i} ({'near a wall' if nearwall[i] else 'ends near a face'}): "
            f"x rel {exi:.3e}, v rel {evi:.3e} > {lim:.1e}")
        ex_l, ev_l = max(ex_l, exi), max(ev_l, evi)
        dh = abs(int(gpu["hits"][i]) - int(orc["hits"][i]))
        assert dh <= (1 if nearwall[i] else 0), f"particle {i}: wall hits differ by {dh}"
        if gpu["elem"][i] != orc["elem"][i] and not nearwall[i]:
            # the GPU's position, brought to the oracle's side of a periodic
            # face, lies in the oracle's owner to within a few bands
            xo = _xi_max(orc_obj, prm, orc["elem"][i], gpu["x"][i] - (raw - dx))
            assert xo <= 1.0 + 4 * band, (
                f"particle {i}: owners {gpu['elem'][i]} (GPU) and {orc['elem'][i]} (oracle) "
                f"differ by more than the band (max |xi| = {xo:.3e} in the oracle's)")
    # frozen states agree (a particle frozen on one side only is a failure)
    fz_g = (stg & oracle.ST_FROZEN) != 0
    fz_o = (sto & oracle.ST_FROZEN) != 0
    bad = np.flatnonzero((fz_g != fz_o) & ~nearwall & ~endnear)
    assert bad.size == 0, (f"frozen-state mismatch at {bad[:5]}: gpu status "
                           f"{stg[bad[:5]]}, oracle {sto[bad[:5]]}")
    near = ((stg | sto) & oracle.ST_NEAR_FACE) != 0
    res = dict(n=n, checked=int(strict.sum()), near_face=int(near.sum()),
               near_wall=int(nearwall.sum()), end_near=int(endnear.sum()),
               loose_checked=int(loose.sum()), frozen=int(frozen.sum()),
               ex=float(ex.max()) if ex.size else 0.0, ev=float(ev.max()) if ev.size else 0.0,
               ex_loose=ex_l, ev_loose=ev_l)
    print("parity:", res)
    return res


def stage_term_errors(wl, ctx, orc, n, seed=0, slip=0.3):
    """Max error of each first-stage term over n sampled particles, relative to
    the largest oracle value of that term (normwise, per component)."""
    rng = np.random.default_rng(seed)
    P = wl.x.shape[0]
    idx = np.sort(rng.choice(P, size=min(n, P), replace=False))
    x = np64(wl.x)[idx]
    v = np64(wl.v)[idx] + slip * rng.normal(size=(len(idx), 3))
    d = np64(wl.d)[idx]
    el = np64(wl.elem).astype(np.int32)[idx]
    from paper_2211_05458_gb300 import pt
    parts = pt.ParticleSet.create(x, v, d, el, ctx.precision, "cuda")
    g = ctx.stage_terms(parts, wl.dt)
    torch.cuda.synchronize()
    assert int((parts.status & pt.ST_FROZEN).sum()) == 0
    prm = oracle_params(wl)
    # the oracle at the GPU's inputs as the kernel reads them (v, d rounded to
    # the particle precision)
    vk, dk = parts.v.T.double().cpu().numpy(), parts.d.double().cpu().numpy()
    ref = {k: [] for k in ("xi", "U", "acc", "dx", "dv")}
    for i in range(len(idx)):
        o = orc.stage1(prm, el[i], x[i], vk[i], dk[i], wl.dt)
        assert o is not None
        for k in ref:
            ref[k].append(o[k][:4] if k == "U" else o[k])
    err = {}
    for k in ref:
        o = np.array(ref[k])
        gk = g[k].T.double().cpu().numpy()
        if k == "xi":
            err[k] = float(np.max(np.abs(gk - o)))  # absolute, reference units
        else:
            err[k] = float(np.max(np.abs(gk - o) / np.abs(o).max(axis=0, keepdims=True)))
    return err
