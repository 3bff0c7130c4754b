"""The staged schedule (one kernel per RK stage over the element-sorted
particle state, exact tracking of the listed segments on full warps) against
the resident one (every particle in registers for the whole call) and against
the FP64 oracle.  Both schedules run the same arithmetic in the same order per
particle, so their results are bitwise equal."""
import numpy as np
import pytest
import torch

from paper_2211_05458_gb300 import pt
from paper_2211_05458_gb300 import workloads as W
from tests import helpers as H

pytestmark = pytest.mark.gpu

FIELDS = ("x", "v", "elem", "hits", "status")


def _speed_up(wl, seed=0):
    rng = np.random.default_rng(seed)
    wl.v = wl.v * 4.0 + torch.as_tensor(rng.normal(size=tuple(wl.v.shape)) * 1.5)


def _both(wl, precision, steps=None, mlp=None, **cfg):
    """Push the same particles with both schedules; returns (resident, staged,
    stats of each)."""
    out, stats = [], []
    for sched in (pt.SCHEDULE_RESIDENT, pt.SCHEDULE_STAGED):
        ctx = H.gpu_context(wl, precision, schedule=sched, **cfg)
        if mlp is not None:
            ctx.mlp_set(*mlp)
            ctx.set_config(guess=pt.GUESS_MLP)
        parts = H.gpu_particles(wl, ctx)
        stats.append(ctx.push(parts, wl.nsteps if steps is None else steps, wl.dt))
        torch.cuda.synchronize()
        out.append(H.gpu_result(parts))
        ctx.close()
    return out[0], out[1], stats


def _assert_same(a, b, sa, sb):
    for k in FIELDS:
        diff = (a[k] != b[k]).reshape(len(a[k]), -1).any(axis=1)
        assert not diff.any(), (k, np.flatnonzero(diff)[:5])
    for k in ("particle_steps", "crossings", "wall_hits", "slow_track", "near_face", "near_wall"):
        assert sa[k] == sb[k], (k, sa[k], sb[k])


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("ngeo,N", [(2, 5), (3, 5), (1, 4), (4, 7)])
def test_staged_equals_resident_curved_channel(precision, ngeo, N):
    wl = W.curved_channel((6, 6, 6), ngeo, N, P=1500, nsteps=25, dt=2e-3, seed=ngeo)
    _speed_up(wl, ngeo)
    h = 2.0 / 6
    band = dict(band_ref=2e-4, band_x=1e-4 * h) if precision == "fp32" else {}
    a, b, (sa, sb) = _both(wl, precision, rebin_every=7, **band)
    assert sa["crossings"] > 100 and sa["wall_hits"] > 5
    _assert_same(a, b, sa, sb)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("cfg", [dict(track=pt.TRACK_REFERENCE), dict(curved_faces=1),
                                 dict(lift=1, sphericity=0.8),
                                 dict(g=(0.0, -9.81, 0.0), buoyancy=1)])
def test_staged_equals_resident_options(precision, cfg):
    wl = W.curved_channel((6, 6, 6), 3, 5, P=1000, nsteps=20, dt=2e-3, seed=3)
    _speed_up(wl, 3)
    if "sphericity" in cfg:
        wl.drag_law = 2  # Haider-Levenspiel
    h = 2.0 / 6
    band = dict(band_ref=2e-4, band_x=1e-4 * h) if precision == "fp32" else {}
    a, b, (sa, sb) = _both(wl, precision, **cfg, **band)
    _assert_same(a, b, sa, sb)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_staged_equals_resident_curved_walls_and_mortars(precision):
    mesh = W.channel_mesh((5, 4, 4), 2, amp=0.1, curved_walls=True)
    wl = W.curved_channel((5, 4, 4), 2, 3, P=600, nsteps=30, dt=5e-3)
    wl.mesh = mesh
    wl.U, _ = W.fluid_channel(mesh, 3, 0, seed=0)
    wl.x, wl.elem = W.seed_particles(mesh, 600, seed=3)
    rng = np.random.default_rng(0)
    wl.v = torch.as_tensor(rng.normal(size=(600, 3)) * 3.0)
    wl.d = torch.full((600,), 4e-3, dtype=torch.float64)
    a, b, (sa, sb) = _both(wl, precision)
    assert sa["wall_hits"] > 20
    _assert_same(a, b, sa, sb)
    wl = W.mortar_tgv(3, 2, "st", N=4, P=400, nsteps=40)
    a, b, (sa, sb) = _both(wl, precision)
    _assert_same(a, b, sa, sb)


def test_staged_equals_resident_learned_start():
    wl = W.curved_channel((6, 6, 6), 3, 5, P=1000, nsteps=20, dt=2e-3, seed=4)
    _speed_up(wl, 4)
    h = 2.0 / 6
    ctx = H.gpu_context(wl, "fp32")
    inp, tgt = ctx.mlp_make_pairs(100_000, seed=9)
    ctx.mlp_train(inp, tgt, epochs=3, batch=1024, lr=2e-3, seed=1)
    net = ctx.mlp_get()
    a, b, (sa, sb) = _both(wl, "fp32", mlp=net, band_ref=2e-4, band_x=1e-4 * h)
    _assert_same(a, b, sa, sb)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
def test_staged_matches_oracle(precision, tol):
    wl = W.curved_channel((6, 6, 6), 3, 5, P=600, nsteps=40, dt=2e-3, seed=1)
    _speed_up(wl, 1)
    h = 2.0 / 6
    band = (2e-4, 1e-4 * h) if precision == "fp32" else (1e-10, 1e-10)
    ctx = H.gpu_context(wl, precision, schedule=pt.SCHEDULE_STAGED, band_ref=band[0],
                        band_x=band[1])
    parts = H.gpu_particles(wl, ctx)
    st = ctx.push(parts, wl.nsteps, wl.dt)
    assert st["particle_steps"] == 600 * 40
    o = H.run_oracle(wl, band_ref=band[0], band_x=band[1])
    H.compare(H.gpu_result(parts), o, tol)


def test_staged_empty_frozen_and_lost_on_entry():
    wl = W.curved_channel((4, 4, 4), 2, 3, P=300, nsteps=5, dt=2e-3)
    for precision in ("fp64", "fp32"):
        ctx = H.gpu_context(wl, precision, schedule=pt.SCHEDULE_STAGED)
        parts = H.gpu_particles(wl, ctx)
        parts.status[:50] = pt.ST_LOST        # frozen on entry: untouched
        parts.elem[50:60] = wl.mesh.nelem + 3  # owner out of range: lost, position kept
        x0 = parts.x.clone()
        ctx.push(parts, 5, wl.dt, stats=False)
        torch.cuda.synchronize()
        assert torch.equal(parts.x[:, :60], x0[:, :60])
        assert bool((parts.status[50:60] & pt.ST_LOST).all())
        assert bool((parts.status[60:] & pt.ST_FROZEN == 0).all())
        empty = pt.ParticleSet.create(np.zeros((0, 3)), np.zeros((0, 3)), np.zeros(0),
                                      np.zeros(0, np.int32), ctx.precision, "cuda")
        assert ctx.push(empty, 3, wl.dt)["particle_steps"] == 0


def test_histograms_count_every_particle_stage():
    wl = W.curved_channel((6, 6, 6), 3, 5, P=3000, nsteps=10, dt=2e-3, seed=6)
    _speed_up(wl, 6)
    h = 2.0 / 6
    ctx = H.gpu_context(wl, "fp32", schedule=pt.SCHEDULE_STAGED, band_ref=2e-4, band_x=1e-4 * h)
    parts = H.gpu_particles(wl, ctx)
    st = ctx.push(parts, 10, wl.dt)
    hist = ctx.histograms()
    stages = 5 * st["particle_steps"]  # no particle froze
    assert sum(hist["newton_fp32"]) == stages and sum(hist["newton_final"]) == stages
    # the totals also hold the walk's inverse maps after a crossing
    assert sum(k * c for k, c in enumerate(hist["newton_fp32"])) <= st["newton_it_fp32"]
    assert sum(hist["crossings"]) == st["slow_track"]
    assert sum(k * c for k, c in enumerate(hist["crossings"][:3])) + 3 * hist["crossings"][3] \
        <= st["crossings"]
    print("histograms", hist)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_push_stage_sequence_equals_one_step_push(precision):
    """pt_push_stage(0..4) with an unchanged fluid state gives bitwise the
    result of pt_push(nsteps = 1) in the staged schedule; a fluid state that
    changes between stages changes the result; calls out of order and other
    pushes while a sequence is open are refused."""
    wl = W.curved_channel((6, 6, 6), 3, 5, P=2000, nsteps=1, dt=2e-3, seed=8)
    _speed_up(wl, 8)
    h = 2.0 / 6
    band = dict(band_ref=2e-4, band_x=1e-4 * h) if precision == "fp32" else {}
    ctx = H.gpu_context(wl, precision, schedule=pt.SCHEDULE_STAGED, **band)
    one = H.gpu_particles(wl, ctx)
    st1 = ctx.push(one, 1, wl.dt)
    stg = H.gpu_particles(wl, ctx)
    x0 = stg.x.clone()
    for s in range(5):
        st = ctx.push_stage(stg, s, wl.dt, stats=(s == 4))
        if s < 4:
            assert torch.equal(stg.x, x0)  # the caller's arrays change at stage 4
    torch.cuda.synchronize()
    a, b = H.gpu_result(one), H.gpu_result(stg)
    for k in FIELDS:
        assert np.array_equal(a[k], b[k]), k
    assert st["particle_steps"] == st1["particle_steps"] and st["crossings"] == st1["crossings"]
    # the fluid state read at every stage: scaling it after stage 2 changes the result
    ctx2 = H.gpu_context(wl, precision, schedule=pt.SCHEDULE_STAGED, **band)
    U = wl.U.to("cuda", torch.float64 if precision == "fp64" else torch.float32).contiguous()
    ctx2.set_fluid(wl.N, wl.node_type, U)
    chg = H.gpu_particles(wl, ctx2)
    for s in range(5):
        if s == 3:
            U[:, 1:4] *= 1.5  # in place: the registered array
        ctx2.push_stage(chg, s, wl.dt)
    torch.cuda.synchronize()
    assert not torch.equal(chg.v, stg.v)
    # order and exclusivity
    with pytest.raises(pt.PtError):
        ctx2.push_stage(chg, 2, wl.dt)
    ctx2.push_stage(chg, 0, wl.dt)
    with pytest.raises(pt.PtError):
        ctx2.push(chg, 1, wl.dt)
    with pytest.raises(pt.PtError):
        ctx2.deposit(chg, pt.DEPOSIT_ATOMIC)
    for s in range(1, 5):
        ctx2.push_stage(chg, s, wl.dt)
    ctx2.push(chg, 1, wl.dt)
