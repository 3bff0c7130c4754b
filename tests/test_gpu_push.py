"""GPU push vs the FP64 oracle, particle by particle (element ids and wall hits
bit-exact outside the 1e-10 near-face band; x, v within 1e-12 relative in FP64
mode and 2e-5 in FP32 mode)."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2211_05458_gb300 import pt
from paper_2211_05458_gb300 import workloads as W
from tests import helpers as H

pytestmark = pytest.mark.gpu


def _speed_up(wl, seed=0):
    # faster particles so that faces and walls are crossed within few steps
    rng = np.random.default_rng(seed)
    wl.v = wl.v * 4.0 + torch.as_tensor(rng.normal(size=tuple(wl.v.shape)) * 1.5)


def _push_and_compare(wl, precision, tol, band=None, idx=None, **cfg):
    ctx = H.gpu_context(wl, precision, **cfg)
    parts = H.gpu_particles(wl, ctx, idx)
    st = ctx.push(parts, wl.nsteps, wl.dt)
    torch.cuda.synchronize()
    g = H.gpu_result(parts)
    band_ref, band_x = (1e-10, 1e-10) if band is None else band
    o = H.run_oracle(wl, idx, band_ref=band_ref, band_x=band_x)
    res = H.compare(g, o, tol)
    res["stats"] = st
    return res, g, o


def test_tgv_box_fp64_matches_oracle():
    """8^3 periodic cube, N=3 Gauss, TGV, Stokes drag, particles at rest."""
    wl = W.tgv_box(8, 3, P=2000, nsteps=100)
    res, g, o = _push_and_compare(wl, "fp64", 1e-12)
    assert res["stats"]["crossings"] > 100


def test_tgv_box_full_config_fp64():
    """The full small workload: 10^4 particles, 100 steps."""
    wl = W.tgv_box(8, 3, P=10_000, nsteps=100)
    res, g, o = _push_and_compare(wl, "fp64", 1e-12)
    assert res["checked"] >= 9900


@pytest.mark.parametrize("ngeo,N", [(2, 5), (3, 5), (1, 4), (2, 7), (4, 5)])
def test_curved_channel_fp64_matches_oracle(ngeo, N):
    wl = W.curved_channel((6, 6, 6), ngeo, N, P=400, nsteps=40, dt=2e-3, st=(0.1, 100.0))
    _speed_up(wl)
    res, g, o = _push_and_compare(wl, "fp64", 1e-12)
    assert res["stats"]["crossings"] > 50
    assert res["stats"]["wall_hits"] >= 1


@pytest.mark.parametrize("ngeo,N", [(2, 5), (3, 5), (4, 5)])
def test_curved_channel_fp32_matches_oracle(ngeo, N):
    wl = W.curved_channel((6, 6, 6), ngeo, N, P=400, nsteps=40, dt=2e-3)
    _speed_up(wl)
    # FP32 mode: positions drift ~1e-7; the near-face band is 1e-4 h
    h = 2.0 / 6
    res, g, o = _push_and_compare(wl, "fp32", 2e-5, band=(2e-4, 1e-4 * h), band_ref=2e-4,
                                  band_x=1e-4 * h)
    assert res["checked"] > 300


def test_walls_reflect_with_curved_walls_fp64():
    mesh = W.channel_mesh((5, 4, 4), 2, amp=0.1, curved_walls=True)
    wl = W.curved_channel((5, 4, 4), 2, 3, P=300, nsteps=30, dt=5e-3)
    wl.mesh = mesh
    U, _ = W.fluid_channel(mesh, 3, 0, seed=0)
    wl.U = U
    x, el = W.seed_particles(mesh, 300, seed=3)
    wl.x, wl.elem = x, el
    rng = np.random.default_rng(0)
    wl.v = torch.as_tensor(rng.normal(size=(300, 3)) * 3.0)
    wl.d = torch.full((300,), 4e-3, dtype=torch.float64)
    res, g, o = _push_and_compare(wl, "fp64", 1e-12)
    assert res["stats"]["wall_hits"] > 20


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_locate_matches_oracle_newton(precision):
    mesh = W.channel_mesh((6, 5, 4), 3, amp=0.15)
    wl = W.curved_channel((6, 5, 4), 3, 3, P=3000, nsteps=1)
    wl.mesh = mesh
    x, el = W.seed_particles(mesh, 3000, seed=21, margin=0.0)
    ctx = H.gpu_context(wl, precision)
    xi, it, st = ctx.locate(x.T.contiguous().cuda(), el.cuda())
    xi = xi.T.cpu().numpy()
    assert int((st != 0).sum()) == 0
    orc = oracle.Oracle(mesh.as_dict())
    for i in range(0, 3000, 7):
        ok, xo, _ = orc.newton(int(el[i]), H.np64(x[i]))
        assert ok
        assert np.max(np.abs(xi[i] - xo)) < 2e-12


def test_empty_and_frozen_particles():
    wl = W.tgv_box(4, 2, P=64, nsteps=3)
    ctx = H.gpu_context(wl, "fp64")
    from paper_2211_05458_gb300 import pt
    empty = pt.ParticleSet.create(torch.zeros((0, 3)), torch.zeros((0, 3)), torch.zeros(0),
                                  torch.zeros(0, dtype=torch.int32), pt.FP64, "cuda")
    st = ctx.push(empty, 5, 1e-3)
    assert st["particle_steps"] == 0
    parts = H.gpu_particles(wl, ctx)
    parts.status[:10] = pt.ST_LOST
    parts.elem[10] = 10 ** 6  # invalid owner -> lost, frozen
    x0 = parts.x.clone()
    st = ctx.push(parts, 3, 1e-3)
    assert st["status_code"] == pt.PT_ERR_LOST
    assert torch.equal(parts.x[:, :11], x0[:, :11])
    assert st["particle_steps"] == 3 * (64 - 11)


def test_fault_injection_caps_are_reported():
    """Host-side fault injection: a Newton cap of 1 and a crossing cap of 1
    freeze the affected particles and return error codes (no device fault)."""
    from paper_2211_05458_gb300 import pt
    wl = W.curved_channel((5, 5, 5), 2, 3, P=200, nsteps=20, dt=5e-3)
    wl.v = wl.v * 5
    ctx = H.gpu_context(wl, "fp64", max_newton=1)
    parts = H.gpu_particles(wl, ctx)
    st = ctx.push(parts, wl.nsteps, wl.dt)
    assert st["status_code"] == pt.PT_ERR_NEWTON and st["newton_fail"] == 200
    ctx = H.gpu_context(wl, "fp64", max_cross=1)
    parts = H.gpu_particles(wl, ctx)
    st = ctx.push(parts, wl.nsteps, wl.dt)
    assert st["cross_cap"] >= 0 and st["status_code"] in (pt.PT_OK, pt.PT_ERR_CROSS)


def test_bad_arguments_are_rejected():
    from paper_2211_05458_gb300 import pt
    wl = W.tgv_box(3, 2, P=10, nsteps=1)
    md = wl.mesh.as_dict()
    md["neighbor"] = md["neighbor"].copy()
    md["neighbor"][0, 1] = 5  # does not point back
    with pytest.raises(pt.PtError) as ei:
        pt.Context(md, precision=pt.FP64)
    assert ei.value.code == pt.PT_ERR_ARG
    ctx = H.gpu_context(wl, "fp64")
    parts = H.gpu_particles(wl, ctx)
    with pytest.raises(pt.PtError):
        ctx.push(parts, 1, -1.0)
    with pytest.raises(pt.PtError):
        ctx.push(parts, 1, float("nan"))


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
@pytest.mark.parametrize("ngeo,N", [(2, 5), (3, 5)])
def test_reference_space_localisation_matches_physical_oracle(precision, tol, ngeo, N):
    """Sec. 3.2.3: with PT_TRACK_REFERENCE only walls are intersected; internal
    and periodic crossings are found by the inverse map and the face walk.  The
    owners, wall hits and states equal the oracle's physical tracking."""
    wl = W.curved_channel((6, 6, 6), ngeo, N, P=400, nsteps=40, dt=2e-3, st=(0.1, 100.0))
    _speed_up(wl)
    band = None if precision == "fp64" else (2e-4, 1e-4 * 2.0 / 6)
    res, g, o = _push_and_compare(wl, precision, tol, band=band, track=pt.TRACK_REFERENCE)
    assert res["stats"]["crossings"] > 50 and res["stats"]["wall_hits"] >= 1


def test_reference_space_localisation_periodic_box():
    wl = W.tgv_box(8, 3, P=2000, nsteps=100)
    res, g, o = _push_and_compare(wl, "fp64", 1e-12, track=pt.TRACK_REFERENCE)
    assert res["stats"]["crossings"] > 100 and res["stats"]["slow_track"] == 0


@pytest.mark.parametrize("ngeo", [2, 3, 4])
def test_bezier_clipping_for_every_curved_face_fp64(ngeo):
    """Sec. 3.2.4: with curved_faces = 1 every curved face is intersected by
    Bezier clipping; owners, wall hits and states equal the oracle's (Bezier
    subdivision), positions within 1e-12."""
    wl = W.curved_channel((6, 6, 6), ngeo, 5, P=300, nsteps=30, dt=2e-3, st=(0.1, 100.0))
    _speed_up(wl)
    res, g, o = _push_and_compare(wl, "fp64", 1e-12, curved_faces=1)
    assert res["stats"]["crossings"] > 50


def test_bezier_clipping_fp32():
    wl = W.curved_channel((6, 6, 6), 3, 5, P=300, nsteps=30, dt=2e-3, st=(0.1, 100.0))
    _speed_up(wl)
    h = 2.0 / 6
    res, g, o = _push_and_compare(wl, "fp32", 2e-5, band=(2e-4, 1e-4 * h), band_ref=2e-4,
                                  band_x=1e-4 * h, curved_faces=1)
    assert res["stats"]["crossings"] > 50


def test_bezier_clipping_on_curved_walls_fp64():
    mesh = W.channel_mesh((5, 4, 4), 2, amp=0.1, curved_walls=True)
    wl = W.curved_channel((5, 4, 4), 2, 3, P=300, nsteps=30, dt=5e-3)
    wl.mesh = mesh
    U, _ = W.fluid_channel(mesh, 3, 0, seed=0)
    wl.U = U
    x, el = W.seed_particles(mesh, 300, seed=3)
    wl.x, wl.elem = x, el
    rng = np.random.default_rng(0)
    wl.v = torch.as_tensor(rng.normal(size=(300, 3)) * 3.0)
    wl.d = torch.full((300,), 4e-3, dtype=torch.float64)
    res, g, o = _push_and_compare(wl, "fp64", 1e-12, curved_faces=1)
    assert res["stats"]["wall_hits"] > 20


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_split_call_resume(precision):
    """A push of 10 steps equals a push of 5 steps followed by another of 5
    (the particle state between calls is x, v, elem, hits, status: restartable
    as the paper's restart files are).  FP64 mode: bitwise.  FP32 mode: inside a
    call the position is a double-float offset from the element centre; at a
    call boundary it becomes an FP64 position and back, a rounding of ~1e-16
    relative that can change the FP32 rounding of a later xi; owners and hits
    stay exact, x and v agree far inside the FP32 tolerance."""
    wl = W.curved_channel((6, 6, 6), 2, 5, P=2000, nsteps=10, dt=2e-3, seed=7)
    _speed_up(wl, seed=7)
    h = 2.0 / 6
    band = dict(band_ref=2e-4, band_x=1e-4 * h) if precision == "fp32" else {}
    ctx = H.gpu_context(wl, precision, **band)
    one = H.gpu_particles(wl, ctx)
    two = H.gpu_particles(wl, ctx)
    st1 = ctx.push(one, 10, wl.dt)
    ctx.push(two, 5, wl.dt)
    ctx.push(two, 5, wl.dt)
    torch.cuda.synchronize()
    assert st1["crossings"] > 100 and st1["wall_hits"] > 5
    a, b = H.gpu_result(one), H.gpu_result(two)
    if precision == "fp64":
        for k in ("x", "v", "elem", "hits", "status"):
            assert np.array_equal(a[k], b[k]), k
    else:
        near = ((a["status"] | b["status"]) & (pt.ST_NEAR_WALL | pt.ST_FROZEN)) != 0
        assert near.mean() < 0.05
        assert np.array_equal(a["elem"][~near], b["elem"][~near])
        assert np.array_equal(a["hits"][~near], b["hits"][~near])
        ex = np.abs(a["x"] - b["x"]) / np.maximum(np.abs(a["x"]), 1.0)
        ev = np.abs(a["v"] - b["v"]) / np.maximum(np.abs(a["v"]), 1.0)
        print("FP32 call boundary: max rel dx %.2e dv %.2e" % (ex[~near].max(), ev[~near].max()))
        assert ex[~near].max() <= 1e-9 and ev[~near].max() <= 1e-6


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("schedule", [pt.SCHEDULE_RESIDENT, pt.SCHEDULE_STAGED])
def test_push_host_equals_device_push(precision, schedule):
    """pt_push_host (host arrays staged through device buffers and copied
    back) gives bitwise the device push, from pinned and from pageable host
    memory."""
    wl = W.curved_channel((6, 6, 6), 2, 5, P=3000, nsteps=4, dt=2e-3, seed=11)
    _speed_up(wl, seed=11)
    h = 2.0 / 6
    band = dict(band_ref=2e-4, band_x=1e-4 * h) if precision == "fp32" else {}
    ctx = H.gpu_context(wl, precision, schedule=schedule, **band)
    dev = H.gpu_particles(wl, ctx)
    st_dev = ctx.push(dev, 4, wl.dt)
    torch.cuda.synchronize()
    ref = H.gpu_result(dev)
    assert st_dev["crossings"] > 50
    for pin in (True, False):
        hp = H.gpu_particles(wl, ctx).to("cpu", pin=pin)
        st = ctx.push_host(hp, 4, wl.dt)
        got = H.gpu_result(hp)
        for k in ("x", "v", "elem", "hits", "status"):
            assert np.array_equal(ref[k], got[k]), (pin, k)
        for k, val in st.items():
            assert st_dev[k] == val, (pin, k)
