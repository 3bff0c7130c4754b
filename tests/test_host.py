"""Host-side checks that need no GPU: the C-ABI library loads and exports
every entry point of include/pt.h, the workload generators are consistent and
seeded, and the multi-rank aggregation of bench.py (gloo, world size 2)."""
import ctypes
import os
import re
import socket

import numpy as np
import pytest
import torch

from paper_2211_05458_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "pt.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(pt_[a-z_0-9]+)\s*\(", txt)))


def test_library_exports_every_declared_entry_point():
    from paper_2211_05458_gb300 import build, pt
    so = build.build()
    lib = ctypes.CDLL(so)
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) <= set(pt.EXPORTS)


def test_binding_refuses_to_run_without_library(tmp_path, monkeypatch):
    from paper_2211_05458_gb300 import build, pt
    monkeypatch.setattr(build, "SO", str(tmp_path / "missing.so"))
    monkeypatch.setattr(pt, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        pt.lib()


@pytest.mark.parametrize("periodic", [(True, True, True), (True, False, True)])
def test_box_mesh_connectivity_is_symmetric(periodic):
    m = W.box_mesh((3, 4, 2), (0, 0, 0), (1, 2, 3), 2, periodic=periodic, warp="channel",
                   amp=0.1)
    for e in range(m.nelem):
        for f in range(6):
            nb, nf, bc = m.neighbor[e, f], m.nbr_face[e, f], m.bc[e, f]
            if bc in (W.BC_INTERNAL, W.BC_PERIODIC):
                assert m.neighbor[nb, nf] == e and m.nbr_face[nb, nf] == f
                assert np.allclose(m.shift[e, f], -m.shift[nb, nf])
            else:
                assert nb == -1
    # shared faces have bitwise identical nodes (internal faces)
    g = 3
    xg = m.xgeo.reshape(m.nelem, g, g, g, 3)  # [e][c][b][a]
    for e in range(m.nelem):
        nb = m.neighbor[e, 1]
        if m.bc[e, 1] == W.BC_INTERNAL:
            assert np.array_equal(xg[e, :, :, g - 1], xg[nb, :, :, 0])


@pytest.mark.parametrize("split", ["st", "s", "t"])
def test_mortar_box_connectivity(split):
    """Conforming faces point back; every big face names one mortar row whose
    small faces name the big face back; small faces cover the big face once."""
    m = W.mortar_box(3, 2, split)
    seen = np.zeros(len(m.mortar), int)
    for e in range(m.nelem):
        for f in range(6):
            nb, nf, bc = m.neighbor[e, f], m.nbr_face[e, f], m.bc[e, f]
            if bc == W.BC_MORTAR:
                seen[nb] += 1
                row = m.mortar[nb]
                ns = 4 if row[0] == W.MORTAR_FOUR else 2
                assert np.all(row[1 + ns:5] == -1) and np.all(row[5 + ns:9] == -1)
                for q in range(ns):
                    es, fs = row[1 + q], row[5 + q]
                    assert m.bc[es, fs] == W.BC_INTERNAL
                    assert m.neighbor[es, fs] == e and m.nbr_face[es, fs] == f
            elif bc == W.BC_INTERNAL and m.bc[nb, nf] == W.BC_MORTAR:
                row = m.mortar[m.neighbor[nb, nf]]
                assert any(row[1 + q] == e and row[5 + q] == f for q in range(4))
            elif bc == W.BC_INTERNAL:
                assert m.neighbor[nb, nf] == e and m.nbr_face[nb, nf] == f
            else:
                assert nb == -1
    assert np.all(seen == 1)
    # every small face is listed exactly once: 4 or 2 per row
    ns = 4 if split == "st" else 2
    n_small = sum(1 for e in range(m.nelem) for f in range(6)
                  if m.bc[e, f] == W.BC_INTERNAL
                  and m.bc[m.neighbor[e, f], m.nbr_face[e, f]] == W.BC_MORTAR)
    assert n_small == len(m.mortar) * ns
    listed = m.mortar[:, 1:1 + ns].ravel()
    assert len(np.unique(listed)) == len(listed)


def test_workloads_are_seeded():
    a = W.curved_channel((4, 4, 4), 2, 3, P=100, nsteps=1, seed=3)
    b = W.curved_channel((4, 4, 4), 2, 3, P=100, nsteps=1, seed=3)
    c = W.curved_channel((4, 4, 4), 2, 3, P=100, nsteps=1, seed=4)
    assert torch.equal(a.x, b.x) and torch.equal(a.U, b.U) and torch.equal(a.d, b.d)
    assert not torch.equal(a.x, c.x)
    # Stokes numbers log-uniform in [0.1, 100]: tau = St (U = L = 1)
    tau = a.rho_p * a.d ** 2 / (18 * a.mu)
    assert float(tau.min()) >= 0.1 - 1e-12 and float(tau.max()) <= 100 + 1e-9


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, q):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = bench.reduce_time_ms(100.0 + 50.0 * rank, world)
    v = bench.throughput(1000, 10, 5, world, ms)
    p_all = bench.sum_over_ranks(1000.0 + 2000.0 * rank, world)
    q.put((rank, ms, v, p_all))
    dist.destroy_process_group()


def test_weak_scaling_aggregation_two_ranks_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, v, p_all in out:
        assert ms == 150.0  # max over ranks
        assert abs(v - 1000 * 10 * 5 * 2 / 0.15) < 1e-6 * v
        assert p_all == 4000.0  # particles of both ranks (uneven, as with the batched boxes)


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_batched_boxes_shard_by_cost(world):
    """The 128 boxes split over ranks: each box once, loads within one box's
    cost of each other, the same split on every rank, and a rank's boxes the
    same as in the unsplit set."""
    import bench
    prm = W.batched_box_params(nbox=128, seed=1)
    costs = [P * (N + 1) ** 3 for _, N, P in prm]
    parts = bench.shard_by_cost(costs, world)
    assert sorted(i for p in parts for i in p) == list(range(128))
    loads = [sum(costs[i] for i in p) for p in parts]
    assert max(loads) - min(loads) <= max(costs)
    assert parts == bench.shard_by_cost(costs, world)
    sel = parts[-1][:2]
    a = W.batched_boxes(nbox=128, seed=1, select=sel, scale_P=1e-3)
    for b, wl in zip(sel, a):
        side, N, P = W.batched_box_params(nbox=128, seed=1, scale_P=1e-3)[b]
        assert wl.mesh.dims == (side,) * 3 and wl.N == N and wl.x.shape[0] == P


def test_particle_set_never_aliases_its_inputs():
    from paper_2211_05458_gb300 import pt
    x = torch.rand(5, 3, dtype=torch.float64)
    v = torch.rand(5, 3, dtype=torch.float32)
    d = torch.rand(5, dtype=torch.float32)
    el = torch.arange(5, dtype=torch.int32)
    ps = pt.ParticleSet.create(x, v, d, el, pt.FP32, "cpu")
    ps.elem[0] = 99
    ps.d[0] = -1.0
    assert int(el[0]) == 0 and float(d[0]) >= 0.0


def _init_rc(md):
    """pt_init_mesh on a mesh description; returns (status, message).
    Malformed meshes are rejected before any device call; a well-formed one
    gets as far as the device allocation (PT_ERR_CUDA without a GPU; with one
    the context is created and destroyed again)."""
    from paper_2211_05458_gb300 import build, pt
    build.build()
    L = pt.lib()
    keep = {k: np.ascontiguousarray(md[k], dtype=np.float64 if k in ("xgeo", "shift")
                                    else np.int32)
            for k in ("xgeo", "neighbor", "nbr_face", "bc", "shift", "mortar")}
    d = pt.MeshDesc()
    d.nelem, d.ngeo = int(md["nelem"]), int(md["ngeo"])
    for k in ("xgeo", "neighbor", "nbr_face", "bc", "shift"):
        setattr(d, k, keep[k].ctypes.data)
    d.nmortar = len(keep["mortar"])
    d.mortar = keep["mortar"].ctypes.data if len(keep["mortar"]) else None
    cfg = pt.default_config()
    h = ctypes.c_void_p()
    rc = L.pt_init_mesh(ctypes.byref(h), ctypes.byref(d), ctypes.byref(cfg), None)
    msg = L.pt_last_error(None).decode()
    if h.value:
        assert rc == pt.PT_OK
        L.pt_destroy(h)
    return rc, msg


def _edit(md, key, idx, val):
    out = {k: (v.copy() if hasattr(v, "copy") else v) for k, v in md.items()}
    out[key][idx] = val
    return out


def test_mesh_validation_rejects_malformed_connectivity():
    """Host-side checks of pt_init_mesh (conforming and mortar connectivity,
    boundary kinds, shifts), each with its own message."""
    from paper_2211_05458_gb300 import pt
    md = W.mortar_box(2, 2, "st").as_dict()
    big = int(np.flatnonzero(md["bc"][:, 1] == W.BC_MORTAR)[0])
    small = int(md["mortar"][0, 1])
    cases = [
        (_edit(md, "mortar", (0, 0), 7), "bad type"),
        (_edit(md, "mortar", (0, 0), W.MORTAR_S), "must be unused"),
        (_edit(md, "mortar", (0, 1), 0), "not a small face"),
        (_edit(md, "mortar", (0, 5), 3), "not a small face"),
        (_edit(md, "neighbor", (big, 1), 99), "bad mortar row"),
        (_edit(md, "neighbor", (big, 1), (md["neighbor"][big, 1] + 1) % len(md["mortar"])),
         "referenced twice"),
        (_edit(md, "nbr_face", (small, 0), 2), "does not point back"),
        (_edit(md, "bc", (0, 0), 5), "bad bc"),
        (_edit(md, "shift", (0, 0, 0), 1.0), "shift on a non-periodic face"),
        (dict(md, mortar=md["mortar"][:-1]), "bad mortar row"),
        (dict(md, ngeo=5), "ngeo"),
    ]
    box = W.box_mesh((3, 3, 3), (0, 0, 0), (1, 1, 1), 1).as_dict()
    cases.append((_edit(box, "neighbor", (0, 1), 5), "does not point back"))
    for mdx, msg in cases:
        rc, err = _init_rc(mdx)
        assert rc == pt.PT_ERR_ARG, (msg, rc, err)
        assert msg in err, (msg, err)
    # the well-formed meshes pass every host check
    for mdx in (md, box, W.mortar_box(2, 3, "s").as_dict(), W.mortar_box(2, 1, "t").as_dict()):
        rc, err = _init_rc(mdx)
        assert rc in (pt.PT_OK, pt.PT_ERR_CUDA), (rc, err)


def test_channel_flow_generator_properties():
    """The synthetic channel turbulence is divergence-free (curl of a vector
    potential), vanishes on the walls y = +-1, is periodic over [0, 2pi] x
    [0, pi] in x and z, and its perturbation has the requested rms."""
    g = torch.Generator().manual_seed(3)
    n = 4000
    x = torch.rand(n, generator=g, dtype=torch.float64) * 2 * np.pi
    y = torch.rand(n, generator=g, dtype=torch.float64) * 1.8 - 0.9
    z = torch.rand(n, generator=g, dtype=torch.float64) * np.pi
    u, v, w, scale = W.channel_velocity(x, y, z, seed=5)
    pert = torch.stack([u - (1 - y * y), v, w])
    assert abs(float(torch.sqrt((pert ** 2).mean())) - 0.1) < 0.02
    h = 1e-5

    def vel(dx, dy, dz):
        return W.channel_velocity(x + dx, y + dy, z + dz, seed=5, scale=scale)[:3]
    div = ((vel(h, 0, 0)[0] - vel(-h, 0, 0)[0]) + (vel(0, h, 0)[1] - vel(0, -h, 0)[1]) +
           (vel(0, 0, h)[2] - vel(0, 0, -h)[2])) / (2 * h)
    assert float(div.abs().max()) < 1e-7
    for yw in (-1.0, 1.0):
        uw = W.channel_velocity(x, torch.full_like(x, yw), z, seed=5, scale=scale)[:3]
        assert max(float(c.abs().max()) for c in uw) < 1e-14
    ux = W.channel_velocity(x + 2 * np.pi, y, z + np.pi, seed=5, scale=scale)[:3]
    u0 = W.channel_velocity(x, y, z, seed=5, scale=scale)[:3]
    assert max(float((a - b).abs().max()) for a, b in zip(ux, u0)) < 1e-12


def test_ctypes_layouts_match_the_header(tmp_path):
    """The binding's ctypes structures have the sizes and field offsets that a
    C compiler gives the structs of include/pt.h."""
    import shutil
    import subprocess
    from paper_2211_05458_gb300 import pt
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    pairs = [("pt_config", pt.Config), ("pt_mesh_desc", pt.MeshDesc),
             ("pt_particles", pt.CParticles), ("pt_stats", pt.Stats),
             ("pt_histograms", pt.Histograms)]
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "pt.h"', "int main(void) {"]
    for cname, cls in pairs:
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True,
                               text=True).stdout.splitlines():
        *key, val = line.split()
        got[tuple(key)] = int(val)
    for cname, cls in pairs:
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert got[(cname, fname)] == getattr(cls, fname).offset, (cname, fname)
