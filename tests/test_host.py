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
    q.put((rank, ms, v))
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
    for rank, ms, v in out:
        assert ms == 150.0  # max over ranks
        assert abs(v - 1000 * 10 * 5 * 2 / 0.15) < 1e-6 * v


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
