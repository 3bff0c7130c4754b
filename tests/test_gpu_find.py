"""Point location without a known element (localisation in reference space,
Sec. 3.2.3) against the oracle's brute-force search: the owner is the unique
element containing the point, one of the elements that contain it on a shared
face, or -1 outside the mesh; xi equals the oracle's Newton result."""
import numpy as np
import pytest
import torch

import oracle
from paper_2211_05458_gb300 import pt
from paper_2211_05458_gb300 import workloads as W
from tests import helpers as H

pytestmark = pytest.mark.gpu


def _check(mesh, precision, pts, xi_tol):
    ctx = pt.Context(mesh, precision=pt.FP64 if precision == "fp64" else pt.FP32)
    x = torch.as_tensor(pts.T.copy()).cuda()
    elem, xi, st = ctx.find_element(x)
    elem, xi, st = elem.cpu().numpy(), xi.cpu().numpy().T, st.cpu().numpy()
    orc = oracle.Oracle(mesh.as_dict())
    p = oracle.make_params()
    n_unique = n_outside = 0
    for i in range(len(pts)):
        owners = list(orc.locate_bruteforce(pts[i], 1e-6, p))
        if not owners:
            assert elem[i] == -1 and st[i] == oracle.ST_LOST, (i, elem[i])
            n_outside += 1
            continue
        assert elem[i] in owners, (i, elem[i], owners)
        n_unique += len(owners) == 1
        ok, xo, _ = orc.newton(int(elem[i]), pts[i])
        assert ok and np.max(np.abs(xi[i] - xo)) < xi_tol
    return n_unique, n_outside


@pytest.mark.parametrize("precision,xi_tol", [("fp64", 1e-12), ("fp32", 2e-12)])
@pytest.mark.parametrize("ngeo", [1, 2, 3, 4])
def test_find_element_curved_channel(precision, xi_tol, ngeo):
    mesh = W.channel_mesh((6, 5, 4), ngeo)
    rng = np.random.default_rng(ngeo)
    pts = np.column_stack([rng.uniform(-0.2, 2 * np.pi + 0.2, 600), rng.uniform(-1.1, 1.1, 600),
                          rng.uniform(-0.1, np.pi + 0.1, 600)])
    n_unique, n_outside = _check(mesh, precision, pts, xi_tol)
    assert n_unique > 400 and n_outside > 20


def test_find_element_on_shared_nodes_and_faces():
    """Points exactly on element corners and faces of a straight lattice: any of
    the elements sharing them is a valid owner."""
    mesh = W.box_mesh((4, 4, 4), (0, 0, 0), (1, 1, 1), 1)
    g = np.linspace(0, 1, 9)
    pts = np.array([[a, b, c] for a in g for b in g for c in g[::2]])
    _check(mesh, "fp64", pts, 1e-12)
