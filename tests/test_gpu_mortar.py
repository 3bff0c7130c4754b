"""GPU push on non-conforming meshes (Sec. 3.2.3: a big face matched to two or
four small faces) vs the FP64 oracle, particle by particle: element ids and
wall hits bit-exact outside the near-face band, x and v within 1e-12 (FP64)
or 2e-5 (FP32) relative."""
import numpy as np
import pytest
import torch

from paper_2211_05458_gb300 import pt
from paper_2211_05458_gb300 import workloads as W
from tests import helpers as H

pytestmark = pytest.mark.gpu

EA = 27  # elements of the coarse block (n = 3)


def _run(wl, precision, tol, band=None, **cfg):
    ctx = H.gpu_context(wl, precision, **cfg)
    parts = H.gpu_particles(wl, ctx)
    st = ctx.push(parts, wl.nsteps, wl.dt)
    torch.cuda.synchronize()
    g = H.gpu_result(parts)
    band_ref, band_x = (1e-10, 1e-10) if band is None else band
    o = H.run_oracle(wl, band_ref=band_ref, band_x=band_x)
    res = H.compare(g, o, tol)
    start = H.np64(wl.elem) < EA
    # both directions through the mortars were taken
    assert np.sum(start & (g["elem"] >= EA)) >= 5 and np.sum(~start & (g["elem"] < EA)) >= 5
    return res, st


@pytest.mark.parametrize("split,ngeo", [("st", 1), ("st", 2), ("st", 3), ("st", 4), ("s", 2),
                                        ("t", 3)])
def test_mortar_fp64_matches_oracle(split, ngeo):
    wl = W.mortar_tgv(3, ngeo, split, N=4, P=400, nsteps=40)
    res, st = _run(wl, "fp64", 1e-12)
    assert st["crossings"] > 100 and st["wall_hits"] >= 5


@pytest.mark.parametrize("split,ngeo", [("st", 3), ("s", 2)])
def test_mortar_fp32_matches_oracle(split, ngeo):
    wl = W.mortar_tgv(3, ngeo, split, N=4, P=400, nsteps=40)
    h = 1.0 / 6
    res, st = _run(wl, "fp32", 2e-5, band=(2e-4, 1e-4 * h), band_ref=2e-4, band_x=1e-4 * h)
    assert st["crossings"] > 100


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_mortar_reference_space_localisation(precision):
    """With PT_TRACK_REFERENCE the walk across a big face enters the small
    element whose part of the big face holds the point."""
    wl = W.mortar_tgv(3, 2, "st", N=4, P=400, nsteps=40)
    if precision == "fp64":
        _run(wl, "fp64", 1e-12, track=pt.TRACK_REFERENCE)
    else:
        h = 1.0 / 6
        _run(wl, "fp32", 2e-5, band=(2e-4, 1e-4 * h), band_ref=2e-4, band_x=1e-4 * h,
             track=pt.TRACK_REFERENCE)


def test_mortar_bezier_clipping_fp64():
    wl = W.mortar_tgv(3, 3, "st", N=4, P=300, nsteps=40)
    _run(wl, "fp64", 1e-12, curved_faces=1)


def test_mortar_deposit_and_locate_are_element_local():
    """Deposition and point location need no connectivity: on the mortar mesh
    the segmented deposition equals the oracle's and pt_find_element finds the
    brute-force owner."""
    wl = W.mortar_tgv(3, 2, "st", N=3, P=300, nsteps=1)
    ctx = H.gpu_context(wl, "fp64")
    parts = H.gpu_particles(wl, ctx)
    S = ctx.deposit(parts, pt.DEPOSIT_SEGMENTED).double().cpu().numpy().reshape(-1)
    orc = H.make_oracle(wl)
    So = orc.deposit(H.oracle_params(wl), H.np64(wl.x), H.np64(wl.v), H.np64(wl.d),
                     H.np64(wl.elem).astype(np.int32)).reshape(-1)
    scale = np.max(np.abs(So))
    assert np.max(np.abs(S - So)) <= 1e-5 * scale
    el, xi, stt = ctx.find_element(wl.x.T.contiguous().to("cuda"))
    assert torch.equal(el.cpu().to(torch.int32), wl.elem.cpu().to(torch.int32))


def _bad(md, **chg):
    md = {k: (v.copy() if hasattr(v, "copy") else v) for k, v in md.items()}
    for k, f in chg.items():
        f(md[k])
    with pytest.raises(pt.PtError) as ei:
        pt.Context(md, precision=pt.FP64)
    assert ei.value.code == pt.PT_ERR_ARG
    return str(ei.value)


def test_malformed_mortar_tables_are_rejected():
    md = W.mortar_box(2, 2, "st").as_dict()
    pt.Context(md, precision=pt.FP64)  # the well-formed mesh is accepted

    def set_(idx, val):
        def f(a):
            a[idx] = val
        return f

    _bad(md, mortar=set_((0, 0), 7))                  # unknown type
    _bad(md, mortar=set_((0, 0), W.MORTAR_S))          # 2 faces but 4 listed
    _bad(md, mortar=set_((0, 1), 0))                   # small face does not point back
    _bad(md, mortar=set_((0, 5), 3))                   # wrong local face
    big = int(np.flatnonzero(md["bc"][:, 1] == W.BC_MORTAR)[0])
    _bad(md, neighbor=set_((big, 1), 99))              # row out of range
    _bad(md, neighbor=set_((big, 1), (md["neighbor"][big, 1] + 1) % len(md["mortar"])))  # twice
    small = int(md["mortar"][0, 1])
    _bad(md, nbr_face=set_((small, 0), 2))             # small face names another big face
    md2 = dict(md)
    md2["mortar"] = md["mortar"][:-1]                  # a big face names a missing row
    with pytest.raises(pt.PtError):
        pt.Context(md2, precision=pt.FP64)
