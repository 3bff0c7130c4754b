"""Plain FP64 CPU oracle for the per-particle push (arXiv 2211.05458).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the product path
(``paper_2211_05458_gb300``) never does.  It shares no code with the CUDA
library: ``oracle.c`` is compiled here with gcc and driven through ctypes.

Every routine restates the paper directly (see ``oracle.h`` for the section
and equation each one follows).  Functions without an independent pin are
listed in the module docstring of ``tests/test_oracle.py``; none is left
"parity unpinned".  The 48 geometry features are pinned by closed forms on
affine and on quadratically warped elements.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = [os.path.join(_HERE, "oracle.c")]
_lock = threading.Lock()
_lib = None

ST_NEWTON_FAIL = 1 << 0
ST_LOST = 1 << 1
ST_CROSS_CAP = 1 << 2
ST_NEAR_FACE = 1 << 3
ST_REP800 = 1 << 4
ST_OPEN = 1 << 5
ST_NEAR_WALL = 1 << 6
ST_FROZEN = ST_NEWTON_FAIL | ST_LOST | ST_CROSS_CAP | ST_OPEN


def build(force: bool = False) -> str:
    """Compile oracle.c into _build/liboracle.so (IEEE FP64, no contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(p) for p in _SRC + [os.path.join(_HERE, "oracle.h")])
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < newest:
        tmp = _SO + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", *_SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


class Params(ctypes.Structure):
    _fields_ = [
        ("mu", ctypes.c_double), ("rho_p", ctypes.c_double),
        ("drag_law", ctypes.c_int), ("max_newton", ctypes.c_int),
        ("g", ctypes.c_double * 3), ("mask", ctypes.c_double * 3),
        ("max_cross", ctypes.c_int), ("pad", ctypes.c_int),
        ("newton_tol", ctypes.c_double), ("band_ref", ctypes.c_double),
        ("band_x", ctypes.c_double), ("lost_tol", ctypes.c_double),
        ("lift", ctypes.c_int), ("buoyancy", ctypes.c_int), ("sphericity", ctypes.c_double),
    ]


def make_params(mu=1e-5, rho_p=1000.0, drag_law=0, g=(0.0, 0.0, 0.0), mask=(1.0, 1.0, 1.0),
                max_newton=50, max_cross=64, newton_tol=1e-12, band_ref=1e-10, band_x=1e-10,
                lost_tol=1e-6, lift=0, sphericity=1.0, buoyancy=0) -> Params:
    p = Params()
    p.lift, p.sphericity, p.buoyancy = lift, sphericity, buoyancy
    p.mu, p.rho_p, p.drag_law, p.max_newton = mu, rho_p, drag_law, max_newton
    p.g[:] = list(g)
    p.mask[:] = list(mask)
    p.max_cross, p.newton_tol = max_cross, newton_tol
    p.band_ref, p.band_x, p.lost_tol = band_ref, band_x, lost_tol
    return p


_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int32)
_U = ctypes.POINTER(ctypes.c_uint32)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            vp = ctypes.c_void_p
            L.or_create.restype = vp
            L.or_create.argtypes = [ctypes.c_int, ctypes.c_int, _D, _I, _I, _I, _D]
            L.or_destroy.argtypes = [vp]
            L.or_set_mortars.argtypes = [vp, ctypes.c_int, _I]
            L.or_set_fluid.argtypes = [vp, ctypes.c_int, ctypes.c_int, _D]
            L.or_nodes.argtypes = [ctypes.c_int, ctypes.c_int, _D]
            L.or_lagrange.restype = ctypes.c_double
            L.or_lagrange.argtypes = [ctypes.c_int, _D, ctypes.c_int, ctypes.c_double]
            L.or_lagrange_deriv.restype = ctypes.c_double
            L.or_lagrange_deriv.argtypes = [ctypes.c_int, _D, ctypes.c_int, ctypes.c_double]
            L.or_elem_map.argtypes = [vp, ctypes.c_int, _D, _D, _D]
            L.or_newton.argtypes = [vp, ctypes.POINTER(Params), ctypes.c_int, _D, _D,
                                    ctypes.POINTER(ctypes.c_int)]
            L.or_interp.argtypes = [vp, ctypes.c_int, _D, _D]
            L.or_interp_grad.argtypes = [vp, ctypes.c_int, _D, _D, _D]
            L.or_velocity_gradient.argtypes = [vp, ctypes.c_int, _D, _D]
            L.or_drag_factor.restype = ctypes.c_double
            L.or_drag_factor.argtypes = [ctypes.POINTER(Params), ctypes.c_double]
            L.or_saffman_force.argtypes = [ctypes.POINTER(Params), ctypes.c_double, _D, _D,
                                           ctypes.c_double, _D]
            L.or_face_hits.argtypes = [vp, ctypes.c_int, ctypes.c_int, _D, _D, ctypes.c_double,
                                       _D, ctypes.c_int]
            L.or_face_ctrl.argtypes = [vp, ctypes.c_int, ctypes.c_int, _D]
            L.or_locate_bruteforce.argtypes = [vp, ctypes.POINTER(Params), _D, ctypes.c_double,
                                               _I, ctypes.c_int]
            L.or_push.argtypes = [vp, ctypes.POINTER(Params), ctypes.c_int64, _D, _D, _D, _I, _I,
                                  _U, ctypes.c_int, ctypes.c_double]
            L.or_stage1.restype = ctypes.c_int
            L.or_stage1.argtypes = [vp, ctypes.POINTER(Params), ctypes.c_int, _D, _D,
                                    ctypes.c_double, ctypes.c_double, _D]
            L.or_deposit.argtypes = [vp, ctypes.POINTER(Params), ctypes.c_int64, _D, _D, _D, _I,
                                     _U, _D]
            L.or_lserk_coeffs.argtypes = [_D, _D, _D]
            L.or_quad_weights.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D]
            L.or_deposit_nearest.argtypes = L.or_deposit.argtypes
            L.or_dt_violations.restype = ctypes.c_int64
            L.or_dt_violations.argtypes = [ctypes.POINTER(Params), ctypes.c_int64, _D,
                                           ctypes.c_double]
            L.or_mlp_features.argtypes = [vp, ctypes.c_int, _D, _D]
            L.or_mlp_forward.argtypes = [_D, ctypes.c_int, _D, _D]
            L.or_mlp_loss_grad.restype = ctypes.c_double
            L.or_mlp_loss_grad.argtypes = [_D, ctypes.c_int, _D, _D, _D]
            L.or_adam.argtypes = [ctypes.c_int, _D, _D, _D, _D, ctypes.c_int, ctypes.c_double,
                                  ctypes.c_double, ctypes.c_double, ctypes.c_double]
            L.or_mlp_nparams.restype = ctypes.c_int
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(_D)


def _ip(a):
    return a.ctypes.data_as(_I)


def _up(a):
    return a.ctypes.data_as(_U)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def nodes(kind: int, n: int) -> np.ndarray:
    out = np.zeros(n)
    lib().or_nodes(kind, n, _dp(out))
    return out


def lagrange(xn, i, x) -> float:
    xn = _f64(xn)
    return lib().or_lagrange(len(xn), _dp(xn), i, float(x))


def lagrange_deriv(xn, i, x) -> float:
    xn = _f64(xn)
    return lib().or_lagrange_deriv(len(xn), _dp(xn), i, float(x))


def quad_weights(kind: int, n: int) -> np.ndarray:
    x = nodes(kind, n)
    w = np.zeros(n)
    lib().or_quad_weights(kind, n, _dp(x), _dp(w))
    return w


def dt_violations(params: Params, d, dt: float) -> int:
    d = _f64(d)
    return int(lib().or_dt_violations(ctypes.byref(params), len(d), _dp(d), float(dt)))


def drag_factor(params: Params, re: float) -> float:
    return float(lib().or_drag_factor(ctypes.byref(params), float(re)))


def saffman_force(params: Params, rho, rel, omega, d):
    F = np.zeros(3)
    lib().or_saffman_force(ctypes.byref(params), float(rho), _dp(_f64(rel)), _dp(_f64(omega)),
                           float(d), _dp(F))
    return F


def lserk_coeffs():
    A, B, C = np.zeros(5), np.zeros(5), np.zeros(5)
    lib().or_lserk_coeffs(_dp(A), _dp(B), _dp(C))
    return A, B, C


class Oracle:
    """One mesh (+ optionally one fluid state) held by the C oracle."""

    def __init__(self, mesh: dict):
        L = lib()
        self._keep = dict(xgeo=_f64(mesh["xgeo"]), neighbor=_i32(mesh["neighbor"]),
                          nbr_face=_i32(mesh["nbr_face"]), bc=_i32(mesh["bc"]),
                          shift=_f64(mesh["shift"]))
        k = self._keep
        self.nelem = int(mesh["nelem"])
        self.ngeo = int(mesh["ngeo"])
        self.h = L.or_create(self.nelem, self.ngeo, _dp(k["xgeo"]), _ip(k["neighbor"]),
                             _ip(k["nbr_face"]), _ip(k["bc"]), _dp(k["shift"]))
        if not self.h:
            raise ValueError("oracle: bad mesh")
        mortar = mesh.get("mortar")
        if mortar is not None and len(mortar):
            self._keep["mortar"] = _i32(mortar)
            if not L.or_set_mortars(self.h, len(mortar), _ip(self._keep["mortar"])):
                raise ValueError("oracle: bad mortar table")
        self.N = None

    def close(self):
        if self.h:
            lib().or_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_fluid(self, N: int, node_type: int, U: np.ndarray):
        U = _f64(U)
        assert U.size == self.nelem * 5 * (N + 1) ** 3
        if not lib().or_set_fluid(self.h, N, node_type, _dp(U)):
            raise ValueError("oracle: bad fluid")
        self.N = N

    def elem_map(self, e, xi):
        xi = _f64(xi)
        x, J = np.zeros(3), np.zeros(9)
        lib().or_elem_map(self.h, int(e), _dp(xi), _dp(x), _dp(J))
        return x, J.reshape(3, 3)

    def newton(self, e, x, params: Params | None = None):
        params = params or make_params()
        x = _f64(x)
        xi = np.zeros(3)
        it = ctypes.c_int(0)
        ok = lib().or_newton(self.h, ctypes.byref(params), int(e), _dp(x), _dp(xi),
                             ctypes.byref(it))
        return bool(ok), xi, it.value

    def interp(self, e, xi):
        xi = _f64(xi)
        U = np.zeros(5)
        lib().or_interp(self.h, int(e), _dp(xi), _dp(U))
        return U

    def interp_grad(self, e, xi):
        xi = _f64(xi)
        U, dU = np.zeros(5), np.zeros(15)
        lib().or_interp_grad(self.h, int(e), _dp(xi), _dp(U), _dp(dU))
        return U, dU.reshape(5, 3)

    def velocity_gradient(self, e, xi):
        G = np.zeros(9)
        lib().or_velocity_gradient(self.h, int(e), _dp(_f64(xi)), _dp(G))
        return G.reshape(3, 3)

    def face_hits(self, e, f, x0, x1, band=0.0):
        out = np.zeros(3 * 16)
        n = lib().or_face_hits(self.h, int(e), int(f), _dp(_f64(x0)), _dp(_f64(x1)),
                               float(band), _dp(out), 16)
        return out[: 3 * n].reshape(n, 3)

    def face_ctrl(self, e, f):
        g = self.ngeo + 1
        out = np.zeros(g * g * 3)
        lib().or_face_ctrl(self.h, int(e), int(f), _dp(out))
        return out.reshape(g, g, 3)  # [k(t)][m(s)][xyz]

    def locate_bruteforce(self, x, tol=1e-10, params: Params | None = None):
        params = params or make_params()
        out = np.zeros(64, dtype=np.int32)
        n = lib().or_locate_bruteforce(self.h, ctypes.byref(params), _dp(_f64(x)), float(tol),
                                       _ip(out), 64)
        return out[:n].copy()

    def push(self, params: Params, x, v, d, elem, hits=None, status=None, nsteps=1, dt=1e-3):
        """Advance particles in place-copies; returns dict of new arrays (AoS x,v)."""
        x = _f64(x).copy()
        v = _f64(v).copy()
        d = _f64(d)
        elem = _i32(elem).copy()
        n = len(d)
        hits = np.zeros(n, np.int32) if hits is None else _i32(hits).copy()
        status = np.zeros(n, np.uint32) if status is None else np.ascontiguousarray(
            status, dtype=np.uint32).copy()
        assert x.shape == (n, 3) and v.shape == (n, 3) and elem.shape == (n,)
        lib().or_push(self.h, ctypes.byref(params), n, _dp(x), _dp(v), _dp(d), _ip(elem),
                      _ip(hits), _up(status), int(nsteps), float(dt))
        return dict(x=x, v=v, elem=elem, hits=hits, status=status)

    def stage1(self, params: Params, e, x, v, d, dt):
        """First RK stage without tracking: dict of xi, U (5), acc, dx, dv, or
        None if the inverse map fails."""
        out = np.zeros(17)
        ok = lib().or_stage1(self.h, ctypes.byref(params), int(e), _dp(_f64(x)), _dp(_f64(v)),
                             float(d), float(dt), _dp(out))
        if not ok:
            return None
        return dict(xi=out[0:3], U=out[3:8], acc=out[8:11], dx=out[11:14], dv=out[14:17])

    def deposit(self, params: Params, x, v, d, elem, status=None):
        n = len(d)
        status = np.zeros(n, np.uint32) if status is None else np.ascontiguousarray(
            status, dtype=np.uint32)
        nn = (self.N + 1) ** 3
        S = np.zeros(self.nelem * 4 * nn)
        lib().or_deposit(self.h, ctypes.byref(params), n, _dp(_f64(x)), _dp(_f64(v)),
                         _dp(_f64(d)), _ip(_i32(elem)), _up(status), _dp(S))
        return S.reshape(self.nelem, 4, nn)

    def deposit_nearest(self, params: Params, x, v, d, elem, status=None):
        n = len(d)
        status = np.zeros(n, np.uint32) if status is None else np.ascontiguousarray(
            status, dtype=np.uint32)
        nn = (self.N + 1) ** 3
        S = np.zeros(self.nelem * 4 * nn)
        lib().or_deposit_nearest(self.h, ctypes.byref(params), n, _dp(_f64(x)), _dp(_f64(v)),
                                 _dp(_f64(d)), _ip(_i32(elem)), _up(status), _dp(S))
        return S.reshape(self.nelem, 4, nn)

    def mlp_features(self, e, x):
        out = np.zeros(51)
        lib().or_mlp_features(self.h, int(e), _dp(_f64(x)), _dp(out))
        return out


def mlp_nparams() -> int:
    return lib().or_mlp_nparams()


def mlp_forward(theta, inp):
    theta, inp = _f64(theta), _f64(inp)
    B = inp.shape[0]
    out = np.zeros((B, 3))
    lib().or_mlp_forward(_dp(theta), B, _dp(inp), _dp(out))
    return out


def mlp_loss_grad(theta, inp, target):
    theta, inp, target = _f64(theta), _f64(inp), _f64(target)
    grad = np.zeros_like(theta)
    loss = lib().or_mlp_loss_grad(_dp(theta), inp.shape[0], _dp(inp), _dp(target), _dp(grad))
    return loss, grad


def adam(theta, g, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """In-place Adam step on float64 arrays."""
    lib().or_adam(len(theta), _dp(theta), _dp(_f64(g)), _dp(m), _dp(v), int(t), lr, b1, b2, eps)
