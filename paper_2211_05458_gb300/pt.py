"""ctypes binding of libpt (include/pt.h): argument marshalling only.

Every step of the push runs in libpt's CUDA kernels; this module only turns
torch tensors into the pointers and sizes of the C ABI.  It raises at import
of the library if libpt.so has not been built -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

from . import build as _build

PT_OK, PT_ERR_ARG, PT_ERR_CUDA, PT_ERR_NEWTON, PT_ERR_LOST, PT_ERR_CROSS = 0, 1, 2, 3, 4, 5
PT_ERR_TIMEOUT, PT_ERR_STATE, PT_WARN_DT = 6, 7, 16
ST_NEWTON_FAIL, ST_LOST, ST_CROSS_CAP, ST_NEAR_FACE, ST_REP800, ST_OPEN = 1, 2, 4, 8, 16, 32
ST_NEAR_WALL = 64
ST_FROZEN = ST_NEWTON_FAIL | ST_LOST | ST_CROSS_CAP | ST_OPEN
FP64, FP32 = 0, 1
STOKES, SCHILLER_NAUMANN = 0, 1
GUESS_TRILINEAR, GUESS_MLP = 0, 1
DEPOSIT_ATOMIC, DEPOSIT_SEGMENTED, DEPOSIT_NEAREST = 0, 1, 2
TRACK_PHYSICAL, TRACK_REFERENCE = 0, 1
SCHEDULE_AUTO, SCHEDULE_RESIDENT, SCHEDULE_STAGED = 0, 1, 2

_vp = ctypes.c_void_p


class Config(ctypes.Structure):
    _fields_ = [("mu", ctypes.c_double), ("rho_p", ctypes.c_double),
                ("g", ctypes.c_double * 3), ("drag_mask", ctypes.c_double * 3),
                ("newton_tol", ctypes.c_double), ("band_ref", ctypes.c_double),
                ("band_x", ctypes.c_double), ("lost_tol", ctypes.c_double),
                ("precision", ctypes.c_int32), ("drag_law", ctypes.c_int32),
                ("guess", ctypes.c_int32), ("max_newton", ctypes.c_int32),
                ("max_cross", ctypes.c_int32), ("rebin_every", ctypes.c_int32),
                ("block", ctypes.c_int32), ("lift", ctypes.c_int32),
                ("sphericity", ctypes.c_double), ("track", ctypes.c_int32),
                ("buoyancy", ctypes.c_int32), ("curved_faces", ctypes.c_int32),
                ("schedule", ctypes.c_int32), ("reserved", ctypes.c_int32 * 2)]


class MeshDesc(ctypes.Structure):
    _fields_ = [("nelem", ctypes.c_int32), ("ngeo", ctypes.c_int32), ("xgeo", _vp),
                ("neighbor", _vp), ("nbr_face", _vp), ("bc", _vp), ("shift", _vp),
                ("nmortar", ctypes.c_int32), ("mortar", _vp)]


class CParticles(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("x", _vp), ("v", _vp), ("d", _vp), ("elem", _vp),
                ("hits", _vp), ("status", _vp)]


STAT_FIELDS = ["particle_steps", "crossings", "wall_hits", "newton_it_fp32", "newton_it_fp64",
               "slow_track", "near_face", "newton_fail", "lost", "cross_cap", "open", "rep800",
               "dt_warn", "near_wall"]


class Histograms(ctypes.Structure):
    _fields_ = [("newton_fp32", ctypes.c_int64 * 8), ("newton_final", ctypes.c_int64 * 8),
                ("crossings", ctypes.c_int64 * 4)]


class Stats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in STAT_FIELDS] + [("reserved", ctypes.c_int64 * 2)]

    def as_dict(self):
        return {f: int(getattr(self, f)) for f in STAT_FIELDS}


_lock = threading.Lock()
_lib = None

EXPORTS = ["pt_config_default", "pt_init_mesh", "pt_set_config", "pt_set_fluid", "pt_push",
           "pt_push_host", "pt_deposit", "pt_locate", "pt_mlp_make_pairs", "pt_mlp_train",
           "pt_mlp_features", "pt_mlp_nparams", "pt_mlp_set", "pt_mlp_get", "pt_mlp_forward",
           "pt_mlp_grad", "pt_push_batch", "pt_profile", "pt_profile_read", "pt_destroy",
           "pt_last_error", "pt_deposit_noalloc", "pt_find_element", "pt_stage_terms",
           "pt_launch_count", "pt_measure_peak", "pt_mlp_start", "pt_read_histograms",
           "pt_batch_tuning", "pt_profile_read_kind", "pt_push_stage"]


def library_path() -> str:
    return _build.SO


def lib():
    """Load libpt.so (built by paper_2211_05458_gb300.build); raises if absent."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_build.SO):
                raise RuntimeError(f"libpt.so is not built ({_build.SO}); run "
                                   "`python -m paper_2211_05458_gb300.build` -- no fallback exists")
            L = ctypes.CDLL(_build.SO)
            st = ctypes.c_int
            L.pt_config_default.argtypes = [ctypes.POINTER(Config)]
            L.pt_config_default.restype = None
            L.pt_init_mesh.argtypes = [ctypes.POINTER(_vp), ctypes.POINTER(MeshDesc),
                                       ctypes.POINTER(Config), _vp]
            L.pt_set_config.argtypes = [_vp, ctypes.POINTER(Config)]
            L.pt_set_fluid.argtypes = [_vp, ctypes.c_int32, ctypes.c_int32, _vp]
            L.pt_push.argtypes = [_vp, ctypes.POINTER(CParticles), ctypes.c_int32, ctypes.c_double,
                                  ctypes.POINTER(Stats)]
            L.pt_push_host.argtypes = L.pt_push.argtypes
            L.pt_push_stage.argtypes = L.pt_push.argtypes
            L.pt_deposit.argtypes = [_vp, ctypes.POINTER(CParticles), ctypes.c_int32, _vp]
            L.pt_deposit_noalloc.argtypes = [_vp, ctypes.POINTER(CParticles), ctypes.c_int32,
                                             _vp]
            L.pt_locate.argtypes = [_vp, ctypes.c_int64, _vp, _vp, _vp, _vp, _vp]
            L.pt_mlp_make_pairs.argtypes = [_vp, ctypes.c_int64, ctypes.c_uint64, _vp, _vp]
            L.pt_mlp_train.argtypes = [_vp, ctypes.c_int64, _vp, _vp, ctypes.c_int32,
                                       ctypes.c_int32, ctypes.c_float, ctypes.c_uint64, _vp]
            L.pt_mlp_features.argtypes = [_vp, ctypes.c_int64, _vp, _vp, _vp]
            L.pt_mlp_nparams.argtypes = []
            L.pt_mlp_nparams.restype = ctypes.c_int32
            L.pt_mlp_set.argtypes = [_vp, _vp, _vp]
            L.pt_mlp_get.argtypes = [_vp, _vp, _vp]
            L.pt_mlp_forward.argtypes = [_vp, ctypes.c_int32, _vp, _vp]
            L.pt_mlp_grad.argtypes = [_vp, ctypes.c_int32, _vp, _vp, _vp, _vp]
            L.pt_push_batch.argtypes = [ctypes.POINTER(_vp), ctypes.POINTER(CParticles),
                                        ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                        ctypes.POINTER(Stats)]
            L.pt_find_element.argtypes = [_vp, ctypes.c_int64, _vp, _vp, _vp, _vp]
            L.pt_stage_terms.argtypes = [_vp, ctypes.POINTER(CParticles), ctypes.c_double, _vp,
                                         _vp, _vp, _vp, _vp]
            L.pt_profile.argtypes = [_vp, ctypes.c_int32]
            L.pt_profile_read.argtypes = [_vp, ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_int64)]
            L.pt_launch_count.argtypes = [_vp, ctypes.POINTER(ctypes.c_int64)]
            L.pt_read_histograms.argtypes = [_vp, ctypes.POINTER(Histograms)]
            L.pt_batch_tuning.argtypes = [_vp, _vp, _vp, _vp, ctypes.c_int32,
                                          ctypes.POINTER(ctypes.c_int32)]
            L.pt_mlp_start.argtypes = [_vp, ctypes.c_int64, _vp, _vp, _vp, ctypes.c_int32]
            L.pt_measure_peak.argtypes = [ctypes.c_int32, _vp, ctypes.POINTER(ctypes.c_double)]
            L.pt_profile_read_kind.argtypes = [_vp, ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                                               ctypes.POINTER(ctypes.c_int64)]
            L.pt_destroy.argtypes = [_vp]
            L.pt_last_error.argtypes = [_vp]
            L.pt_last_error.restype = ctypes.c_char_p
            for name in EXPORTS:
                if name not in ("pt_config_default", "pt_mlp_nparams", "pt_last_error"):
                    getattr(L, name).restype = st
            _lib = L
    return _lib


class PtError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libpt status {code}: {msg}")
        self.code = code


def _ptr(t: torch.Tensor | None):
    if t is None:
        return None
    assert t.is_contiguous(), "libpt needs contiguous tensors"
    return ctypes.c_void_p(t.data_ptr())


def default_config(**kw) -> Config:
    c = Config()
    lib().pt_config_default(ctypes.byref(c))
    for k, v in kw.items():
        if k in ("g", "drag_mask"):
            getattr(c, k)[:] = list(v)
        else:
            setattr(c, k, v)
    return c


class ParticleSet:
    """Particle state as structure-of-arrays tensors (device or host)."""

    def __init__(self, x, v, d, elem, hits=None, status=None):
        n = x.shape[1]
        self.x, self.v, self.d, self.elem = x, v, d, elem
        self.hits = torch.zeros(n, dtype=torch.int32, device=x.device) if hits is None else hits
        self.status = torch.zeros(n, dtype=torch.int32, device=x.device) if status is None else status

    @property
    def n(self):
        return self.x.shape[1]

    @classmethod
    def create(cls, x, v, d, elem, precision: int, device, pin: bool = False):
        """x, v: [n][3]; d, elem: [n] (any tensor/array); returns SoA tensors."""
        rd = torch.float64 if precision == FP64 else torch.float32

        def T(a, dt):
            # always a private copy: the push updates these arrays in place
            t = torch.as_tensor(a).to(device=device, dtype=dt, copy=True).contiguous()
            return t.pin_memory() if pin and t.device.type == "cpu" else t
        x = T(torch.as_tensor(x).T.contiguous(), torch.float64)
        v = T(torch.as_tensor(v).T.contiguous(), rd)
        return cls(x, v, T(d, rd), T(elem, torch.int32), None if not pin else
                   torch.zeros(x.shape[1], dtype=torch.int32).pin_memory(),
                   None if not pin else torch.zeros(x.shape[1], dtype=torch.int32).pin_memory())

    def struct(self) -> CParticles:
        p = CParticles()
        p.n = self.n
        p.x, p.v, p.d = _ptr(self.x), _ptr(self.v), _ptr(self.d)
        p.elem, p.hits, p.status = _ptr(self.elem), _ptr(self.hits), _ptr(self.status)
        return p

    def clone(self):
        return ParticleSet(self.x.clone(), self.v.clone(), self.d.clone(), self.elem.clone(),
                           self.hits.clone(), self.status.clone())

    def to(self, device, pin=False):
        def T(t):
            t = t.to(device).contiguous()
            return t.pin_memory() if pin and t.device.type == "cpu" else t
        return ParticleSet(T(self.x), T(self.v), T(self.d), T(self.elem), T(self.hits),
                           T(self.status))


class Context:
    """One mesh on the current CUDA device; work goes to the current torch stream."""

    def __init__(self, mesh, stream: torch.cuda.Stream | None = None, **cfg):
        L = lib()
        md = mesh.as_dict() if hasattr(mesh, "as_dict") else mesh
        import numpy as np
        self._host = dict(xgeo=np.ascontiguousarray(md["xgeo"], dtype=np.float64),
                          neighbor=np.ascontiguousarray(md["neighbor"], dtype=np.int32),
                          nbr_face=np.ascontiguousarray(md["nbr_face"], dtype=np.int32),
                          bc=np.ascontiguousarray(md["bc"], dtype=np.int32),
                          shift=np.ascontiguousarray(md["shift"], dtype=np.float64))
        mortar = md.get("mortar")
        if mortar is not None and len(mortar):
            self._host["mortar"] = np.ascontiguousarray(mortar, dtype=np.int32).reshape(-1, 9)
        d = MeshDesc()
        d.nelem, d.ngeo = int(md["nelem"]), int(md["ngeo"])
        d.nmortar = len(self._host["mortar"]) if "mortar" in self._host else 0
        for k, a in self._host.items():
            setattr(d, k, a.ctypes.data)
        self.cfg = default_config(**cfg)
        self.stream = stream or torch.cuda.current_stream()
        h = _vp()
        rc = L.pt_init_mesh(ctypes.byref(h), ctypes.byref(d), ctypes.byref(self.cfg),
                            _vp(self.stream.cuda_stream))
        if rc != PT_OK:
            raise PtError(rc, L.pt_last_error(None).decode())
        self.h = h
        self.nelem, self.ngeo = d.nelem, d.ngeo
        self.N = None
        self._U = None

    def _check(self, rc, allow=(PT_OK,)):
        if rc not in allow:
            raise PtError(rc, lib().pt_last_error(self.h).decode())
        return rc

    @property
    def precision(self):
        return self.cfg.precision

    def set_config(self, **kw):
        c = Config()
        ctypes.memmove(ctypes.byref(c), ctypes.byref(self.cfg), ctypes.sizeof(Config))
        for k, v in kw.items():
            if k in ("g", "drag_mask"):
                getattr(c, k)[:] = list(v)
            else:
                setattr(c, k, v)
        self._check(lib().pt_set_config(self.h, ctypes.byref(c)))
        self.cfg = c

    def set_fluid(self, N: int, node_type: int, U: torch.Tensor):
        want = torch.float64 if self.cfg.precision == FP64 else torch.float32
        assert U.is_cuda and U.dtype == want and U.is_contiguous()
        assert U.numel() == self.nelem * 5 * (N + 1) ** 3
        self._check(lib().pt_set_fluid(self.h, N, node_type, _ptr(U)))
        self._U = U
        self.N = N

    def push(self, parts: ParticleSet, nsteps: int, dt: float, stats: bool = True,
             allow_errors: bool = True):
        st = Stats() if stats else None
        allow = (PT_OK, PT_WARN_DT, PT_ERR_NEWTON, PT_ERR_LOST, PT_ERR_CROSS) if allow_errors \
            else (PT_OK, PT_WARN_DT)
        p = parts.struct()
        rc = lib().pt_push(self.h, ctypes.byref(p), int(nsteps), float(dt),
                           ctypes.byref(st) if st is not None else None)
        self._check(rc, allow)
        if st is None:
            return None
        out = st.as_dict()
        out["status_code"] = rc
        return out

    def push_stage(self, parts: ParticleSet, stage: int, dt: float, stats: bool = False):
        """One RK stage (0..4 in turn) for a solver that updates the fluid state
        between stages; the particle arrays are updated at stage 4."""
        st = Stats() if stats else None
        p = parts.struct()
        rc = lib().pt_push_stage(self.h, ctypes.byref(p), int(stage), float(dt),
                                 ctypes.byref(st) if st is not None else None)
        self._check(rc, (PT_OK, PT_WARN_DT, PT_ERR_NEWTON, PT_ERR_LOST, PT_ERR_CROSS))
        return st.as_dict() if st is not None else None

    def push_host(self, parts: ParticleSet, nsteps: int, dt: float, stats: bool = True):
        st = Stats() if stats else None
        p = parts.struct()
        rc = lib().pt_push_host(self.h, ctypes.byref(p), int(nsteps), float(dt),
                                ctypes.byref(st) if st is not None else None)
        self._check(rc, (PT_OK, PT_WARN_DT, PT_ERR_NEWTON, PT_ERR_LOST, PT_ERR_CROSS))
        return st.as_dict() if st is not None else None

    def deposit(self, parts: ParticleSet, mode: int, S: torch.Tensor | None = None):
        n3 = (self.N + 1) ** 3
        if S is None:
            S = torch.empty((self.nelem, 4, n3), dtype=torch.float32, device=parts.x.device)
        p = parts.struct()
        self._check(lib().pt_deposit(self.h, ctypes.byref(p), int(mode), _ptr(S)))
        return S

    def stage_terms(self, parts: ParticleSet, dt: float):
        """First-stage terms by the push's code (no tracking): dict of xi [3][n]
        float64, U [4][n], acc, dx, dv [3][n] in the particle precision; the
        particles' status receives the per-particle status bits."""
        n = parts.n
        dev, rd = parts.x.device, parts.v.dtype
        out = dict(xi=torch.zeros((3, n), dtype=torch.float64, device=dev),
                   U=torch.zeros((4, n), dtype=rd, device=dev),
                   acc=torch.zeros((3, n), dtype=rd, device=dev),
                   dx=torch.zeros((3, n), dtype=rd, device=dev),
                   dv=torch.zeros((3, n), dtype=rd, device=dev))
        p = parts.struct()
        self._check(lib().pt_stage_terms(self.h, ctypes.byref(p), float(dt), _ptr(out["xi"]),
                                          _ptr(out["U"]), _ptr(out["acc"]), _ptr(out["dx"]),
                                          _ptr(out["dv"])))
        return out

    def find_element(self, x: torch.Tensor):
        """x: [3][n] float64 cuda -> (elem [n] int32, -1 if outside; xi [3][n]; status)."""
        n = x.shape[1]
        elem = torch.empty(n, dtype=torch.int32, device=x.device)
        xi = torch.empty_like(x)
        st = torch.empty(n, dtype=torch.int32, device=x.device)
        self._check(lib().pt_find_element(self.h, n, _ptr(x), _ptr(elem), _ptr(xi), _ptr(st)))
        return elem, xi, st

    def locate(self, x: torch.Tensor, elem: torch.Tensor):
        """x: [3][n] float64 cuda, elem: [n] int32 cuda -> (xi [3][n], iters, status)."""
        n = x.shape[1]
        xi = torch.empty_like(x)
        it = torch.empty(n, dtype=torch.int32, device=x.device)
        st = torch.empty(n, dtype=torch.int32, device=x.device)
        self._check(lib().pt_locate(self.h, n, _ptr(x), _ptr(elem), _ptr(xi), _ptr(it), _ptr(st)))
        return xi, it, st

    # learned guess -------------------------------------------------------
    def mlp_make_pairs(self, n: int, seed: int, device="cuda"):
        inp = torch.empty((n, 51), dtype=torch.float32, device=device)
        tgt = torch.empty((n, 3), dtype=torch.float32, device=device)
        self._check(lib().pt_mlp_make_pairs(self.h, n, seed, _ptr(inp), _ptr(tgt)))
        return inp, tgt

    def mlp_train(self, inp, tgt, epochs=20, batch=4096, lr=1e-3, seed=0):
        loss = (ctypes.c_float * max(1, epochs))()
        self._check(lib().pt_mlp_train(self.h, inp.shape[0], _ptr(inp), _ptr(tgt), epochs, batch,
                                       ctypes.c_float(lr), seed, loss))
        return list(loss)[:epochs]

    def mlp_start(self, x, elem, engine: int = 1):
        """Learned Newton start of x [3][n] float64 cuda in elem [n] int32:
        guess [3][n] float32 (engine 1 tensor cores, 0 warp mma.sync)."""
        n = x.shape[1]
        g = torch.zeros((3, n), dtype=torch.float32, device=x.device)
        self._check(lib().pt_mlp_start(self.h, n, _ptr(x), _ptr(elem), _ptr(g), int(engine)))
        return g

    def mlp_features(self, x, elem):
        n = x.shape[1]
        f = torch.empty((n, 51), dtype=torch.float32, device=x.device)
        self._check(lib().pt_mlp_features(self.h, n, _ptr(x), _ptr(elem), _ptr(f)))
        return f

    def mlp_get(self):
        n = lib().pt_mlp_nparams()
        th = torch.zeros(n, dtype=torch.float32)
        nm = torch.zeros(105, dtype=torch.float32)
        self._check(lib().pt_mlp_get(self.h, _ptr(th), _ptr(nm)))
        return th, nm

    def mlp_set(self, theta, norm):
        theta = torch.as_tensor(theta, dtype=torch.float32).contiguous()
        norm = torch.as_tensor(norm, dtype=torch.float32).contiguous()
        self._check(lib().pt_mlp_set(self.h, _ptr(theta), _ptr(norm)))

    def mlp_forward(self, inp):
        out = torch.empty((inp.shape[0], 3), dtype=torch.float32, device=inp.device)
        self._check(lib().pt_mlp_forward(self.h, inp.shape[0], _ptr(inp), _ptr(out)))
        return out

    def mlp_grad(self, inp, tgt):
        n = lib().pt_mlp_nparams()
        g = torch.empty(n, dtype=torch.float32, device=inp.device)
        loss = ctypes.c_float(0.0)
        self._check(lib().pt_mlp_grad(self.h, inp.shape[0], _ptr(inp), _ptr(tgt), _ptr(g),
                                      ctypes.byref(loss)))
        return float(loss.value), g

    def profile(self, enable: bool = True):
        self._check(lib().pt_profile(self.h, 1 if enable else 0))

    def profile_read(self):
        ms, k = ctypes.c_double(0.0), ctypes.c_int64(0)
        self._check(lib().pt_profile_read(self.h, ctypes.byref(ms), ctypes.byref(k)))
        return float(ms.value), int(k.value)

    def histograms(self):
        """Histograms of the last push (staged schedule): dict of lists."""
        h = Histograms()
        self._check(lib().pt_read_histograms(self.h, ctypes.byref(h)))
        return {"newton_fp32": list(h.newton_fp32), "newton_final": list(h.newton_final),
                "crossings": list(h.crossings)}

    def profile_read_kind(self, kind: int):
        """(ms, launches) of one kernel kind: 0 push/chunk, 1 stage, 2 learned
        start, 3 exact tracking; clears that record only."""
        ms, k = ctypes.c_double(0.0), ctypes.c_int64(0)
        self._check(lib().pt_profile_read_kind(self.h, int(kind), ctypes.byref(ms),
                                               ctypes.byref(k)))
        return float(ms.value), int(k.value)

    def launch_count(self):
        """Kernel launches this context queued since the last call (then cleared)."""
        k = ctypes.c_int64(0)
        self._check(lib().pt_launch_count(self.h, ctypes.byref(k)))
        return int(k.value)

    def close(self):
        if getattr(self, "h", None):
            lib().pt_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def push_batch(ctxs, parts, nsteps: int, dt: float, stats: bool = True):
    n = len(ctxs)
    hs = (_vp * n)(*[c.h for c in ctxs])
    ps = (CParticles * n)(*[p.struct() for p in parts])
    st = (Stats * n)() if stats else None
    rc = lib().pt_push_batch(hs, ps, n, int(nsteps), float(dt), st)
    if rc not in (PT_OK, PT_WARN_DT, PT_ERR_NEWTON, PT_ERR_LOST, PT_ERR_CROSS):
        raise PtError(rc, lib().pt_last_error(ctxs[0].h).decode())
    return [s.as_dict() for s in st] if st is not None else None


def measure_peak(kind: int, stream=None) -> float:
    """Measured FMA throughput of the current device in TFLOP/s (kind 0 FP32,
    1 FP64), from libpt's own probe kernel."""
    t = ctypes.c_double(0.0)
    s = None if stream is None else ctypes.c_void_p(stream.cuda_stream)
    rc = lib().pt_measure_peak(int(kind), s, ctypes.byref(t))
    if rc != 0:
        raise PtError(rc, "pt_measure_peak failed")
    return float(t.value)


def batch_tuning(ctx0):
    """Per degree group of the batched push led by ctx0: list of dicts
    (N, chosen block size, ms per step of the 64/96/128 candidates)."""
    ng = ctypes.c_int32(0)
    n = (ctypes.c_int32 * 8)()
    b = (ctypes.c_int32 * 8)()
    ms = (ctypes.c_float * 24)()
    rc = lib().pt_batch_tuning(ctx0.h, n, b, ms, 8, ctypes.byref(ng))
    if rc != 0:
        raise PtError(rc, "pt_batch_tuning failed")
    return [{"N": int(n[i]), "block": int(b[i]), "ms_per_step": [float(ms[3 * i + k]) for k in range(3)]}
            for i in range(min(ng.value, 8))]
