"""Seeded synthetic inputs for the particle push: meshes, fluid states, particles.

This module holds none of the push's arithmetic.  It only places geometry
nodes by analytic formulas, writes the element connectivity of structured
hexahedral meshes, samples analytic flow fields at the DG solution nodes and
draws particles.  Both the CUDA path and the oracle consume what it produces.

Recipes (the readings of arXiv 2211.05458 used for the five workloads):

* periodic box  [0,1]^3 (or any box), straight hexahedra, Taylor-Green vortex
  u = (sin 2pi x cos 2pi y cos 2pi z, -cos 2pi x sin 2pi y cos 2pi z, 0),
  rho = 1, p = p0 + (cos 4pi x + cos 4pi y)(cos 4pi z + 2)/16, p0 = 100/1.4.
* curved channel [0,2pi] x [-1,1] x [0,pi], walls at y = +-1 (specular),
  periodic in x and z, geometry nodes equidistant per element and moved by
  y' = y + A (1 - y^2) sin(x) sin(2z), A = 0.05 (walls stay planar).  The
  "curved_walls" variant uses y' = y + A sin(x) sin(2z) (walls curved too).
* channel fluid: Poiseuille (1 - y^2) e_x plus the curl of a vector potential
  (1 - y^2)^2 psi(x), psi a sum of random-phase Fourier modes with |k| <= 8,
  integer k_x, even k_z, amplitude |k|^(-5/6) / |k| (energy spectrum ~ k^-5/3),
  scaled to u'_rms = 0.1 at the nodes; rho = 1, p = 100/1.4.
* mortar box: [0,1]^3 with n^3 elements joined at x = 1 by non-conforming
  faces to [1,2]x[0,1]^2 refined by two in x and in one or both transverse
  directions (each big face matched to four or two small faces), walls
  outside; geometry moved by a warp of degree <= 2 per direction
  (x' = x + A (y^2 - y z), y' = y + A x (2 - x)(1 + z), z' = z + A x y) or of
  degree 1 (x' = x + A y z, y' = y + A x z, z' = z + A x y), which both
  blocks' nodes reproduce exactly at NGeo >= 2 (>= 1), so the small faces
  tile the big one to rounding.
* particles: element drawn uniformly, reference position uniform in
  [-(1-m), 1-m]^3 mapped by the same analytic node placement (so the draw is
  uniform in reference space, not exactly uniform in x); margin m keeps the
  seeded owner unambiguous.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch

P0 = 100.0 / 1.4
GAMMA = 1.4

# local faces: 0: xi1=-1, 1: xi1=+1, 2: xi2=-1, 3: xi2=+1, 4: xi3=-1, 5: xi3=+1
BC_INTERNAL, BC_WALL, BC_PERIODIC, BC_OPEN, BC_MORTAR = 0, 1, 2, 3, 4
# mortar table rows: type (1: four small faces, 2: two split along s, 3: two
# split along t), four small elements, their four local faces (-1 unused)
MORTAR_FOUR, MORTAR_S, MORTAR_T = 1, 2, 3


def gauss_nodes(n: int) -> np.ndarray:
    """Legendre-Gauss nodes (numpy's library routine)."""
    return np.polynomial.legendre.leggauss(n)[0]


def gll_nodes(n: int) -> np.ndarray:
    """Legendre-Gauss-Lobatto nodes: -1, 1 and the roots of P_{n-1}' (numpy)."""
    if n == 1:
        return np.zeros(1)
    c = np.zeros(n)
    c[-1] = 1.0
    inner = np.polynomial.legendre.Legendre(c).deriv().roots()
    return np.concatenate([[-1.0], np.sort(inner.real), [1.0]])


def solution_nodes(N: int, node_type: int) -> np.ndarray:
    return gauss_nodes(N + 1) if node_type == 0 else gll_nodes(N + 1)


@dataclass
class Mesh:
    nelem: int
    ngeo: int
    xgeo: np.ndarray       # [nelem][(ngeo+1)^3][3]
    neighbor: np.ndarray   # [nelem][6] int32
    nbr_face: np.ndarray   # [nelem][6] int32
    bc: np.ndarray         # [nelem][6] int32
    shift: np.ndarray      # [nelem][6][3]
    dims: tuple = (1, 1, 1)
    lo: tuple = (0.0, 0.0, 0.0)
    hi: tuple = (1.0, 1.0, 1.0)
    warp: str = "none"
    amp: float = 0.0
    extra: dict = field(default_factory=dict)
    mortar: np.ndarray = field(default_factory=lambda: np.zeros((0, 9), np.int32))

    def as_dict(self) -> dict:
        return dict(nelem=self.nelem, ngeo=self.ngeo, xgeo=self.xgeo, neighbor=self.neighbor,
                    nbr_face=self.nbr_face, bc=self.bc, shift=self.shift, mortar=self.mortar)


def _warp_torch(kind: str, amp: float, x, y, z):
    if kind == "none":
        return x, y, z
    if kind == "channel":
        return x, y + amp * (1.0 - y * y) * torch.sin(x) * torch.sin(2.0 * z), z
    if kind == "channel_curved_walls":
        return x, y + amp * torch.sin(x) * torch.sin(2.0 * z), z
    if kind == "poly":
        # a polynomial warp of degree 2 per axis (exactly representable at NGeo >= 2)
        return x, y + amp * x * x * (1.0 + z), z + 0.5 * amp * x * y
    if kind == "mortar_poly":
        # degree <= 2 per direction; the plane x = 1 becomes curved
        return (x + amp * (y * y - y * z), y + amp * x * (2.0 - x) * (1.0 + z),
                z + amp * x * y)
    if kind == "mortar_trilinear":
        # degree 1 per direction (exactly representable at NGeo >= 1)
        return x + amp * y * z, y + amp * x * z, z + amp * x * y
    raise ValueError(kind)


def box_mesh(dims, lo, hi, ngeo: int, periodic=(True, True, True), warp: str = "none",
             amp: float = 0.0, boundary_bc: int = BC_WALL) -> Mesh:
    """Structured hexahedral mesh on a box; node (a,b,c) of element (i,j,k) sits
    at the global lattice point (i*ngeo+a, j*ngeo+b, k*ngeo+c), so shared
    nodes are bitwise identical in both elements, then is moved by the warp."""
    nx, ny, nz = dims
    g = ngeo + 1
    E = nx * ny * nz
    lat = [lo[d] + (hi[d] - lo[d]) * torch.arange(dims[d] * ngeo + 1, dtype=torch.float64)
           / (dims[d] * ngeo) for d in range(3)]
    # exact end points
    for d in range(3):
        lat[d][-1] = hi[d]
    ii = torch.arange(nx).view(1, 1, nx, 1, 1, 1)
    jj = torch.arange(ny).view(1, ny, 1, 1, 1, 1)
    kk = torch.arange(nz).view(nz, 1, 1, 1, 1, 1)
    aa = torch.arange(g).view(1, 1, 1, 1, 1, g)
    bb = torch.arange(g).view(1, 1, 1, 1, g, 1)
    cc = torch.arange(g).view(1, 1, 1, g, 1, 1)
    shape = (nz, ny, nx, g, g, g)
    X = lat[0][(ii * ngeo + aa).expand(shape)]
    Y = lat[1][(jj * ngeo + bb).expand(shape)]
    Z = lat[2][(kk * ngeo + cc).expand(shape)]
    X, Y, Z = _warp_torch(warp, amp, X, Y, Z)
    xgeo = torch.stack([X, Y, Z], dim=-1).reshape(E, g * g * g, 3).numpy().copy()

    e = np.arange(E)
    i, j, k = e % nx, (e // nx) % ny, e // (nx * ny)
    idx = [i, j, k]
    n = [nx, ny, nz]
    neighbor = np.full((E, 6), -1, np.int32)
    nbr_face = np.full((E, 6), -1, np.int32)
    bc = np.zeros((E, 6), np.int32)
    shift = np.zeros((E, 6, 3))
    for d in range(3):
        L = hi[d] - lo[d]
        for side in (0, 1):
            f = 2 * d + side
            step = 1 if side else -1
            q = idx[d] + step
            inside = (q >= 0) & (q < n[d])
            qq = q % n[d]
            nb_idx = [i.copy(), j.copy(), k.copy()]
            nb_idx[d] = qq
            nb = nb_idx[0] + nx * (nb_idx[1] + ny * nb_idx[2])
            if periodic[d]:
                neighbor[:, f] = nb
                nbr_face[:, f] = f ^ 1
                bc[:, f] = np.where(inside, BC_INTERNAL, BC_PERIODIC)
                shift[~inside, f, d] = -step * L
            else:
                neighbor[:, f] = np.where(inside, nb, -1)
                nbr_face[:, f] = np.where(inside, f ^ 1, -1)
                bc[:, f] = np.where(inside, BC_INTERNAL, boundary_bc)
    return Mesh(E, ngeo, xgeo, neighbor, nbr_face, bc, shift, dims=tuple(dims), lo=tuple(lo),
                hi=tuple(hi), warp=warp, amp=amp)


def channel_mesh(dims, ngeo: int, amp: float = 0.05, curved_walls: bool = False) -> Mesh:
    return box_mesh(dims, (0.0, -1.0, 0.0), (2.0 * math.pi, 1.0, math.pi), ngeo,
                    periodic=(True, False, True),
                    warp="channel_curved_walls" if curved_walls else "channel", amp=amp)


def mortar_box(n: int = 4, ngeo: int = 2, split: str = "st", amp: float = 0.04,
               warp: str = "mortar_poly", boundary_bc: int = BC_WALL) -> Mesh:
    """Non-conforming mesh: block A = [0,1]^3 with n^3 elements, block B =
    [1,2]x[0,1]^2 with (2n, 2n, 2n) elements (split "st": every big face of A
    at x = 1 matched to four small faces of B), (2n, 2n, n) (split "s": two
    small faces along y, the big face's s) or (2n, n, 2n) (split "t": along
    z).  Small face k of a big face covers the part of its (s,t) range given
    by the mortar type (MORTAR_FOUR: k = i_s + 2 i_t; MORTAR_S: k = i_s;
    MORTAR_T: k = i_t; i = 0 below the midpoint, 1 above).  Outer faces get
    boundary_bc.  Block B's element (i, j, k) has index n^3 + i + nbx (j + nby k)."""
    ry, rz = {"st": (2, 2), "s": (2, 1), "t": (1, 2)}[split]
    mtype = {"st": MORTAR_FOUR, "s": MORTAR_S, "t": MORTAR_T}[split]
    per = (False, False, False)
    A = box_mesh((n, n, n), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0), ngeo, per, warp, amp, boundary_bc)
    fd = (2 * n, ry * n, rz * n)
    B = box_mesh(fd, (1.0, 0.0, 0.0), (2.0, 1.0, 1.0), ngeo, per, warp, amp, boundary_bc)
    Ea, Eb = A.nelem, B.nelem
    xgeo = np.concatenate([A.xgeo, B.xgeo])
    nbrB = np.where(B.neighbor >= 0, B.neighbor + Ea, -1).astype(np.int32)
    neighbor = np.concatenate([A.neighbor, nbrB])
    nbr_face = np.concatenate([A.nbr_face, B.nbr_face])
    bc = np.concatenate([A.bc, B.bc])
    shift = np.concatenate([A.shift, B.shift])
    mortar = np.full((n * n, 9), -1, np.int32)
    mortar[:, 0] = mtype
    for kc in range(n):
        for jc in range(n):
            m = jc + n * kc
            big = (n - 1) + n * (jc + n * kc)
            neighbor[big, 1], nbr_face[big, 1], bc[big, 1] = m, -1, BC_MORTAR
            for it in range(rz):
                for is_ in range(ry):
                    jf, kf = ry * jc + is_, rz * kc + it
                    small = Ea + 0 + fd[0] * (jf + fd[1] * kf)
                    slot = is_ + 2 * it if mtype == MORTAR_FOUR else (is_ if ry == 2 else it)
                    mortar[m, 1 + slot], mortar[m, 5 + slot] = small, 0
                    neighbor[small, 0], nbr_face[small, 0], bc[small, 0] = big, 1, BC_INTERNAL
    lo = np.zeros((Ea + Eb, 3))
    h = np.zeros((Ea + Eb, 3))
    for blk, (dims, off, base) in enumerate(((A.dims, (0.0, 0.0, 0.0), 0),
                                             (fd, (1.0, 0.0, 0.0), Ea))):
        e = np.arange(dims[0] * dims[1] * dims[2])
        ijk = (e % dims[0], (e // dims[0]) % dims[1], e // (dims[0] * dims[1]))
        for d in range(3):
            h[base + e, d] = 1.0 / dims[d]
            lo[base + e, d] = off[d] + ijk[d] / dims[d]
    return Mesh(Ea + Eb, ngeo, xgeo, neighbor, nbr_face, bc, shift, dims=(3 * n, n, n),
                lo=(0.0, 0.0, 0.0), hi=(2.0, 1.0, 1.0), warp=warp, amp=amp,
                extra=dict(elem_lo=lo, elem_h=h, split=split), mortar=mortar)


def _element_points(mesh: Mesh, ref: torch.Tensor, elem: torch.Tensor):
    """Analytic physical position of reference points ref[..., 3] in elements
    elem[...] (straight lattice map followed by the warp)."""
    if "elem_lo" in mesh.extra:
        # blocks of different resolution: per-element lower corner and size
        lo = torch.as_tensor(mesh.extra["elem_lo"], device=elem.device)[elem.long()]
        h = torch.as_tensor(mesh.extra["elem_h"], device=elem.device)[elem.long()]
        X, Y, Z = (lo[..., d] + 0.5 * (ref[..., d] + 1.0) * h[..., d] for d in range(3))
        return _warp_torch(mesh.warp, mesh.amp, X, Y, Z)
    nx, ny, nz = mesh.dims
    i = elem % nx
    j = (elem // nx) % ny
    k = elem // (nx * ny)
    h = [(mesh.hi[d] - mesh.lo[d]) / mesh.dims[d] for d in range(3)]
    X = mesh.lo[0] + (i.to(torch.float64) + 0.5 * (ref[..., 0] + 1.0)) * h[0]
    Y = mesh.lo[1] + (j.to(torch.float64) + 0.5 * (ref[..., 1] + 1.0)) * h[1]
    Z = mesh.lo[2] + (k.to(torch.float64) + 0.5 * (ref[..., 2] + 1.0)) * h[2]
    return _warp_torch(mesh.warp, mesh.amp, X, Y, Z)


def node_positions(mesh: Mesh, N: int, node_type: int, device="cpu"):
    """Physical positions [nelem][n^3] of the DG solution nodes (i fastest)."""
    xs = torch.tensor(solution_nodes(N, node_type), dtype=torch.float64, device=device)
    n = N + 1
    rk, rj, ri = torch.meshgrid(xs, xs, xs, indexing="ij")
    ref = torch.stack([ri, rj, rk], dim=-1).reshape(1, n ** 3, 3)
    elem = torch.arange(mesh.nelem, device=device).view(-1, 1)
    return _element_points(mesh, ref, elem)


def _conservative(rho, u, v, w, p):
    rhoE = p / (GAMMA - 1.0) + 0.5 * rho * (u * u + v * v + w * w)
    return torch.stack([rho, rho * u, rho * v, rho * w, rhoE], dim=1)


def tgv_velocity(x, y, z):
    tp = 2.0 * math.pi
    u = torch.sin(tp * x) * torch.cos(tp * y) * torch.cos(tp * z)
    v = -torch.cos(tp * x) * torch.sin(tp * y) * torch.cos(tp * z)
    return u, v, torch.zeros_like(u)


def fluid_tgv(mesh: Mesh, N: int, node_type: int = 0, device="cpu") -> np.ndarray:
    X, Y, Z = node_positions(mesh, N, node_type, device)
    u, v, w = tgv_velocity(X, Y, Z)
    fp = 4.0 * math.pi
    p = P0 + (torch.cos(fp * X) + torch.cos(fp * Y)) * (torch.cos(fp * Z) + 2.0) / 16.0
    return _conservative(torch.ones_like(X), u, v, w, p)


def fluid_uniform(mesh: Mesh, N: int, u0=(1.0, 0.0, 0.0), node_type: int = 0,
                  device="cpu") -> torch.Tensor:
    X, Y, Z = node_positions(mesh, N, node_type, device)
    one = torch.ones_like(X)
    return _conservative(one, u0[0] * one, u0[1] * one, u0[2] * one, P0 * one)


def fluid_linear_shear(mesh: Mesh, N: int, y0: float, node_type: int = 0, device="cpu"):
    """rho = p = 1, u = (y / y0, 0, 0): the high-order time-integration case."""
    X, Y, Z = node_positions(mesh, N, node_type, device)
    one = torch.ones_like(X)
    zero = torch.zeros_like(X)
    return _conservative(one, Y / y0, zero, zero, one)


def fluid_linear(mesh: Mesh, N: int, A, u0, rho_slope, node_type: int = 0, device="cpu"):
    """rho = 1.2 + rho_slope . x, u = u0 + A x, p = 1 at the DG nodes: a flow
    with a constant velocity gradient A (vorticity and shear for the lift)."""
    X, Y, Z = node_positions(mesh, N, node_type, device)
    A = torch.as_tensor(np.asarray(A), dtype=torch.float64, device=device)
    u0 = [float(c) for c in u0]
    rho = 1.2 + rho_slope[0] * X + rho_slope[1] * Y + rho_slope[2] * Z
    u = [u0[i] + A[i, 0] * X + A[i, 1] * Y + A[i, 2] * Z for i in range(3)]
    return _conservative(rho, u[0], u[1], u[2], torch.ones_like(X))


def fluid_polynomial(mesh: Mesh, N: int, coeffs: np.ndarray, node_type: int = 0, device="cpu"):
    """U_v(x) = sum_{abc} coeffs[v,a,b,c] X^a Y^b Z^c with X,Y,Z the physical
    node coordinates (straight meshes: degree <= N per axis in xi too)."""
    X, Y, Z = node_positions(mesh, N, node_type, device)
    nv, na, nb, nc = coeffs.shape
    out = torch.zeros((mesh.nelem, nv) + X.shape[1:], dtype=torch.float64, device=device)
    cf = torch.as_tensor(coeffs, dtype=torch.float64, device=device)
    for a in range(na):
        for b in range(nb):
            for c in range(nc):
                mono = X ** a * Y ** b * Z ** c
                out += cf[:, a, b, c].view(1, nv, 1) * mono.unsqueeze(1)
    return out


def _channel_modes(seed: int, nmodes: int = 24, kmax: float = 8.0):
    rng = np.random.default_rng(seed)
    modes = []
    while len(modes) < nmodes:
        kx = int(rng.integers(-8, 9))
        kz = 2 * int(rng.integers(-4, 5))
        ky = 0.5 * math.pi * int(rng.integers(0, 6))
        kk = math.sqrt(kx * kx + ky * ky + kz * kz)
        if kk == 0.0 or kk > kmax:
            continue
        amp = kk ** (-5.0 / 6.0) / kk
        phase = rng.uniform(0.0, 2.0 * math.pi, size=3)
        dirv = rng.normal(size=3)
        modes.append((kx, ky, kz, amp, phase, dirv / np.linalg.norm(dirv)))
    return modes


def channel_velocity(x, y, z, seed: int = 0, urms: float | None = 0.1, scale: float | None = None):
    """Poiseuille flow plus a divergence-free, wall-vanishing perturbation
    u' = curl((1-y^2)^2 psi).  Returns (u, v, w, scale) where scale is the
    factor that set the perturbation's rms (reuse it to sample elsewhere)."""
    modes = _channel_modes(seed)
    s = (1.0 - y * y) ** 2
    ds = -4.0 * y * (1.0 - y * y)
    # psi components and their gradients
    up = torch.zeros_like(x)
    vp = torch.zeros_like(x)
    wp = torch.zeros_like(x)
    for kx, ky, kz, amp, phase, dirv in modes:
        for comp in range(3):
            arg = kx * x + ky * y + kz * z + phase[comp]
            c = amp * dirv[comp] * torch.cos(arg)
            sn = -amp * dirv[comp] * torch.sin(arg)
            # A_comp = s * c ; grad A_comp = (s*sn*kx, ds*c + s*sn*ky, s*sn*kz)
            gx, gy, gz = s * sn * kx, ds * c + s * sn * ky, s * sn * kz
            if comp == 0:      # A_x contributes  (0, dAx/dz, -dAx/dy)
                vp = vp + gz
                wp = wp - gy
            elif comp == 1:    # A_y contributes  (-dAy/dz, 0, dAy/dx)
                up = up - gz
                wp = wp + gx
            else:              # A_z contributes  (dAz/dy, -dAz/dx, 0)
                up = up + gy
                vp = vp - gx
    if scale is None:
        rms = torch.sqrt((up * up + vp * vp + wp * wp).mean() / 3.0).item()
        scale = (urms / rms) if rms > 0 else 0.0
    return (1.0 - y * y) + scale * up, scale * vp, scale * wp, scale


def fluid_channel(mesh: Mesh, N: int, node_type: int = 0, seed: int = 0, device="cpu",
                  chunk: int = 1 << 15):
    """Channel state at the DG nodes; returns (U [nelem][5][n^3], scale)."""
    n3 = (N + 1) ** 3
    out = torch.empty((mesh.nelem, 5, n3), dtype=torch.float64, device=device)
    # fix the rms scale on the first chunk of elements (or all, if small)
    scale = None
    sub = Mesh(**{**mesh.__dict__})
    for e0 in range(0, mesh.nelem, chunk):
        e1 = min(mesh.nelem, e0 + chunk)
        xs = torch.tensor(solution_nodes(N, node_type), dtype=torch.float64, device=device)
        rk, rj, ri = torch.meshgrid(xs, xs, xs, indexing="ij")
        ref = torch.stack([ri, rj, rk], dim=-1).reshape(1, n3, 3)
        elem = torch.arange(e0, e1, device=device).view(-1, 1)
        X, Y, Z = _element_points(sub, ref, elem)
        u, v, w, scale = channel_velocity(X, Y, Z, seed=seed, scale=scale)
        out[e0:e1] = _conservative(torch.ones_like(X), u, v, w, P0 * torch.ones_like(X))
    return out, scale


def seed_particles(mesh: Mesh, P: int, seed: int = 0, margin: float = 0.01, device="cpu",
                   elem: np.ndarray | None = None):
    """Positions [P][3] (float64) and owning elements [P] (int32)."""
    gen = torch.Generator(device="cpu").manual_seed(seed)
    if elem is None:
        el = torch.randint(0, mesh.nelem, (P,), generator=gen)
    else:
        el = torch.as_tensor(elem).long()
    ref = (torch.rand((P, 3), generator=gen, dtype=torch.float64) * 2.0 - 1.0) * (1.0 - margin)
    el = el.to(device)
    ref = ref.to(device)
    X, Y, Z = _element_points(mesh, ref, el)
    return torch.stack([X, Y, Z], dim=1), el.to(torch.int32)


def stokes_diameters(P: int, st_lo: float, st_hi: float, mu: float, rho_p: float, seed: int,
                     U: float = 1.0, L: float = 1.0, device="cpu"):
    """Diameters from Stokes numbers drawn log-uniform in [st_lo, st_hi]:
    tau = St L / U and d = sqrt(18 mu tau / rho_p)."""
    gen = torch.Generator(device="cpu").manual_seed(seed + 7919)
    lst = math.log(st_lo) + torch.rand(P, generator=gen, dtype=torch.float64) * (
        math.log(st_hi) - math.log(st_lo))
    tau = torch.exp(lst) * L / U
    return torch.sqrt(18.0 * mu * tau / rho_p).to(device)


# ----------------------------------------------------------------------------
# the five workloads
# ----------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    mesh: Mesh
    N: int
    node_type: int
    U: torch.Tensor          # [nelem][5][n^3] float64
    x: torch.Tensor          # [P][3] float64
    v: torch.Tensor          # [P][3] float64
    d: torch.Tensor          # [P] float64
    elem: torch.Tensor       # [P] int32
    mu: float
    rho_p: float
    drag_law: int
    dt: float
    nsteps: int
    precision: str           # "fp64" | "fp32"
    guess: str = "trilinear"
    info: dict = field(default_factory=dict)


def tgv_box(n_side=8, N=3, P=10_000, nsteps=100, seed=0, device="cpu", precision="fp64",
            d=1e-4, rho_p=1000.0, mu=1e-5, dt=1e-3) -> Workload:
    """Periodic unit cube of n_side^3 straight hexahedra, Taylor-Green vortex on
    Gauss nodes, particles at rest, Stokes drag."""
    mesh = box_mesh((n_side,) * 3, (0.0, 0.0, 0.0), (1.0, 1.0, 1.0), 1)
    U = fluid_tgv(mesh, N, 0, device)
    x, el = seed_particles(mesh, P, seed, device=device)
    v = torch.zeros_like(x)
    dd = torch.full((P,), d, dtype=torch.float64, device=device)
    return Workload("tgv_box", mesh, N, 0, U, x, v, dd, el, mu, rho_p, 0, dt, nsteps, precision)


def curved_channel(dims=(32, 32, 32), ngeo=2, N=5, P=1_000_000, nsteps=200, seed=0,
                   device="cpu", precision="fp64", st=(0.1, 100.0), rho_p=1000.0, mu=1e-5,
                   dt=1e-3, guess="trilinear", mass_loading=None) -> Workload:
    """Curved channel with synthetic turbulence, Schiller-Naumann drag, particles
    start at the analytic fluid velocity.  With mass_loading set, all particles
    share one diameter chosen so that P m_p = mass_loading * rho * volume."""
    mesh = channel_mesh(dims, ngeo)
    U, scale = fluid_channel(mesh, N, 0, seed, device)
    x, el = seed_particles(mesh, P, seed, device=device)
    u, v, w, _ = channel_velocity(x[:, 0], x[:, 1], x[:, 2], seed=seed, scale=scale)
    vel = torch.stack([u, v, w], dim=1)
    if mass_loading is None:
        dd = stokes_diameters(P, st[0], st[1], mu, rho_p, seed, device=device)
    else:
        vol = 2.0 * math.pi * 2.0 * math.pi
        mp = mass_loading * 1.0 * vol / P
        dval = (6.0 * mp / (math.pi * rho_p)) ** (1.0 / 3.0)
        dd = torch.full((P,), dval, dtype=torch.float64, device=device)
    return Workload("curved_channel", mesh, N, 0, U, x, vel, dd, el, mu, rho_p, 1, dt, nsteps,
                    precision, guess=guess, info=dict(scale=scale))


def mortar_tgv(n=3, ngeo=2, split="st", N=4, P=400, nsteps=40, seed=0, device="cpu",
               precision="fp64", st=(0.1, 100.0), rho_p=1000.0, mu=1e-5, dt=2e-3,
               warp=None, amp=0.04) -> Workload:
    """Non-conforming two-block box (mortar_box) with the Taylor-Green vortex of
    period 1 and Schiller-Naumann drag; particles start at the fluid velocity
    times 4 plus N(0, 1.5^2) noise, in the elements next to the mortar
    interface at x = 1, so that they cross it both ways and hit the walls
    within a few steps."""
    warp = warp or ("mortar_trilinear" if ngeo == 1 else "mortar_poly")
    mesh = mortar_box(n, ngeo, split, amp, warp)
    U = fluid_tgv(mesh, N, 0, device)
    # owners drawn from the elements next to the interface: the last column of
    # the coarse block and the first two of the fine one
    lo = mesh.extra["elem_lo"]
    near = np.flatnonzero((lo[:, 0] >= 1.0 - 1.0 / n - 1e-12) & (lo[:, 0] < 1.0 + 1.0 / n - 1e-12))
    pick = torch.randint(0, len(near), (P,), generator=torch.Generator().manual_seed(seed + 1))
    x, el = seed_particles(mesh, P, seed, device=device, elem=near[pick.numpy()])
    u, v, w = tgv_velocity(x[:, 0], x[:, 1], x[:, 2])
    gen = torch.Generator(device="cpu").manual_seed(seed + 104729)
    vel = 4.0 * torch.stack([u, v, w], dim=1) + 1.5 * torch.randn(
        (P, 3), generator=gen, dtype=torch.float64).to(device)
    dd = stokes_diameters(P, st[0], st[1], mu, rho_p, seed, device=device)
    return Workload(f"mortar_{split}", mesh, N, 0, U, x, vel, dd, el, mu, rho_p, 1, dt, nsteps,
                    precision)


def batched_box_params(nbox=128, seed=1, side_range=(8, 40), N_set=(3, 4, 5, 6, 7),
                       P_range=(1_000, 1_000_000), scale_P=1.0):
    """(side, N, P) of each box of batched_boxes, in order, without building them."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(nbox):
        side = int(round(math.exp(rng.uniform(math.log(side_range[0]), math.log(side_range[1])))))
        N = int(rng.choice(N_set))
        P = int(round(math.exp(rng.uniform(math.log(P_range[0]), math.log(P_range[1])))))
        out.append((side, N, max(1, int(P * scale_P))))
    return out


def batched_boxes(nbox=128, seed=1, device="cpu", side_range=(8, 40), N_set=(3, 4, 5, 6, 7),
                  P_range=(1_000, 1_000_000), nsteps=50, dt=1e-3, scale_P=1.0, select=None):
    """Independent periodic TGV boxes of uneven size: side log-uniform in
    side_range, N uniform in N_set, particle count log-uniform in P_range.
    select: indices of the boxes to build (all if None); a box is the same
    whichever others are built."""
    params = batched_box_params(nbox, seed, side_range, N_set, P_range, scale_P)
    out = []
    for b in (range(nbox) if select is None else select):
        side, N, P = params[b]
        wl = tgv_box(side, N, P, nsteps, seed=seed * 100003 + b, device=device,
                     precision="fp32", dt=dt)
        wl.name = f"box{b}"
        out.append(wl)
    return out
