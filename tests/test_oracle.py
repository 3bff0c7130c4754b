"""Pins of the FP64 oracle against what the paper and mathematics fix.

Each test checks the oracle against something other than itself: a library
routine (numpy Gauss nodes), a closed form (polynomial reproduction, analytic
maps, the Stokes relaxation, the analytic high-order time-integration case of
Sec. 5.1, bounce counts between planar walls), an invariant (order conditions
of the RK table, partition of unity, speed under reflection, particle count)
or brute force (point location over every element).

Readings pinned here (arXiv 2211.05458):
  * Sec. 5.1 prints x_1,ex with t^3 where integrating its own v_1,ex gives t^3/3;
    the integrated form is used.
  * Sec. 5.1 starts the particle on the domain boundary y = 2; the domain is
    shifted to y in [0.5, 4.5] (flow u = y/2 unchanged) so the start is interior.
"""
import math

import numpy as np
import pytest
from scipy import optimize

import oracle
from paper_2211_05458_gb300 import workloads as W


def _np(t):
    return t.detach().cpu().numpy() if hasattr(t, "detach") else np.asarray(t)


# ---------------------------------------------------------------------------
# nodes and Lagrange basis
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n", range(1, 10))
def test_gauss_nodes_match_numpy(n):
    assert np.allclose(oracle.nodes(0, n), np.polynomial.legendre.leggauss(n)[0], atol=1e-15)


@pytest.mark.parametrize("n", range(2, 10))
def test_gll_nodes_are_legendre_derivative_roots(n):
    c = np.zeros(n)
    c[-1] = 1.0
    roots = np.sort(np.polynomial.legendre.Legendre(c).deriv().roots().real)
    ref = np.concatenate([[-1.0], roots, [1.0]])
    assert np.allclose(oracle.nodes(1, n), ref, atol=1e-14)


@pytest.mark.parametrize("kind", [0, 1, 2])
@pytest.mark.parametrize("n", [2, 4, 6, 8])
def test_lagrange_reproduces_polynomials(kind, n):
    xn = oracle.nodes(kind, n)
    rng = np.random.default_rng(n + 10 * kind)
    for x in rng.uniform(-1, 1, 5):
        for j in range(n):
            assert abs(oracle.lagrange(xn, j, xn[j]) - 1.0) < 1e-14
            for m in range(n):
                if m != j:
                    assert abs(oracle.lagrange(xn, j, xn[m])) < 1e-14
        for k in range(n):
            val = sum(xn[i] ** k * oracle.lagrange(xn, i, x) for i in range(n))
            der = sum(xn[i] ** k * oracle.lagrange_deriv(xn, i, x) for i in range(n))
            assert abs(val - x ** k) < 1e-12
            assert abs(der - (k * x ** (k - 1) if k else 0.0)) < 1e-10


# ---------------------------------------------------------------------------
# element map and Newton inverse
# ---------------------------------------------------------------------------

def _poly_warp(x, y, z, amp):
    return x, y + amp * x * x * (1.0 + z), z + 0.5 * amp * x * y


def _poly_warp_jac(x, y, z, amp):
    return np.array([[1.0, 0.0, 0.0],
                     [2 * amp * x * (1 + z), 1.0, amp * x * x],
                     [0.5 * amp * y, 0.5 * amp * x, 1.0]])


def _straight(mesh, e, xi):
    nx, ny, nz = mesh.dims
    i, j, k = e % nx, (e // nx) % ny, e // (nx * ny)
    h = [(mesh.hi[d] - mesh.lo[d]) / mesh.dims[d] for d in range(3)]
    ijk = (i, j, k)
    return np.array([mesh.lo[d] + (ijk[d] + 0.5 * (xi[d] + 1)) * h[d] for d in range(3)]), h


@pytest.mark.parametrize("ngeo", [2, 3])
def test_elem_map_matches_polynomial_warp(ngeo):
    amp = 0.3
    mesh = W.box_mesh((2, 3, 2), (0.0, -1.0, 0.5), (1.0, 1.0, 1.5), ngeo,
                      periodic=(False, False, False), warp="poly", amp=amp)
    orc = oracle.Oracle(mesh.as_dict())
    rng = np.random.default_rng(1)
    for _ in range(20):
        e = int(rng.integers(mesh.nelem))
        xi = rng.uniform(-1, 1, 3)
        xs, h = _straight(mesh, e, xi)
        ref = np.array(_poly_warp(*xs, amp))
        Jref = _poly_warp_jac(*xs, amp) @ np.diag([0.5 * hd for hd in h])
        x, J = orc.elem_map(e, xi)
        assert np.allclose(x, ref, atol=1e-13)
        assert np.allclose(J, Jref, atol=1e-12)
        ok, xin, it = orc.newton(e, ref)
        assert ok and np.allclose(xin, xi, atol=1e-12)


def test_newton_affine_closed_form():
    mesh = W.box_mesh((3, 2, 4), (0.0, 0.0, 0.0), (1.5, 1.0, 2.0), 1)
    orc = oracle.Oracle(mesh.as_dict())
    rng = np.random.default_rng(2)
    for _ in range(20):
        e = int(rng.integers(mesh.nelem))
        xi = rng.uniform(-1, 1, 3)
        x, _ = _straight(mesh, e, xi)
        ok, xin, it = orc.newton(e, x)
        assert ok and it <= 2
        assert np.allclose(xin, xi, atol=1e-14)


@pytest.mark.parametrize("ngeo", [2, 3])
def test_newton_curved_roundtrip_and_residual(ngeo):
    mesh = W.channel_mesh((4, 4, 3), ngeo, amp=0.2)
    orc = oracle.Oracle(mesh.as_dict())
    rng = np.random.default_rng(3)
    for _ in range(30):
        e = int(rng.integers(mesh.nelem))
        xi = rng.uniform(-1, 1, 3)
        x, _ = orc.elem_map(e, xi)
        ok, xin, it = orc.newton(e, x)
        assert ok
        assert np.max(np.abs(xin - xi)) < 1e-12
        xr, _ = orc.elem_map(e, xin)
        assert np.max(np.abs(xr - x)) < 1e-13


# ---------------------------------------------------------------------------
# interpolation
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("node_type", [0, 1])
@pytest.mark.parametrize("N", [1, 3, 5, 7])
def test_interp_exact_for_tensor_polynomials(N, node_type):
    mesh = W.box_mesh((2, 2, 2), (0.0, 0.0, 0.0), (1.0, 2.0, 0.5), 1)
    rng = np.random.default_rng(N)
    coeffs = rng.normal(size=(5, N + 1, N + 1, N + 1))
    U = W.fluid_polynomial(mesh, N, coeffs, node_type)
    orc = oracle.Oracle(mesh.as_dict())
    orc.set_fluid(N, node_type, _np(U))
    for _ in range(10):
        e = int(rng.integers(mesh.nelem))
        xi = rng.uniform(-1, 1, 3)
        x, _ = _straight(mesh, e, xi)
        ref = np.zeros(5)
        for a in range(N + 1):
            for b in range(N + 1):
                for c in range(N + 1):
                    ref += coeffs[:, a, b, c] * x[0] ** a * x[1] ** b * x[2] ** c
        got = orc.interp(e, xi)
        assert np.allclose(got, ref, rtol=1e-11, atol=1e-11)


# ---------------------------------------------------------------------------
# LSERK coefficients
# ---------------------------------------------------------------------------

def butcher_from_2n(A, B):
    """Butcher tableau (a, b, c) of the 2N-storage scheme du <- A_i du + dt F,
    u <- u + B_i du, stage i evaluated at the state after stage i-1."""
    s = len(A)

    def w(j, l):  # prod_{m=j+1}^{l} A_m
        p = 1.0
        for m in range(j + 1, l + 1):
            p *= A[m]
        return p
    a = np.zeros((s, s))
    for k in range(s):
        for j in range(k):
            a[k, j] = sum(B[l] * w(j, l) for l in range(j, k))
    b = np.array([sum(B[l] * w(j, l) for l in range(j, s)) for j in range(s)])
    return a, b, a.sum(axis=1)


def test_lserk_order_conditions():
    A, B, C = oracle.lserk_coeffs()
    a, b, c = butcher_from_2n(A, B)
    assert np.allclose(c, C, atol=1e-14)
    conds = [
        (b.sum(), 1.0), (b @ c, 1 / 2), (b @ c ** 2, 1 / 3), (b @ (a @ c), 1 / 6),
        (b @ c ** 3, 1 / 4), (b @ (c * (a @ c)), 1 / 8), (b @ (a @ c ** 2), 1 / 12),
        (b @ (a @ (a @ c)), 1 / 24),
    ]
    for got, want in conds:
        assert abs(got - want) < 1e-14


# ---------------------------------------------------------------------------
# drag + LSERK against closed forms
# ---------------------------------------------------------------------------

def _uniform_setup(u0, N=2, dims=(4, 4, 4)):
    mesh = W.box_mesh(dims, (0.0, 0.0, 0.0), (1.0, 1.0, 1.0), 1)
    U = W.fluid_uniform(mesh, N, u0)
    orc = oracle.Oracle(mesh.as_dict())
    orc.set_fluid(N, 0, _np(U))
    return mesh, orc


def test_stokes_relaxation_discrete_and_analytic():
    u0 = np.array([0.7, -0.2, 0.4])
    mesh, orc = _uniform_setup(u0)
    mu, rho_p, d = 1e-5, 1000.0, 1e-4
    tau = rho_p * d * d / (18 * mu)
    dt, nsteps = 5e-3, 40
    p = oracle.make_params(mu=mu, rho_p=rho_p, drag_law=0)
    x0 = np.array([[0.43, 0.51, 0.47]])
    out = orc.push(p, x0, np.zeros((1, 3)), [d], orc.locate_bruteforce(x0[0])[:1],
                   nsteps=nsteps, dt=dt)
    A, B, _ = oracle.lserk_coeffs()
    a, b, _ = butcher_from_2n(A, B)
    z = -dt / tau
    R = 1.0 + sum(z ** k * (b @ np.linalg.matrix_power(a, k - 1) @ np.ones(5)) for k in range(1, 6))
    want = u0 + R ** nsteps * (0.0 - u0)
    assert np.allclose(out["v"][0], want, rtol=0, atol=1e-13)
    t = dt * nsteps
    exact = u0 * (1 - math.exp(-t / tau))
    assert np.allclose(out["v"][0], exact, atol=1e-6)
    xex = x0[0] + u0 * t - tau * u0 * (1 - math.exp(-t / tau))
    shift = np.round(out["x"][0] - xex)  # periodic wraps of the unit cube
    assert np.allclose(out["x"][0] - shift, xex, atol=1e-6)


def _golden(name):
    """key = value fixture under tests/golden (lists comma-separated)."""
    import os
    out = {}
    for line in open(os.path.join(os.path.dirname(__file__), "golden", name)):
        line = line.split("#", 1)[0].strip()
        if line:
            k, v = (t.strip() for t in line.split("=", 1))
            vals = [float(x) for x in v.split(",")]
            out[k] = vals if len(vals) > 1 else vals[0]
    return out


_SEC51 = _golden("sec5_1_high_order_time_integration.txt")


@pytest.mark.parametrize("St", _SEC51["stokes_numbers"])
def test_high_order_time_integration_case(St):
    """Sec. 5.1 with the printed setup: linear shear u = (y/y0, 0, 0), gravity
    in y, drag on x only (f_D = 1), the printed time steps; the oracle's
    position error against the analytic solution falls with the printed
    order 4."""
    G = _SEC51
    y0, g = G["y0"], G["gravity"][1]
    n = int(G["elements_per_direction"])
    lo, hi = G["domain_lo"], G["domain_hi"]
    # reading: the printed start (0, 2, 0.5) lies on the boundary of [0,2]^3;
    # the particle starts at (0.5, 2, 0.5) in [0,2] x [0.5,4.5] x [0,2], with
    # elements of the printed size (the flow u = y/2 is unchanged)
    shift = 0.5
    mesh = W.box_mesh((n, 2 * n, n), (lo[0], lo[1] + shift, lo[2]),
                      (hi[0], hi[1] + shift + (hi[1] - lo[1]), hi[2]), 1,
                      periodic=(False, False, False))
    N = 3
    U = W.fluid_linear_shear(mesh, N, y0)
    orc = oracle.Oracle(mesh.as_dict())
    orc.set_fluid(N, 0, _np(U))
    # Eq. stokesnumber with u_c = y/2 = 1 at the start and L_c = 2
    tau = St * G["characteristic_length"] / 1.0
    mu, rho_p = 1e-5, 1000.0
    d = math.sqrt(18 * mu * tau / rho_p)
    p = oracle.make_params(mu=mu, rho_p=rho_p, drag_law=0, g=(0, g, 0), mask=(1, 0, 0))
    x0 = np.array([[G["start_position"][0] + shift, G["start_position"][1],
                    G["start_position"][2]]])
    e0 = orc.locate_bruteforce(x0[0])
    assert len(e0) == 1
    T = G["t_end"]
    c = g / (2 * y0)
    x1 = x0[0, 0] + T - tau * (1 - math.exp(-T / tau)) + c * (
        T ** 3 / 3 - T ** 2 * tau + 2 * tau ** 2 * T + 2 * tau ** 3 * (math.exp(-T / tau) - 1))
    v1 = 1 - math.exp(-T / tau) + c * (T ** 2 - 2 * T * tau + 2 * tau ** 2 -
                                        2 * tau ** 2 * math.exp(-T / tau))
    errs = []
    dts = sorted(G["dt"], reverse=True)
    for dt in dts:
        out = orc.push(p, x0, np.zeros((1, 3)), [d], e0, nsteps=int(round(T / dt)), dt=dt)
        assert out["status"][0] & oracle.ST_FROZEN == 0
        assert abs(out["x"][0, 1] - (y0 + 0.5 * g * T ** 2)) < 1e-12
        assert abs(out["v"][0, 1] - g * T) < 1e-12
        errs.append(abs(out["x"][0, 0] - x1))
        if dt == dts[-1]:
            assert abs(out["v"][0, 0] - v1) < 1e-6
    errs = np.array(errs)
    slopes = np.log2(errs[:-1] / errs[1:])
    assert errs[-1] < 1e-7
    # observed order between successive halvings, where rounding (~1e-12) does
    # not yet dominate the truncation error
    usable = errs[1:] > 5e-11
    assert usable.sum() >= 1
    order = G["order"]
    assert np.all(slopes[usable] > order - 0.4) and np.all(slopes[usable] < order + 0.6), (
        errs, slopes)


def test_schiller_naumann_terminal_velocity():
    """Quiescent fluid, gravity: v_t solves f_D(Re(v_t)) v_t / tau = |g|."""
    mesh, orc = _uniform_setup(np.zeros(3), N=1, dims=(3, 3, 3))
    mu, rho_p, d, g = 1e-5, 1000.0, 1e-4, 9.81
    tau = rho_p * d * d / (18 * mu)
    p = oracle.make_params(mu=mu, rho_p=rho_p, drag_law=1, g=(0, -g, 0))

    def resid(vt):
        re = vt * d / mu
        return (1 + 0.15 * re ** 0.687) * vt / tau - g
    vt = optimize.brentq(resid, 1e-6, 10.0, xtol=1e-15)
    x0 = np.array([[0.3, 0.6, 0.7]])
    out = orc.push(p, x0, np.zeros((1, 3)), [d], orc.locate_bruteforce(x0[0]),
                   nsteps=1000, dt=1e-3)
    assert out["status"][0] & oracle.ST_FROZEN == 0
    assert abs(out["v"][0, 1] + vt) < 1e-6 * vt
    assert abs(out["v"][0, 0]) < 1e-14 and abs(out["v"][0, 2]) < 1e-14


def test_stokes_settling_with_buoyancy():
    """Eq. theory:maxey with gravity on m_p - m_f: quiescent fluid of density
    rho_f (fluid_uniform: rho = 1), Stokes drag; the settling speed tends to
    Stokes' terminal velocity g tau_p (1 - rho_f/rho_p)."""
    mesh, orc = _uniform_setup(np.zeros(3), N=1, dims=(3, 3, 3))
    mu, rho_p, d, g = 1e-5, 2.5, 2e-5, 9.81   # light particles: buoyancy 40 %
    tau = rho_p * d * d / (18 * mu)
    x0 = np.array([[0.3, 0.6, 0.7]])
    el = orc.locate_bruteforce(x0[0])
    vt = g * tau * (1 - 1.0 / rho_p)
    for b, want in [(1, vt), (0, g * tau)]:
        p = oracle.make_params(mu=mu, rho_p=rho_p, g=(0, -g, 0), buoyancy=b)
        out = orc.push(p, x0, np.zeros((1, 3)), [d], el, nsteps=200, dt=1e-5)
        assert abs(out["v"][0, 1] + want) < 1e-9 * want, (b, out["v"][0, 1], want)


# ---------------------------------------------------------------------------
# tracking
# ---------------------------------------------------------------------------

def _fold_periodic(x, lo, hi):
    L = hi - lo
    return lo + np.mod(x - lo, L)


def test_free_stream_straight_lines_through_curved_faces():
    mesh = W.channel_mesh((6, 4, 3), 3, amp=0.2)
    N = 2
    u0 = np.array([1.0, 0.0, 0.3])
    U = W.fluid_uniform(mesh, N, u0)
    orc = oracle.Oracle(mesh.as_dict())
    orc.set_fluid(N, 0, _np(U))
    x, el = W.seed_particles(mesh, 40, seed=5, margin=0.05)
    x = _np(x)
    v = np.tile(u0, (len(x), 1))
    d = np.full(len(x), 1e-4)
    p = oracle.make_params(drag_law=0)
    dt, nsteps = 0.01, 100
    out = orc.push(p, x, v, d, _np(el), nsteps=nsteps, dt=dt)
    T = dt * nsteps
    want = x + u0 * T
    want[:, 0] = _fold_periodic(want[:, 0], 0.0, 2 * math.pi)
    want[:, 2] = _fold_periodic(want[:, 2], 0.0, math.pi)
    got = out["x"].copy()
    got[:, 0] = _fold_periodic(got[:, 0], 0.0, 2 * math.pi)
    got[:, 2] = _fold_periodic(got[:, 2], 0.0, math.pi)
    assert np.allclose(got, want, atol=1e-10)
    assert np.all(out["status"] & oracle.ST_FROZEN == 0)
    assert np.all(out["hits"] == 0)
    ncheck = 0
    for i in range(len(x)):
        if out["status"][i] & oracle.ST_NEAR_FACE:
            continue
        owners = orc.locate_bruteforce(out["x"][i], tol=1e-10)
        assert list(owners) == [out["elem"][i]]
        ncheck += 1
    assert ncheck >= 35


@pytest.mark.parametrize("ngeo,N", [(2, 3), (3, 4)])
def test_turbulent_channel_owner_is_bruteforce_owner(ngeo, N):
    mesh = W.channel_mesh((5, 4, 3), ngeo, amp=0.1)
    U, scale = W.fluid_channel(mesh, N, 0, seed=3)
    orc = oracle.Oracle(mesh.as_dict())
    orc.set_fluid(N, 0, _np(U))
    P = 60
    x, el = W.seed_particles(mesh, P, seed=9)
    x = _np(x)
    rng = np.random.default_rng(4)
    vel = rng.normal(size=(P, 3)) * 2.0  # fast, so that walls and faces are crossed
    d = np.full(P, 4e-3)
    p = oracle.make_params(drag_law=1)
    out = orc.push(p, x, vel, d, _np(el), nsteps=30, dt=5e-3)
    assert np.all(out["status"] & oracle.ST_FROZEN == 0)  # nothing lost: count conserved
    assert out["hits"].sum() > 0
    ncheck = 0
    for i in range(P):
        if out["status"][i] & oracle.ST_NEAR_FACE:
            continue
        owners = orc.locate_bruteforce(out["x"][i], tol=1e-10)
        assert list(owners) == [out["elem"][i]], (i, owners, out["elem"][i])
        assert -1.0 <= out["x"][i, 1] <= 1.0
        ncheck += 1
    assert ncheck >= P - 3


def test_reflection_between_planar_walls_matches_unfolded_ray():
    mesh = W.channel_mesh((4, 5, 3), 2, amp=0.15)
    N = 1
    U = W.fluid_uniform(mesh, N, (0.0, 0.0, 0.0))
    orc = oracle.Oracle(mesh.as_dict())
    orc.set_fluid(N, 0, _np(U))
    P = 30
    x, el = W.seed_particles(mesh, P, seed=11)
    x = _np(x)
    rng = np.random.default_rng(12)
    vel = rng.normal(size=(P, 3)) * 3.0
    p = oracle.make_params(mask=(0.0, 0.0, 0.0))
    dt, nsteps = 0.01, 60
    out = orc.push(p, x, vel, np.full(P, 1e-4), _np(el), nsteps=nsteps, dt=dt)
    T = dt * nsteps
    yu = x[:, 1] + vel[:, 1] * T
    nb = np.abs(np.floor((yu + 1) / 2) - np.floor((x[:, 1] + 1) / 2)).astype(int)
    yf = np.mod(yu + 1, 4.0)
    yf = np.where(yf > 2.0, 4.0 - yf, yf) - 1.0
    speed0 = np.linalg.norm(vel, axis=1)
    speed1 = np.linalg.norm(out["v"], axis=1)
    assert np.allclose(speed1, speed0, rtol=1e-14 * 8)
    ok = out["status"] & oracle.ST_NEAR_FACE == 0
    assert ok.sum() >= P - 2
    assert np.array_equal(out["hits"][ok], nb[ok])
    assert np.allclose(out["x"][ok, 1], yf[ok], atol=1e-11)
    assert np.allclose(np.abs(out["v"][ok, 1]), np.abs(vel[ok, 1]), rtol=1e-13)


def test_reflection_on_curved_walls_conserves_speed():
    mesh = W.channel_mesh((4, 3, 3), 3, amp=0.15, curved_walls=True)
    N = 1
    U = W.fluid_uniform(mesh, N, (0.0, 0.0, 0.0))
    orc = oracle.Oracle(mesh.as_dict())
    orc.set_fluid(N, 0, _np(U))
    P = 20
    x, el = W.seed_particles(mesh, P, seed=13)
    rng = np.random.default_rng(14)
    vel = rng.normal(size=(P, 3)) * 3.0
    p = oracle.make_params(mask=(0.0, 0.0, 0.0))
    out = orc.push(p, _np(x), vel, np.full(P, 1e-4), _np(el), nsteps=60, dt=0.01)
    assert np.all(out["status"] & oracle.ST_FROZEN == 0)
    assert out["hits"].sum() >= 10
    assert np.allclose(np.linalg.norm(out["v"], axis=1), np.linalg.norm(vel, axis=1),
                       rtol=1e-13)
    for i in range(P):
        if out["status"][i] & oracle.ST_NEAR_FACE:
            continue
        assert list(orc.locate_bruteforce(out["x"][i])) == [out["elem"][i]]


def test_planar_face_hit_matches_plane_formula():
    """Sec. 3.2.4: alpha = (x_m.n - x.n) / (t.n) for a planar face."""
    mesh = W.box_mesh((2, 2, 2), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0), 1)
    orc = oracle.Oracle(mesh.as_dict())
    rng = np.random.default_rng(15)
    for _ in range(20):
        x0 = rng.uniform(0.05, 0.45, 3)
        x1 = x0 + rng.normal(size=3) * 0.6
        td = (x1 - x0) / np.linalg.norm(x1 - x0)
        for f in range(6):
            ctrl = orc.face_ctrl(0, f)
            xm = ctrl.reshape(-1, 3).mean(axis=0)
            nrm = np.zeros(3)
            nrm[f // 2] = 1.0
            if abs(td @ nrm) < 1e-6:
                continue
            alpha = (xm @ nrm - x0 @ nrm) / (td @ nrm)
            hits = orc.face_hits(0, f, x0, x1)
            inside = alpha > 0 and alpha <= np.linalg.norm(x1 - x0)
            xh = x0 + alpha * td
            others = [k for k in range(3) if k != f // 2]
            inside = inside and all(0.0 <= xh[k] <= 0.5 for k in others)
            if inside:
                assert len(hits) == 1 and abs(hits[0, 0] - alpha) < 1e-13
            elif alpha > 0.01 and alpha < np.linalg.norm(x1 - x0) - 0.01 and all(
                    0.01 <= xh[k] <= 0.49 or xh[k] < -0.01 or xh[k] > 0.51 for k in others):
                assert len(hits) == 0


@pytest.mark.parametrize("warp,ngeo", [("none_twist", 1), ("channel", 3)])
def test_face_hits_lie_on_face_and_ray(warp, ngeo):
    if warp == "none_twist":
        mesh = W.box_mesh((1, 1, 1), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0), 1,
                          periodic=(False, False, False))
        mesh.xgeo[0, 7] += np.array([0.15, 0.2, -0.1])  # twisted: bilinear faces
    else:
        mesh = W.channel_mesh((3, 2, 2), ngeo, amp=0.3)
    orc = oracle.Oracle(mesh.as_dict())
    rng = np.random.default_rng(16)
    nh = 0
    for _ in range(40):
        e = int(rng.integers(mesh.nelem))
        x0, _ = orc.elem_map(e, rng.uniform(-0.9, 0.9, 3))
        x1, _ = orc.elem_map(e, rng.uniform(-1, 1, 3) * 2.5)
        td = (x1 - x0) / np.linalg.norm(x1 - x0)
        for f in range(6):
            for alpha, s, t in orc.face_hits(e, f, x0, x1):
                xi = [0.0, 0.0, 0.0]
                fixed = f // 2
                free = [k for k in range(3) if k != fixed]
                xi[fixed] = 1.0 if f & 1 else -1.0
                xi[free[0]], xi[free[1]] = s, t
                xf, _ = orc.elem_map(e, np.array(xi))
                assert np.linalg.norm(x0 + alpha * td - xf) < 1e-12
                nh += 1
    assert nh >= 30


def test_bezier_control_points_reproduce_face():
    mesh = W.channel_mesh((2, 2, 2), 3, amp=0.3)
    orc = oracle.Oracle(mesh.as_dict())
    from math import comb
    rng = np.random.default_rng(17)
    for f in range(6):
        ctrl = orc.face_ctrl(1, f)  # [k][m][xyz]
        p = ctrl.shape[0] - 1
        for _ in range(5):
            s, t = rng.uniform(-1, 1, 2)
            u, w = 0.5 * (s + 1), 0.5 * (t + 1)
            bu = [comb(p, m) * u ** m * (1 - u) ** (p - m) for m in range(p + 1)]
            bw = [comb(p, k) * w ** k * (1 - w) ** (p - k) for k in range(p + 1)]
            pt = sum(bw[k] * bu[m] * ctrl[k, m] for k in range(p + 1) for m in range(p + 1))
            xi = [0.0, 0.0, 0.0]
            free = [k for k in range(3) if k != f // 2]
            xi[f // 2] = 1.0 if f & 1 else -1.0
            xi[free[0]], xi[free[1]] = s, t
            xf, _ = orc.elem_map(1, np.array(xi))
            assert np.allclose(pt, xf, atol=1e-13)


# ---------------------------------------------------------------------------
# two-way coupling source
# ---------------------------------------------------------------------------

def test_deposit_partition_of_unity_sign_and_kronecker():
    mesh = W.box_mesh((2, 2, 2), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0), 1)
    N = 3
    U = W.fluid_uniform(mesh, N, (0.0, 0.0, 0.0))
    orc = oracle.Oracle(mesh.as_dict())
    orc.set_fluid(N, 0, _np(U))
    mu, rho_p = 1e-5, 1000.0
    p = oracle.make_params(mu=mu, rho_p=rho_p, drag_law=1)
    rng = np.random.default_rng(18)
    P = 50
    x, el = W.seed_particles(mesh, P, seed=18)
    vel = rng.normal(size=(P, 3))
    d = rng.uniform(1e-4, 1e-3, P)
    S = orc.deposit(p, _np(x), vel, d, _np(el))
    # force on each particle from the closed forms of Sec. 2.2 (fluid at rest)
    tau = rho_p * d * d / (18 * mu)
    re = np.linalg.norm(vel, axis=1) * d / mu
    fD = 1 + 0.15 * re ** 0.687
    mp = rho_p * math.pi * d ** 3 / 6
    F = (mp * fD / tau)[:, None] * (0.0 - vel)
    assert np.allclose(S[:, :3, :].sum(axis=(0, 2)), -F.sum(axis=0), rtol=1e-12, atol=1e-18)
    assert np.allclose(S[:, 3, :].sum(), -(F * vel).sum(), rtol=1e-12)
    # fluid gains momentum along the particle's motion (action = -reaction)
    assert np.all(np.sign(-F) == np.sign(vel))
    # a particle sitting on a solution node deposits on that node only
    xn = W.gauss_nodes(N + 1)
    xi = np.array([xn[1], xn[2], xn[0]])
    xs, _ = _straight(mesh, 3, xi)
    S1 = orc.deposit(p, xs[None], np.array([[0.3, 0.0, 0.0]]), [5e-4], [3])
    big = np.abs(S1[3]).max()
    nz = np.flatnonzero(np.abs(S1[3, 0]) > 1e-12 * big)
    n = N + 1
    assert list(nz) == [1 + n * (2 + n * 0)]
    assert np.all(np.flatnonzero(np.abs(S1[3]).max(axis=0) > 1e-12 * big) == nz)
    assert np.abs(S1[[0, 1, 2, 4, 5, 6, 7]]).max() == 0.0


# ---------------------------------------------------------------------------
# learned-guess network (no counterpart in the paper)
# ---------------------------------------------------------------------------

def test_mlp_gradient_matches_central_differences():
    n = oracle.mlp_nparams()
    assert n == 64 * 51 + 64 + 2 * (64 * 64 + 64) + 3 * 64 + 3
    rng = np.random.default_rng(19)
    theta = rng.normal(size=n) * 0.2
    inp = rng.normal(size=(7, 51))
    tgt = rng.normal(size=(7, 3))
    loss, grad = oracle.mlp_loss_grad(theta, inp, tgt)
    idx = rng.choice(n, 60, replace=False)
    idx = np.concatenate([idx, [n - 1, n - 4, 64 * 51 + 3]])
    for i in idx:
        h = 1e-5
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (oracle.mlp_loss_grad(tp, inp, tgt)[0] - oracle.mlp_loss_grad(tm, inp, tgt)[0]) / (2 * h)
        assert abs(fd - grad[i]) <= 1e-7 * max(1.0, abs(fd)) + 1e-9, (i, fd, grad[i])


def test_mlp_forward_special_cases():
    n = oracle.mlp_nparams()
    theta = np.zeros(n)
    theta[-3:] = [0.5, -1.0, 2.0]
    out = oracle.mlp_forward(theta, np.ones((2, 51)))
    assert np.allclose(out, [[0.5, -1.0, 2.0]] * 2, atol=0)
    # single path: x0 -> unit weights -> GELU(1) = Phi(1) = 0.8413447460685429
    theta = np.zeros(n)
    W1, b1 = 0, 64 * 51
    W2 = b1 + 64
    W3 = W2 + 64 * 64 + 64
    W4 = W3 + 64 * 64 + 64
    theta[W1 + 0] = 1.0
    theta[W2 + 0] = 1.0
    theta[W3 + 0] = 1.0
    theta[W4 + 0] = 1.0
    gelu = lambda z: 0.5 * z * (1 + math.erf(z / math.sqrt(2)))
    x = np.zeros((1, 51))
    x[0, 0] = 1.0
    out = oracle.mlp_forward(theta, x)
    assert abs(gelu(1.0) - 0.8413447460685429) < 1e-15
    assert abs(out[0, 0] - gelu(gelu(gelu(1.0)))) < 1e-15


def test_adam_first_step_closed_form():
    theta = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    m, v = np.zeros(3), np.zeros(3)
    oracle.adam(theta, g, m, v, 1, lr=0.01, eps=1e-8)
    # first step: m_hat = g, v_hat = g^2 => step = lr g / (|g| + eps)
    want = np.array([1.0, -2.0, 0.5]) - 0.01 * g / (np.abs(g) + 1e-8)
    assert np.allclose(theta, want, atol=1e-15)


def test_mlp_features_affine_element():
    mesh = W.box_mesh((2, 2, 2), (0.0, 0.0, 0.0), (1.0, 2.0, 1.0), 3)
    orc = oracle.Oracle(mesh.as_dict())
    rng = np.random.default_rng(20)
    for _ in range(5):
        e = int(rng.integers(mesh.nelem))
        xi = rng.uniform(-1, 1, 3)
        x, _ = _straight(mesh, e, xi)
        f = orc.mlp_features(e, x)
        assert np.allclose(f[:3], xi, atol=1e-14)
        assert np.abs(f[3:]).max() < 1e-13


def test_mlp_features_quadratic_warp_closed_form():
    """The 48 deviation features on elements of the warp y' = y + A x^2 (1 + z):
    the trilinear map of the corners reproduces y and interpolates x^2 (1 + z)
    linearly in x, so a node's y deviation is A (1 + z)(x - x0)(x - x1) (lattice
    coordinates), divided by the y length of the element's xi2-edges."""
    A = 0.05
    mesh = W.box_mesh((2, 2, 2), (0.0, 0.0, 0.0), (1.0, 2.0, 1.0), 3,
                      periodic=(False, False, False), warp="poly", amp=A)
    orc = oracle.Oracle(mesh.as_dict())
    hx, hy, hz = 0.5, 1.0, 0.5
    for e in range(mesh.nelem):
        i, k = e % 2, e // 4
        x0, z0 = i * hx, k * hz
        f = orc.mlp_features(e, mesh.xgeo[e].mean(axis=0))
        want = []
        for c in range(4):
            for b in range(4):
                for a in range(4):
                    nb = (a in (0, 3)) + (b in (0, 3)) + (c in (0, 3))
                    if nb not in (1, 2):
                        continue
                    x, z = x0 + a * hx / 3, z0 + c * hz / 3
                    want.append(A * (1 + z) * (x - x0) * (x - x0 - hx) / hy)
        assert len(want) == 48
        assert np.allclose(f[3:], want, rtol=0, atol=1e-14), e
        assert np.abs(np.asarray(want)).max() > 1e-3


@pytest.mark.parametrize("n", range(2, 9))
def test_quadrature_weights(n):
    # Gauss weights against numpy; GLL weights integrate polynomials of degree 2n-3
    assert np.allclose(oracle.quad_weights(0, n), np.polynomial.legendre.leggauss(n)[1], atol=1e-14)
    x, w = oracle.nodes(1, n), oracle.quad_weights(1, n)
    for k in range(2 * n - 2):
        exact = (1 - (-1) ** (k + 1)) / (k + 1)
        assert abs(np.dot(w, x ** k) - exact) < 1e-13


def test_nearest_dof_projection_conserves_and_picks_nearest_node():
    """Sec. 2.3: P{a} = a / V_ijk at the nearest node; sum_ijk S_ijk V_ijk = a."""
    mesh = W.channel_mesh((3, 3, 2), 2, amp=0.2)
    N = 3
    U = W.fluid_uniform(mesh, N, (0.3, 0.0, 0.1))
    orc = oracle.Oracle(mesh.as_dict())
    orc.set_fluid(N, 0, _np(U))
    p = oracle.make_params(drag_law=1)
    rng = np.random.default_rng(21)
    P = 40
    x, el = W.seed_particles(mesh, P, seed=21)
    vel = rng.normal(size=(P, 3))
    d = rng.uniform(1e-4, 1e-3, P)
    S = orc.deposit_nearest(p, _np(x), vel, d, _np(el))
    Sl = orc.deposit(p, _np(x), vel, d, _np(el))  # Lagrange form: nodal amounts
    n = N + 1
    xn, wq = oracle.nodes(0, n), oracle.quad_weights(0, n)
    # node volumes from the element map
    tot = np.zeros(4)
    for e in range(mesh.nelem):
        for k in range(n):
            for j in range(n):
                for i in range(n):
                    s_ = S[e, :, i + n * (j + n * k)]
                    if not np.any(s_):
                        continue
                    _, J = orc.elem_map(e, np.array([xn[i], xn[j], xn[k]]))
                    tot += s_ * wq[i] * wq[j] * wq[k] * abs(np.linalg.det(J))
    assert np.allclose(tot, Sl.sum(axis=(0, 2)), rtol=1e-12)
    # one particle: exactly one non-zero node, the nearest in reference space
    ok, xi, _ = orc.newton(int(el[0]), _np(x[0]))
    S1 = orc.deposit_nearest(p, _np(x[:1]), vel[:1], d[:1], _np(el[:1]))
    nzn = np.flatnonzero(np.abs(S1[int(el[0])]).max(axis=0))
    idx = [int(np.argmin(np.abs(xn - xi[q]))) for q in range(3)]
    assert list(nzn) == [idx[0] + n * (idx[1] + n * idx[2])]


def test_dt_violations_threshold():
    """Sec. 2.3: dt <= 2.75 tau_p, tau_p = rho_p d^2 / (18 mu): a particle just
    inside the limit passes, one just outside fails."""
    p = oracle.make_params(mu=1e-5, rho_p=1000.0)
    d = np.array([1e-4, 2e-4, 5e-5])
    taus = 1000.0 * d ** 2 / 18e-5
    dt = 2.75 * taus[0]
    assert oracle.dt_violations(p, d, dt * (1 - 1e-12)) == 1  # only the 5e-5 particle
    assert oracle.dt_violations(p, d, dt * (1 + 1e-12)) == 2
    assert oracle.dt_violations(p, d, 0.0) == 0


# ---------------------------------------------------------------------------
# extra force models (Sec. 2.2): velocity gradient, Saffman lift, Haider-Levenspiel
# ---------------------------------------------------------------------------

def test_velocity_gradient_exact_for_linear_velocity_on_curved_mesh():
    """u = u0 + A x with a linearly varying density on a mesh warped by a
    polynomial of degree 2 per axis (NGeo = 2 reproduces it): rho u has degree
    <= 4 per reference direction <= N, so the interpolant is exact and du/dx = A
    (the quotient-rule term u_i drho/dxi is needed for that)."""
    mesh = W.box_mesh((3, 3, 2), (0, 0, 0), (1, 1, 1), 2, periodic=(False, False, False),
                      warp="poly", amp=0.1)
    N = 5
    rng = np.random.default_rng(8)
    A = rng.normal(size=(3, 3))
    U = W.fluid_linear(mesh, N, A, (0.3, -0.2, 0.1), (0.05, -0.03, 0.02))
    orc = oracle.Oracle(mesh.as_dict())
    orc.set_fluid(N, 0, _np(U))
    for e in rng.choice(mesh.nelem, 6, replace=False):
        xi = rng.uniform(-1, 1, 3)
        G = orc.velocity_gradient(int(e), xi)
        assert np.allclose(G, A, atol=1e-10), (G, A)


def test_saffman_lift_direction_and_low_reynolds_limit():
    """Shear u = (g y, 0, 0), particle at rest above the axis: the lift points to
    the faster fluid (+y); for Re_p -> 0, C_S -> 1 and the force is Saffman's
    6.46 mu a^2 |u - v| sqrt(|w| / nu), a = d/2."""
    mu, rho, g, d = 1e-5, 1.0, 3.0, 1e-6
    p = oracle.make_params(mu=mu, lift=1)
    rel = np.array([g * 3e-4, 0.0, 0.0])         # u - v at y = 3e-4
    w = np.array([0.0, 0.0, -g])                  # curl of (g y, 0, 0)
    F = oracle.saffman_force(p, rho, rel, w, d)
    assert F[1] > 0 and abs(F[0]) < 1e-30 and abs(F[2]) < 1e-30
    a, nu = d / 2, mu / rho
    classic = 6.46 * mu * a ** 2 * np.linalg.norm(rel) * np.sqrt(abs(g) / nu)
    re = rho * np.linalg.norm(rel) * d / mu
    assert re < 1e-3
    assert abs(F[1] - classic) <= 1e-3 * classic
    # no shear or no slip: no lift
    assert np.all(oracle.saffman_force(p, rho, rel, np.zeros(3), d) == 0)
    assert np.all(oracle.saffman_force(p, rho, np.zeros(3), w, d) == 0)


def test_saffman_mei_branches_meet_at_re_40():
    """0.0524 sqrt(40) = 0.3314: above Re_p = 40 the correction is
    0.3314 sqrt(th) at the branch point (th = d |w| / (2 |u - v|))."""
    mu, rho = 1e-5, 1.0
    p = oracle.make_params(mu=mu, lift=1)
    d = 1e-3
    rn = 40.0001 * mu / (rho * d)
    rel = np.array([0.0, rn, 0.0])
    w = np.array([0.0, 0.0, 2 * rn * 0.1 / d])   # th = 0.1
    F = np.linalg.norm(oracle.saffman_force(p, rho, rel, w, d))
    k = 6.46 / 4 * d * d * np.sqrt(rho * mu / np.linalg.norm(w)) * np.linalg.norm(w) * rn
    assert abs(F / k - 0.3314 * np.sqrt(0.1)) < 2e-4


def test_haider_levenspiel_sphere_limits():
    """phi = 1: Stokes limit f_D -> 1, within 10% of Schiller-Naumann (an
    independent sphere correlation) over 0.1 <= Re <= 800, and the Newton
    regime C_D = 24 f_D / Re ~ 0.44 at Re = 1e4."""
    hl = oracle.make_params(drag_law=2, sphericity=1.0)
    sn = oracle.make_params(drag_law=1)
    assert abs(oracle.drag_factor(hl, 1e-8) - 1.0) < 1e-4
    for re in np.geomspace(0.1, 800, 25):
        a, b = oracle.drag_factor(hl, re), oracle.drag_factor(sn, re)
        assert abs(a / b - 1) < 0.10, (re, a, b)
    cd = 24 * oracle.drag_factor(hl, 1e4) / 1e4
    assert 0.40 < cd < 0.48
    # less spherical particles drag more at the same Re
    lo = oracle.make_params(drag_law=2, sphericity=0.6)
    assert oracle.drag_factor(lo, 100.0) > oracle.drag_factor(hl, 100.0)


def test_push_with_lift_drifts_toward_faster_fluid_and_deposits_it():
    """Shear u = (g (y - 0.5), 0, 0) in a periodic box, particle released at
    rest at y > 0.5 (it lags the fluid): without lift its y stays fixed; with
    lift it drifts to larger y, toward the faster fluid.  The y-momentum source
    of the deposit is then minus the lift force."""
    mesh = W.box_mesh((4, 4, 4), (0, 0, 0), (1, 1, 1), 1)
    N = 3
    g = 2.0
    A = np.zeros((3, 3))
    A[0, 1] = g
    U = W.fluid_linear(mesh, N, A, (-0.5 * g, 0.0, 0.0), (0.0, 0.0, 0.0))
    orc = oracle.Oracle(mesh.as_dict())
    orc.set_fluid(N, 0, _np(U))
    x = np.array([[0.4, 0.8, 0.5]])
    el = np.array([int(0.4 * 4) + 4 * (int(0.8 * 4) + 4 * int(0.5 * 4))], np.int32)
    v = np.zeros((1, 3))
    d = np.array([2e-4])
    common = dict(mu=1e-5, rho_p=1000.0, drag_law=1)
    r0 = orc.push(oracle.make_params(**common), x, v, d, el, nsteps=20, dt=1e-3)
    r1 = orc.push(oracle.make_params(lift=1, **common), x, v, d, el, nsteps=20, dt=1e-3)
    assert r0["x"][0, 1] == x[0, 1]
    assert r1["x"][0, 1] > x[0, 1] and r1["v"][0, 1] > 0
    # deposit: with lift the y source is -F_S,y (drag has no y component here)
    S0 = orc.deposit(oracle.make_params(**common), x, v, d, el)
    S1 = orc.deposit(oracle.make_params(lift=1, **common), x, v, d, el)
    assert abs(S0[:, 1].sum()) < 1e-30
    rel = np.array([g * (0.8 - 0.5), 0.0, 0.0])
    FS = oracle.saffman_force(oracle.make_params(lift=1, **common), 1.2, rel,
                              np.array([0.0, 0.0, -g]), d[0])
    assert abs(S1[:, 1].sum() + FS[1]) <= 1e-9 * abs(FS[1])


# ---------------------------------------------------------------------------
# non-conforming (mortar) faces, Sec. 3.2.3
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("split,ngeo", [("st", 1), ("st", 3), ("s", 2), ("t", 2)])
def test_mortar_small_faces_tile_the_big_face(split, ngeo):
    """The generator's small faces are the parts of the big face that the row
    layout names: mapped into the big element, the corners of small face k lie
    on the big face (xi_1 = +1) at the corners of its half / quarter."""
    warp = "mortar_trilinear" if ngeo == 1 else "mortar_poly"
    mesh = W.mortar_box(2, ngeo, split, warp=warp)
    orc = oracle.Oracle(mesh.as_dict())
    g = ngeo + 1
    p = oracle.make_params()
    for m, row in enumerate(mesh.mortar):
        big = int(np.flatnonzero((mesh.bc[:, 1] == W.BC_MORTAR) & (mesh.neighbor[:, 1] == m))[0])
        ns = 4 if row[0] == W.MORTAR_FOUR else 2
        for q in range(ns):
            es, fs = int(row[1 + q]), int(row[5 + q])
            assert fs == 0
            X = mesh.xgeo[es].reshape(g, g, g, 3)  # [c][b][a]
            i_s = q % 2 if row[0] != W.MORTAR_T else 0
            i_t = (q // 2 if row[0] == W.MORTAR_FOUR else (q if row[0] == W.MORTAR_T else 0))
            for cb, cc in ((0, 0), (g - 1, 0), (0, g - 1), (g - 1, g - 1)):
                ok, xi, _ = orc.newton(big, X[cc, cb, 0], p)
                assert ok
                assert abs(xi[0] - 1.0) < 1e-12
                s_lo, s_hi = (-1.0, 1.0) if row[0] == W.MORTAR_T else ((-1.0, 0.0), (0.0, 1.0))[i_s]
                t_lo, t_hi = (-1.0, 1.0) if row[0] == W.MORTAR_S else ((-1.0, 0.0), (0.0, 1.0))[i_t]
                want_s = s_lo if cb == 0 else s_hi
                want_t = t_lo if cc == 0 else t_hi
                assert abs(xi[1] - want_s) < 1e-12 and abs(xi[2] - want_t) < 1e-12


def _mortar_run(wl):
    orc = oracle.Oracle(wl.mesh.as_dict())
    orc.set_fluid(wl.N, 0, _np(wl.U))
    p = oracle.make_params(mu=wl.mu, rho_p=wl.rho_p, drag_law=wl.drag_law)
    out = orc.push(p, _np(wl.x), _np(wl.v), _np(wl.d), _np(wl.elem), nsteps=wl.nsteps, dt=wl.dt)
    return orc, out


@pytest.mark.parametrize("split,ngeo", [("st", 1), ("st", 3), ("s", 2), ("t", 2), ("st", 4)])
def test_mortar_tracking_owner_is_bruteforce_owner(split, ngeo):
    """Tracking across big -> small and small -> big mortar faces ends every
    particle in the one element that brute-force location finds."""
    wl = W.mortar_tgv(3, ngeo, split, N=3, P=120, nsteps=40)
    orc, out = _mortar_run(wl)
    assert np.all(out["status"] & oracle.ST_FROZEN == 0)
    Ea = 27
    start_a, end_a = _np(wl.elem) < Ea, out["elem"] < Ea
    assert np.sum(start_a & ~end_a) >= 5 and np.sum(~start_a & end_a) >= 5
    ncheck = 0
    for i in range(len(out["elem"])):
        if out["status"][i] & oracle.ST_NEAR_FACE:
            continue
        owners = orc.locate_bruteforce(out["x"][i], tol=1e-10)
        assert list(owners) == [out["elem"][i]], (i, owners, out["elem"][i])
        ncheck += 1
    assert ncheck >= 110


def test_mortar_entry_face_is_found_by_intersection_not_by_row_order():
    """The small face entered is the one the ray crosses (the search on the
    small faces), so permuting a row's small faces changes nothing."""
    wl = W.mortar_tgv(3, 2, "st", N=3, P=120, nsteps=40)
    _, out = _mortar_run(wl)
    perm = wl.mesh.mortar.copy()
    perm[:, 1:5] = perm[:, [4, 3, 2, 1]]
    perm[:, 5:9] = perm[:, [8, 7, 6, 5]]
    wl.mesh.mortar = perm
    _, out2 = _mortar_run(wl)
    for k in ("x", "v", "elem", "hits", "status"):
        assert np.array_equal(out[k], out2[k]), k
