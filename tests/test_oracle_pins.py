"""Pins of the FP64 CPU oracle to what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: exactness on
polynomial data, closed forms, invariants of the scheme, an independent numpy
solve of the least-squares problems, brute force on tiny meshes, the exact
translating vortex, and the paper's observed convergence orders."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2607_10809_b300 import inputs as I

GL = 0.28867513459481288225  # sqrt(3)/6


# ---------------------------------------------------------------- helpers
def interior_cells(nbr, rings=2):
    """Cells whose `rings`-ring neighbourhood contains no boundary cell."""
    bad = np.any(nbr < 0, axis=1)
    for _ in range(rings):
        grow = bad.copy()
        for j in range(3):
            nb = nbr[:, j]
            ok = nb >= 0
            grow[ok] |= bad[nb[ok]]
        bad = grow
    return np.nonzero(~bad)[0]


def quad_fn(q):
    def f(x, y):
        return (q[0] + q[1] * x + q[2] * y + q[3] * x * x + q[4] * x * y + q[5] * y * y)[None]
    return f


def quad_jet(q, x, y):
    return np.array([q[0] + q[1] * x + q[2] * y + q[3] * x * x + q[4] * x * y + q[5] * y * y,
                     q[1] + 2 * q[3] * x + q[4] * y, q[2] + q[4] * x + 2 * q[5] * y,
                     2 * q[3] + 0 * x, q[4] + 0 * x, 2 * q[5] + 0 * x])


# ---------------------------------------------------------------- constants
def test_linear_weights_are_the_papers_and_sum_to_one(golden_dir):
    g = json.load(open(os.path.join(golden_dir, "paper_constants.json")))
    gl = g["linear_weights"]["value"]
    o = oracle.Oracle(I.structured_periodic(4, 1.0))
    assert list(o._gl) == gl
    # Eq. pxy is an identity only when the linear weights sum to one
    assert abs(sum(gl) - 1.0) < 1e-15


def test_pxy_identity_linear_weights_give_p1():
    """Eq. pxy: with the nonlinear weights replaced by the linear ones, the
    combination of Eq. recon is p1 itself, for any data."""
    mesh = I.jittered_periodic(6, 1.0, seed=11)
    rng = np.random.default_rng(0)
    U = rng.normal(size=(3, 1, mesh.nt))
    o = oracle.Oracle(mesh, linear_only=True)
    for cell in (0, 17, 40):
        r = o.reconstruct_cell(U, cell)
        np.testing.assert_allclose(r["recon"], r["polys"][0], rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(r["omega"], [0.94, 0.02, 0.02, 0.02], rtol=0, atol=1e-15)


# ---------------------------------------------------------------- reconstruction
def test_p1_reproduces_quadratics_and_p2_p4_linears():
    mesh = I.jittered_box(7, 1.0, seed=3)
    o = oracle.Oracle(mesh)
    nbr, _ = o.neighbors()
    rng = np.random.default_rng(1)
    q = rng.normal(size=6)
    U = I.initial_state(mesh, quad_fn(q), 1)
    for cell in interior_cells(nbr, rings=0)[:12]:
        r = o.reconstruct_cell(U, int(cell))
        gp = r["gp"]
        exact = quad_jet(q, gp[:, 0], gp[:, 1]).T      # [6 points, 6 derivs]
        np.testing.assert_allclose(r["polys"][0], exact, rtol=1e-10, atol=1e-10)
    ql = np.array([q[0], q[1], q[2], 0, 0, 0])
    U = I.initial_state(mesh, quad_fn(ql), 1)
    for cell in interior_cells(nbr, rings=0)[:12]:
        r = o.reconstruct_cell(U, int(cell))
        gp = r["gp"]
        exact = quad_jet(ql, gp[:, 0], gp[:, 1]).T
        for l in range(4):
            np.testing.assert_allclose(r["polys"][l], exact, rtol=1e-10, atol=1e-10)
        # linear data: all indicators equal, kappa = 0, omega = gamma, exact
        np.testing.assert_allclose(r["beta"], r["beta"][0], rtol=1e-9)
        np.testing.assert_allclose(r["omega"], [0.94, 0.02, 0.02, 0.02], rtol=1e-9)
        np.testing.assert_allclose(r["recon"], exact, rtol=1e-10, atol=1e-10)


def _numpy_p1(mesh, U, cell, nbr):
    """Independent solve of Step 1 by the null-space method (scipy), with cell
    means from a collapsed Gauss rule instead of edge midpoints."""
    from scipy.linalg import null_space
    P = mesh.unwrapped()
    u, v, wt = I._tri_rule(5)

    def pts(T):
        return (T[0][None] + u[:, None] * (T[1] - T[0])[None] + v[:, None] * (T[2] - T[0])[None])

    T0 = P[cell]
    A = lambda T: 0.5 * ((T[1, 0] - T[0, 0]) * (T[2, 1] - T[0, 1]) - (T[2, 0] - T[0, 0]) * (T[1, 1] - T[0, 1]))
    A0 = A(T0); h0 = np.sqrt(A0); c0 = T0.mean(axis=0)
    X0 = (pts(T0) - c0) / h0
    M = [(wt * X0[:, 0] ** 2).sum(), (wt * X0[:, 0] * X0[:, 1]).sum(), (wt * X0[:, 1] ** 2).sum()]

    def phis(X):   # phi_1..phi_5 at points X [q, 2]
        xi, et = X[:, 0], X[:, 1]
        return np.stack([xi, et, xi * xi - M[0], xi * et - M[1], et * et - M[2]], axis=1)

    def dphis(X):  # d/dxi and d/deta of phi_1..phi_5
        xi, et = X[:, 0], X[:, 1]
        z, o = 0 * xi, 1 + 0 * xi
        return (np.stack([o, z, 2 * xi, et, z], axis=1), np.stack([z, o, z, xi, 2 * et], axis=1))

    Cm, e, B, d = [], [], [], []
    for j in range(3):
        nb = nbr[cell, j]
        Tn = P[nb]
        Xn = (pts(Tn) - c0) / h0
        An = A(Tn)
        Cm.append((wt[:, None] * phis(Xn)).sum(0))
        e.append(U[0, 0, nb] - U[0, 0, cell])
        dx0, dy0 = dphis(X0); dxn, dyn = dphis(Xn)
        B.append((An * (wt[:, None] * dxn).sum(0) + A0 * (wt[:, None] * dx0).sum(0)) / (An + A0))
        B.append((An * (wt[:, None] * dyn).sum(0) + A0 * (wt[:, None] * dy0).sum(0)) / (An + A0))
        d.append(h0 * (An * U[1, 0, nb] + A0 * U[1, 0, cell]) / (An + A0))
        d.append(h0 * (An * U[2, 0, nb] + A0 * U[2, 0, cell]) / (An + A0))
    Cm, e, B, d = map(np.array, (Cm, e, B, d))
    cp = np.linalg.lstsq(Cm, e, rcond=None)[0]
    N = null_space(Cm)
    z = np.linalg.lstsq(B @ N, d - B @ cp, rcond=None)[0]
    c = cp + N @ z
    return c, c0, h0, M


def test_p1_constrained_least_squares_matches_independent_solve():
    mesh = I.jittered_box(6, 1.0, seed=5)
    o = oracle.Oracle(mesh)
    nbr, _ = o.neighbors()
    rng = np.random.default_rng(2)
    U = rng.normal(size=(3, 1, mesh.nt))    # inconsistent data: the LS part matters
    for cell in interior_cells(nbr, rings=0)[:8]:
        cell = int(cell)
        r = o.reconstruct_cell(U, cell)
        c, c0, h0, M = _numpy_p1(mesh, U, cell, nbr)
        gp = r["gp"]
        xi = (gp[:, 0] - c0[0]) / h0; et = (gp[:, 1] - c0[1]) / h0
        val = U[0, 0, cell] + c[0] * xi + c[1] * et + c[2] * (xi * xi - M[0]) + c[3] * (xi * et - M[1]) + c[4] * (et * et - M[2])
        px = (c[0] + 2 * c[2] * xi + c[3] * et) / h0
        np.testing.assert_allclose(r["polys"][0][:, 0], val, rtol=1e-10, atol=1e-10)
        np.testing.assert_allclose(r["polys"][0][:, 1], px, rtol=1e-10, atol=1e-10)
        # the equality constraints (cell averages on K1..K3) hold exactly
        # (checked through the independent solution having the same values)


def test_smoothness_indicators_formula_on_quadratic():
    """Eq. smoo1 for p1 = Q: |K0| (Qx^2 + Qy^2) + |K0|^2 (Qxx^2 + Qxy^2 + Qyy^2) at the barycenter."""
    mesh = I.jittered_box(6, 1.0, seed=8)
    o = oracle.Oracle(mesh)
    nbr, _ = o.neighbors()
    geo = o.cell_geometry()
    q = np.array([0.3, -1.1, 0.7, 2.0, -0.5, 1.3])
    U = I.initial_state(mesh, quad_fn(q), 1)
    cell = int(interior_cells(nbr, rings=0)[3])
    r = o.reconstruct_cell(U, cell)
    a = geo["area"][cell]; x, y = geo["cx"][cell], geo["cy"][cell]
    J = quad_jet(q, x, y)
    b1 = a * (J[1] ** 2 + J[2] ** 2) + a * a * (J[3] ** 2 + J[4] ** 2 + J[5] ** 2)
    assert abs(r["beta"][0] - b1) < 1e-10 * b1


def test_nonlinear_weights_switch_off_p1_at_a_jump():
    mesh = I.jittered_box(10, 1.0, seed=4)
    fn = lambda x, y: (1.0 + (x > 0.5))[None] * 1.0
    U = I.initial_state(mesh, fn, 1)
    o = oracle.Oracle(mesh)
    nbr, _ = o.neighbors()
    geo = o.cell_geometry()
    # a cell cut by the jump vs a cell far from it
    near = int(np.argmin(np.abs(geo["cx"] - 0.5) + np.abs(geo["cy"] - 0.5)))
    far = int(np.argmin(np.abs(geo["cx"] - 0.2) + np.abs(geo["cy"] - 0.5)))
    rn = o.reconstruct_cell(U, near)
    rf = o.reconstruct_cell(U, far)
    assert rn["omega"][0] < 0.05 * 0.94
    np.testing.assert_allclose(rf["omega"], [0.94, 0.02, 0.02, 0.02], rtol=1e-12)


# ---------------------------------------------------------------- Lax-Wendroff
def test_lw_advection_closed_form():
    rng = np.random.default_rng(3)
    a = (0.7, -1.3)
    for _ in range(5):
        J = rng.normal(size=(6, 1))
        out = oracle.lax_wendroff("advection", J, a=a)
        W, Wx, Wy, Wxx, Wxy, Wyy = J[:, 0]
        Wt = -(a[0] * Wx + a[1] * Wy)
        Wtx = -(a[0] * Wxx + a[1] * Wxy)
        Wty = -(a[0] * Wxy + a[1] * Wyy)
        Wtt = a[0] ** 2 * Wxx + 2 * a[0] * a[1] * Wxy + a[1] ** 2 * Wyy
        np.testing.assert_allclose(out[:, 0], [Wt, Wtx, Wty, Wtt], rtol=1e-14, atol=1e-14)


def test_lw_burgers_closed_form():
    rng = np.random.default_rng(4)
    for _ in range(5):
        J = rng.normal(size=(6, 1))
        out = oracle.lax_wendroff("burgers", J)
        W, Wx, Wy, Wxx, Wxy, Wyy = J[:, 0]
        s = Wx + Wy
        Wt = -W * s
        Wtx = -(Wx * s + W * (Wxx + Wxy))
        Wty = -(Wy * s + W * (Wxy + Wyy))
        Wtt = -(Wt * s + W * (Wtx + Wty))
        np.testing.assert_allclose(out[:, 0], [Wt, Wtx, Wty, Wtt], rtol=1e-13, atol=1e-13)


def euler_jacobians(W, g=1.4):
    """Textbook flux Jacobians of the 2D Euler equations."""
    rho, m, n, E = W
    u, v = m / rho, n / rho
    q2 = u * u + v * v
    p = (g - 1) * (E - 0.5 * rho * q2)
    H = (E + p) / rho
    A = np.array([[0, 1, 0, 0],
                  [-u * u + 0.5 * (g - 1) * q2, (3 - g) * u, -(g - 1) * v, g - 1],
                  [-u * v, v, u, 0],
                  [u * (0.5 * (g - 1) * q2 - H), H - (g - 1) * u * u, -(g - 1) * u * v, g * u]])
    B = np.array([[0, 0, 1, 0],
                  [-u * v, v, u, 0],
                  [-v * v + 0.5 * (g - 1) * q2, -(g - 1) * u, (3 - g) * v, g - 1],
                  [v * (0.5 * (g - 1) * q2 - H), -(g - 1) * u * v, H - (g - 1) * v * v, g * v]])
    return A, B


def test_euler_flux_jacobian_matches_textbook_and_hessian_matches_fd():
    rng = np.random.default_rng(5)
    W = I.euler_from_primitive(np.array(1.2), np.array(0.3), np.array(-0.8), np.array(0.9))
    for _ in range(4):
        a = rng.normal(size=4); b = rng.normal(size=4)
        out = oracle.flux_derivs("euler", W, a, b)
        A, B = euler_jacobians(W)
        np.testing.assert_allclose(out[0], A @ a, rtol=1e-13, atol=1e-13)
        np.testing.assert_allclose(out[1], A @ b, rtol=1e-13, atol=1e-13)
        np.testing.assert_allclose(out[3], B @ a, rtol=1e-13, atol=1e-13)
        h = 1e-5
        Ap, Bp = euler_jacobians(W + h * b); Am, Bm = euler_jacobians(W - h * b)
        np.testing.assert_allclose(out[2], (Ap - Am) @ a / (2 * h), rtol=1e-7, atol=1e-8)
        np.testing.assert_allclose(out[5], (Bp - Bm) @ a / (2 * h), rtol=1e-7, atol=1e-8)


def _fd_jet(fn, x, y, h=2e-3):
    """Value and derivatives up to second order by 4th-order central differences."""
    c1 = np.array([1, -8, 0, 8, -1]) / (12 * h)
    c2 = np.array([-1, 16, -30, 16, -1]) / (12 * h * h)
    s = np.arange(-2, 3) * h
    F = np.array([[fn(x + a, y + b) for b in s] for a in s])   # [5, 5, m]
    W = F[2, 2]
    Wx = np.tensordot(c1, F[:, 2], axes=1); Wy = np.tensordot(c1, F[2, :], axes=1)
    Wxx = np.tensordot(c2, F[:, 2], axes=1); Wyy = np.tensordot(c2, F[2, :], axes=1)
    Wxy = np.einsum("i,j,ijm->m", c1, c1, F)
    return np.stack([W, Wx, Wy, Wxx, Wxy, Wyy])


def test_lw_euler_reproduces_translating_vortex():
    """The isentropic vortex translates with velocity (1, 1): W_t = -(W_x + W_y)
    and W_tt = W_xx + 2 W_xy + W_yy hold exactly, so the Lax-Wendroff procedure
    fed with the exact spatial jet must return them."""
    fn = lambda x, y: I.vortex(np.array(x), np.array(y))
    for (x, y) in ((5.7, 4.6), (4.2, 5.9), (6.1, 6.3)):
        J = _fd_jet(fn, x, y)
        out = oracle.lax_wendroff("euler", J)
        Wt = -(J[1] + J[2]); Wtt = J[3] + 2 * J[4] + J[5]
        Wtx = -(J[3] + J[4]); Wty = -(J[4] + J[5])
        np.testing.assert_allclose(out[0], Wt, rtol=0, atol=2e-9)
        np.testing.assert_allclose(out[1], Wtx, rtol=0, atol=1e-7)
        np.testing.assert_allclose(out[2], Wty, rtol=0, atol=1e-7)
        np.testing.assert_allclose(out[3], Wtt, rtol=0, atol=1e-7)


# ---------------------------------------------------------------- whole step
@pytest.mark.parametrize("time_rule", ["lobatto", "gauss"])
def test_step_exact_for_advected_quadratic_with_linear_weights(time_rule):
    """Quadratic data + linear weights: the reconstruction is exact, the
    second-order Taylor expansion in time is exact, both time rules (three
    Lobatto nodes, two Gauss-Legendre nodes) are exact for the quadratic time
    dependence and two Gauss points are exact on the edges, so one step
    reproduces the exact cell averages of W, W_x, W_y (Eqs. flx, derave2d2)
    away from the boundary."""
    mesh = I.jittered_box(9, 1.0, seed=6)
    q = np.array([0.4, 0.9, -0.6, 1.1, 0.8, -0.7])
    a = (0.8, -0.5)
    o = oracle.Oracle(mesh, "advection", a=a, linear_only=True, time_rule=time_rule)
    nbr, _ = o.neighbors()
    U = I.initial_state(mesh, quad_fn(q), 1)
    dt = 0.04
    Un = o.step(U, dt)
    shifted = lambda x, y: quad_fn(q)(x - a[0] * dt, y - a[1] * dt)
    Ue = I.initial_state(mesh, shifted, 1)
    cells = interior_cells(nbr, rings=2)
    assert cells.size > 20
    np.testing.assert_allclose(Un[:, :, cells], Ue[:, :, cells], rtol=0, atol=1e-12)


@pytest.mark.parametrize("time_rule", ["lobatto", "gauss"])
@pytest.mark.parametrize("eq", ["advection", "burgers", "euler"])
def test_conservation_on_periodic_mesh(eq, time_rule):
    mesh = I.jittered_periodic(8, 10.0 if eq == "euler" else 2.0, seed=12)
    m = 4 if eq == "euler" else 1
    fn = I.vortex if eq == "euler" else (I.advection_sine if eq == "advection" else I.burgers_sine)
    U = I.initial_state(mesh, fn, m)
    o = oracle.Oracle(mesh, eq, time_rule=time_rule)
    area = o.cell_geometry()["area"]
    s0 = (U[0] * area).sum(axis=1)
    for _ in range(4):
        U = o.step(U, 0.5 * o.cfl_dt(U))
    s1 = (U[0] * area).sum(axis=1)
    np.testing.assert_allclose(s1, s0, rtol=1e-13)
    scale = (np.abs(U[1]) * area).sum(axis=1) + (np.abs(U[2]) * area).sum(axis=1)
    assert np.all(np.abs((U[1] * area).sum(axis=1)) < 1e-13 * scale)
    assert np.all(np.abs((U[2] * area).sum(axis=1)) < 1e-13 * scale)


@pytest.mark.parametrize("time_rule", ["lobatto", "gauss"])
@pytest.mark.parametrize("eq", ["advection", "burgers", "euler"])
@pytest.mark.parametrize("kind", ["jittered", "poisson", "box"])
def test_free_stream_preserved(eq, kind, time_rule):
    if kind == "jittered":
        mesh = I.jittered_periodic(7, 1.0, seed=21)
    elif kind == "poisson":
        mesh = I.poisson_delaunay_periodic(1.0, 150, seed=22)
    else:
        mesh = I.jittered_box(7, 1.0, seed=23)
    m = 4 if eq == "euler" else 1
    const = {"advection": [2.5], "burgers": [0.7], "euler": list(I.euler_from_primitive(1.3, 0.4, -0.7, 0.9))}[eq]
    U = np.zeros((3, m, mesh.nt)); U[0] = np.array(const)[:, None]
    o = oracle.Oracle(mesh, eq, time_rule=time_rule)
    U1 = U
    for _ in range(3):
        U1 = o.step(U1, o.cfl_dt(U1))
    np.testing.assert_allclose(U1[0], U[0], rtol=2e-14)
    assert np.abs(U1[1:]).max() < 1e-12


def test_connectivity_matches_brute_force():
    for mesh in (I.jittered_periodic(4, 1.0, seed=1), I.jittered_box(4, seed=2),
                 I.poisson_delaunay_periodic(1.0, 40, seed=3)):
        o = oracle.Oracle(mesh)
        nbr, nbe = o.neighbors()
        T = mesh.tri
        for t in range(mesh.nt):
            for j in range(3):
                a, b = T[t, j], T[t, (j + 1) % 3]
                hits = [(u, k) for u in range(mesh.nt) for k in range(3)
                        if u != t and {T[u, k], T[u, (k + 1) % 3]} == {a, b}]
                if hits:
                    assert len(hits) == 1
                    assert (nbr[t, j], nbe[t, j]) == hits[0]
                else:
                    assert nbr[t, j] == -1 and mesh.bc == 1


def test_dual_numbers_give_the_directional_derivative():
    mesh = I.jittered_periodic(4, 10.0, seed=31)
    U0 = I.initial_state(mesh, I.vortex, 4)
    rng = np.random.default_rng(7)
    dU = rng.normal(size=U0.shape) * np.abs(U0).mean(axis=2, keepdims=True) * 0.1
    o = oracle.Oracle(mesh, "euler")
    dts = [0.05, 0.05, 0.04]
    U1, dU1 = o.run_dual(U0, dU, dts)
    np.testing.assert_allclose(U1, o.run_dts(U0, dts), rtol=1e-15, atol=1e-15)
    h = 1e-6
    fd = (o.run_dts(U0 + h * dU, dts) - o.run_dts(U0 - h * dU, dts)) / (2 * h)
    assert np.abs(fd - dU1).max() < 1e-6 * np.abs(dU1).max()


# ---------------------------------------------------------------- convergence
def _orders(errs):
    return [np.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]


def test_third_order_on_smooth_advection(golden_dir):
    errs = []
    for n in (10, 20, 40, 80):
        mesh = I.config1_mesh(n)
        U0 = I.initial_state(mesh, I.advection_sine, 1)
        U, _ = oracle.Oracle(mesh, "advection").run_to(U0, 0.5)
        We = I.cell_averages(mesh, lambda x, y: I.advection_sine(x - 0.5, y - 0.5), 1)[0]
        errs.append(I.error_norms(mesh, U[0, 0], We)[0])
    paper = json.load(open(os.path.join(golden_dir, "paper_convergence.json")))
    fine = min(min(v["order"][-2:]) for k, v in paper.items() if not k.startswith("_"))
    o = _orders(errs)
    assert o[-1] > fine - 0.1 and o[-1] < 3.3, (errs, o)


def test_gauss_legendre_time_rule_is_third_order_and_close_to_lobatto():
    """The two-node Gauss-Legendre time rule (with the central values of Eq.
    timeflux from a separate Taylor evaluation at t_{n+1}) keeps third order on
    smooth advection, and its errors stay within a factor 2 of the Lobatto
    rule's (both integrate the quadratic Taylor polynomials exactly)."""
    errs = {"lobatto": [], "gauss": []}
    for n in (10, 20, 40):
        mesh = I.config1_mesh(n)
        U0 = I.initial_state(mesh, I.advection_sine, 1)
        We = I.cell_averages(mesh, lambda x, y: I.advection_sine(x - 0.5, y - 0.5), 1)[0]
        for rule in errs:
            U, _ = oracle.Oracle(mesh, "advection", time_rule=rule).run_to(U0, 0.5)
            errs[rule].append(I.error_norms(mesh, U[0, 0], We)[0])
    o = _orders(errs["gauss"])
    assert o[-1] > 2.8 and o[-1] < 3.3, (errs, o)
    ratio = np.array(errs["gauss"]) / np.array(errs["lobatto"])
    assert np.all(ratio > 0.5) and np.all(ratio < 2.0), ratio


def test_burgers_and_vortex_converge():
    T = 0.5 / np.pi
    errs = []
    for n in (10, 20, 40):
        mesh = I.jittered_periodic(n, 4.0, 0.15, seed=2)
        U0 = I.initial_state(mesh, I.burgers_sine, 1)
        U, _ = oracle.Oracle(mesh, "burgers").run_to(U0, T)
        We = I.cell_averages(mesh, lambda x, y: I.burgers_exact(x, y, T), 1)[0]
        errs.append(I.error_norms(mesh, U[0, 0], We)[0])
    assert min(_orders(errs)) > 2.5, errs
    errs = []
    for n in (10, 20, 40):
        mesh = I.jittered_periodic(n, 10.0, 0.15, seed=5)
        U0 = I.initial_state(mesh, I.vortex, 4)
        U, _ = oracle.Oracle(mesh, "euler").run_to(U0, 1.0)
        We = I.cell_averages(mesh, lambda x, y: I.vortex(x, y, 1.0), 4)[0]
        errs.append(I.error_norms(mesh, U[0, 0], We)[0])
    o = _orders(errs)
    # the paper's vortex orders rise from about 2 to 3 over the same range
    assert o[0] > 1.8 and o[1] > 2.3, (errs, o)


# ---------------------------------------------------------------- invariances
@pytest.mark.parametrize("eq", ["burgers", "euler"])
def test_step_independent_of_numbering(eq):
    """The scheme does not depend on how cells are numbered or which vertex
    comes first: reversing the cell order and rotating every triangle's vertex
    list must give the same step (this fixes the symmetric roles of the
    interior and exterior sides in Eq. timeflux and of K1, K2, K3 in Eq.
    nonlinearweight)."""
    L = 10.0 if eq == "euler" else 4.0
    mesh = I.jittered_periodic(6, L, seed=41)
    m = 4 if eq == "euler" else 1
    rng = np.random.default_rng(9)
    fn = I.vortex if eq == "euler" else I.burgers_sine
    U = I.initial_state(mesh, fn, m)
    U[0] *= 1 + 0.05 * rng.random(U[0].shape)     # make the data rough
    perm = np.arange(mesh.nt)[::-1]
    rot = rng.integers(0, 3, mesh.nt)
    tri2 = np.array([np.roll(t, -r) for t, r in zip(mesh.tri[perm], rot[perm])], dtype=np.int32)
    mesh2 = I.Mesh(mesh.xy, tri2, mesh.Lx, mesh.Ly, mesh.bc)
    dt = 0.02
    A = oracle.Oracle(mesh, eq).step(U, dt)
    B = oracle.Oracle(mesh2, eq).step(U[:, :, perm], dt)
    np.testing.assert_allclose(B, A[:, :, perm], rtol=1e-12, atol=1e-12 * np.abs(A).max())


@pytest.mark.parametrize("eq", ["advection", "euler"])
def test_step_invariant_under_scaling_of_space_and_time(eq):
    """x -> s x, t -> s t leaves the conservation law unchanged; the scheme
    (dimensionless least-squares rows, |K0|^|s| in Eq. smoo1, dimensionless
    weights) must then map cell averages of W to themselves and derivative
    averages to 1/s times themselves."""
    s = 3.7
    mesh = I.jittered_periodic(6, 10.0, seed=43)
    mesh_s = I.Mesh(mesh.xy * s, mesh.tri, mesh.Lx * s, mesh.Ly * s, mesh.bc)
    m = 4 if eq == "euler" else 1
    fn = I.vortex if eq == "euler" else (lambda x, y: I.advection_sine(x / 5, y / 5))
    U = I.initial_state(mesh, fn, m)
    rng = np.random.default_rng(10)
    U[0] *= 1 + 0.05 * rng.random(U[0].shape)
    Us = U.copy(); Us[1:] /= s
    dt = 0.03
    A = oracle.Oracle(mesh, eq).step(U, dt)
    B = oracle.Oracle(mesh_s, eq).step(Us, dt * s)
    np.testing.assert_allclose(B[0], A[0], rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(B[1:] * s, A[1:], rtol=1e-10, atol=1e-10 * np.abs(A[1:]).max())


# ---------------------------------------------------------------- scale limiter
def test_scale_limiter_is_identity_on_smooth_positive_data():
    mesh = I.jittered_periodic(10, 10.0, seed=51)
    U = I.initial_state(mesh, I.vortex, 4)
    a = oracle.Oracle(mesh, "euler")
    b = oracle.Oracle(mesh, "euler", positivity=True)
    dt = a.cfl_dt(U)
    np.testing.assert_array_equal(b.step(U, dt), a.step(U, dt))


def _pressure(U):
    rho = U[0, 0]
    return 0.4 * (U[0, 3] - 0.5 * (U[0, 1] ** 2 + U[0, 2] ** 2) / rho)


def test_scale_limiter_keeps_a_riemann_problem_positive_and_conservative():
    """Four-quadrant data whose unlimited step produces negative pressure at once
    (the 'extreme case' of Section 3) stay positive with the limiter, and the
    limited scheme still conserves the total of every component."""
    mesh = I.jittered_box(20, seed=4)
    U0 = I.initial_state(mesh, I.quadrant_fn(I.quadrant_states(4)), 4, nq=4)
    plain = oracle.Oracle(mesh, "euler")
    U = U0
    for _ in range(2):
        U = plain.step(U, plain.cfl_dt(U))
    assert np.nanmin(_pressure(U)) < 0
    lim = oracle.Oracle(mesh, "euler", positivity=True)
    area = lim.cell_geometry()["area"]
    U = U0
    flux_total = 0.0
    for _ in range(30):
        U = lim.step(U, lim.cfl_dt(U))
        assert U[0, 0].min() > 0 and _pressure(U).min() > 0
    # transmissive boundaries let mass out, so compare with a periodic run instead
    pmesh = I.jittered_periodic(12, 1.0, seed=4)
    Up = I.initial_state(pmesh, I.quadrant_fn(I.quadrant_states(4)), 4, nq=4)
    limp = oracle.Oracle(pmesh, "euler", positivity=True)
    ap = limp.cell_geometry()["area"]
    s0 = (Up[0] * ap).sum(axis=1)
    for _ in range(5):
        Up = limp.step(Up, limp.cfl_dt(Up))
    np.testing.assert_allclose((Up[0] * ap).sum(axis=1), s0, rtol=1e-13)


# ---------------------------------------------------------------- LLF viscosity and CFL speed
def _random_euler_states(rng, n):
    rho = rng.uniform(0.05, 3.0, n); u = rng.uniform(-3, 3, n); v = rng.uniform(-3, 3, n)
    p = rng.uniform(0.01, 4.0, n)
    return I.euler_from_primitive(rho, u, v, p).T


def test_llf_viscosity_is_the_spectral_radius_of_the_normal_jacobian():
    """R10: alpha is the largest |eigenvalue| of d(F.n)/dW = A nx + B ny (the
    LLF flux of Section 2.1), checked against the eigenvalues of the textbook
    Euler Jacobians; R12: the CFL speed is its maximum over all directions."""
    rng = np.random.default_rng(17)
    for W in _random_euler_states(rng, 25):
        A, B = euler_jacobians(W)
        th = rng.uniform(0, 2 * np.pi)
        n = (np.cos(th), np.sin(th))
        lam_n, lam_all = oracle.spectral_radius("euler", W, n)
        ref = np.abs(np.linalg.eigvals(A * n[0] + B * n[1])).max()
        assert abs(lam_n - ref) <= 1e-12 * ref, (lam_n, ref)
        thetas = np.linspace(0, 2 * np.pi, 3601)
        over = max(np.abs(np.linalg.eigvals(A * np.cos(t) + B * np.sin(t))).max() for t in thetas[::40])
        dense = max(oracle.spectral_radius("euler", W, (np.cos(t), np.sin(t)))[0] for t in thetas)
        assert over <= lam_all * (1 + 1e-12)
        assert lam_all <= dense * (1 + 1e-5)
    # scalar equations: |f'(u) nx + g'(u) ny|
    for u in rng.uniform(-2, 2, 6):
        th = rng.uniform(0, 2 * np.pi); n = (np.cos(th), np.sin(th))
        lam_n, lam_all = oracle.spectral_radius("burgers", np.array([u]), n)
        assert abs(lam_n - abs(u * (n[0] + n[1]))) <= 1e-15
        assert abs(lam_all - np.sqrt(2) * abs(u)) <= 1e-15
        lam_n, lam_all = oracle.spectral_radius("advection", np.array([u]), n, a=(0.7, -1.3))
        assert abs(lam_n - abs(0.7 * n[0] - 1.3 * n[1])) <= 1e-15
        assert abs(lam_all - np.hypot(0.7, 1.3)) <= 1e-15


# ---------------------------------------------------------------- Eq. nonlinearweight
def _jump_with_flat_side():
    """Data with a jump through the stencil of some cells while one side of it
    is flat: several smoothness indicators vanish there, so the epsilon term
    of Eq. nonlinearweight decides those weights."""
    mesh = I.jittered_box(12, 1.0, seed=8)
    fn = lambda x, y: (1.5 + 0.8 * (x + 0.3 * y > 0.55))[None] * 1.0
    return mesh, I.initial_state(mesh, fn, 1)


def test_nonlinear_weights_invariant_under_scaling_of_the_data():
    """Eq. nonlinearweight is homogeneous: under W -> s W the indicators scale
    by s^2, kappa and both terms of the denominator by s^4 (W_ave is the mean
    of the stencil averages), so the weights do not change (the 1e-30 of
    W_ave is negligible here).  A wrong power of W_ave in either term, or of
    the sum in kappa, breaks the invariance."""
    mesh, U = _jump_with_flat_side()
    o = oracle.Oracle(mesh)
    geo = o.cell_geometry()
    near = np.nonzero(np.abs(geo["cx"] + 0.3 * geo["cy"] - 0.55) < 0.08)[0]
    moved = 0
    for cell in near:
        r1 = o.reconstruct_cell(U, int(cell))
        if np.abs(r1["omega"] - np.array([0.94, 0.02, 0.02, 0.02])).max() > 1e-3:
            moved += 1
        for s in (1e-3, 7.0, 1e3):
            rs = o.reconstruct_cell(s * U, int(cell))
            np.testing.assert_allclose(rs["beta"], s * s * r1["beta"], rtol=1e-12, atol=1e-300)
            np.testing.assert_allclose(rs["omega"], r1["omega"], rtol=1e-13, atol=1e-15)
    assert moved >= 5


def test_nonlinear_weights_hand_case():
    """Eq. nonlinearweight on the oracle's own indicators of one cell, with the
    stencil mean taken from the cell averages: omega_l proportional to
    gamma_l (1 + kappa / (eps W_ave^4 + W_ave^2 beta_l))."""
    mesh, U = _jump_with_flat_side()
    o = oracle.Oracle(mesh)
    nbr, _ = o.neighbors()
    geo = o.cell_geometry()
    near = np.nonzero(np.abs(geo["cx"] + 0.3 * geo["cy"] - 0.55) < 0.08)[0]
    cell = int(min(near, key=lambda k: o.reconstruct_cell(U, int(k))["omega"][0]))
    r = o.reconstruct_cell(U, cell)
    b = r["beta"]
    st = [cell] + [int(k) if k >= 0 else cell for k in nbr[cell]]
    Wave = U[0, 0, st].mean() + 1e-30
    g = np.array([0.94, 0.02, 0.02, 0.02])
    kappa = (abs(b[0] - b[1]) + abs(b[0] - b[2]) + abs(b[0] - b[3])) ** 2 / 9
    w = g * (1 + kappa / (1e-8 * Wave ** 4 + Wave ** 2 * b))
    np.testing.assert_allclose(r["omega"], w / w.sum(), rtol=1e-13)
    assert r["omega"][0] < 0.5 * g[0]     # a visibly nonlinear case


# ---------------------------------------------------------------- scale limiter fraction
def test_limiter_fraction_is_the_largest_admissible_fraction():
    """R18: the fraction pulls a point value toward the cell average just far
    enough that density and pressure are >= eps.  Checked against the
    definition on random segments: the state at f is admissible, the state a
    little beyond f is not, and where the pressure bound is the active one
    |p - eps| <= 1e-12 p_bar."""
    rng = np.random.default_rng(23)
    Wb_all = _random_euler_states(rng, 300)
    active_p = 0
    for Wb in Wb_all:
        # a far-away point value, often with negative density or pressure
        w = Wb + rng.normal(size=4) * np.array([1.0, 2.0, 2.0, 3.0]) * rng.uniform(0.2, 3.0)
        pb = 0.4 * (Wb[3] - 0.5 * (Wb[1] ** 2 + Wb[2] ** 2) / Wb[0])
        eps = min(1e-13, Wb[0], pb)
        f = oracle.admissible_fraction(Wb, w, eps)
        assert 0.0 <= f <= 1.0

        def state(ff):
            x = Wb + ff * (w - Wb)
            return x[0], 0.4 * (x[3] - 0.5 * (x[1] ** 2 + x[2] ** 2) / x[0])
        rho, p = state(f)
        assert rho >= eps * (1 - 1e-12) and p >= eps - 1e-12 * pb, (rho, p, eps)
        for ff in np.linspace(0, f, 7):
            r_, p_ = state(ff)
            assert r_ >= eps * (1 - 1e-12) and p_ >= eps - 1e-12 * pb
        if f < 1.0:
            r2, p2 = state(min(1.0, f * (1 + 1e-9) + 1e-12))
            assert r2 < eps or p2 < eps
            if abs(rho - eps) > 1e-12 * Wb[0]:      # the pressure bound is the active one
                active_p += 1
                assert abs(p - eps) <= 1e-12 * pb, (p, eps, pb)
    assert active_p >= 50


def test_flux_blending_keeps_averages_positive_where_the_scale_limiter_alone_fails():
    """R23: with the scale limiter alone the first step of these four-quadrant
    data (those of the batched workload's solve 244) already gives a negative
    pressure; blending each edge flux with the first-order LLF flux keeps every
    average admissible, leaves smooth data untouched (theta = 1) and
    conserves the totals on a periodic mesh."""
    st = I.quadrant_states(4 + 244)
    mesh = I.jittered_box(I.config4_sizes(256)[244], seed=4000 + 244)     # 8,192 triangles
    U0 = I.initial_state(mesh, I.quadrant_fn(st), 4, nq=4)
    alone = oracle.Oracle(mesh, "euler", positivity="scale_only")
    U1 = alone.step(U0, alone.cfl_dt(U0))
    assert min(U1[0, 0].min(), _pressure(U1).min()) < 0
    blend = oracle.Oracle(mesh, "euler", positivity=True)
    U = U0
    for _ in range(20):
        U = blend.step(U, blend.cfl_dt(U))
        assert U[0, 0].min() > 0 and _pressure(U).min() > 0
    pmesh = I.jittered_periodic(16, 1.0, seed=9)
    Up = I.initial_state(pmesh, I.quadrant_fn(st), 4, nq=4)
    bp = oracle.Oracle(pmesh, "euler", positivity=True)
    ap = bp.cell_geometry()["area"]
    s0 = (Up[0] * ap).sum(axis=1)
    for _ in range(10):
        Up = bp.step(Up, bp.cfl_dt(Up))
        assert Up[0, 0].min() > 0 and _pressure(Up).min() > 0
    np.testing.assert_allclose((Up[0] * ap).sum(axis=1), s0, rtol=1e-13)


# ---------------------------------------------------------------- walls and inflow (R25)
def _channel_and_mirror(nx=8, ny=5, seed=31):
    """A channel [0, 1) x [0, 1], periodic in x, and the doubled torus
    [0, 1) x [0, 2) made of the channel and its mirror image across y = 1
    (the channel's cells first, in the same order)."""
    ch = I.jittered_rect(nx, ny, 0.0, 1.0, 0.0, 1.0, seed=seed, periodic_x=True)
    nv = ch.nv
    xy = ch.xy
    rows = np.round(xy[:, 1] * ny).astype(int)          # grid row of each vertex (jitter < h/2)
    inner = np.nonzero((rows > 0) & (rows < ny))[0]
    mirror_id = np.arange(nv)
    mirror_id[inner] = nv + np.arange(inner.size)        # rows 0 and ny are their own mirrors
    mxy = xy[inner].copy(); mxy[:, 1] = 2.0 - mxy[:, 1]
    full_xy = np.concatenate([xy, mxy])
    mt = mirror_id[ch.tri][:, [0, 2, 1]]                  # mirrored triangles, counter-clockwise again
    full = I.Mesh(xy=full_xy, tri=np.concatenate([ch.tri, mt]).astype(np.int32), Lx=1.0, Ly=2.0, bc=0)
    ch.edge_bc = I.side_boundary_types(ch, bottom=I.BC_REFLECTIVE, top=I.BC_REFLECTIVE)
    return ch, full


def _symmetric_flow(x, y):
    """Even in y about y = 0 and y = 1 except v, which is odd there; period 2."""
    c = np.cos(np.pi * y)
    rho = 1.0 + 0.2 * np.sin(2 * np.pi * x) * c
    u = 0.5 + 0.1 * np.cos(2 * np.pi * x) * c
    v = 0.3 * np.sin(np.pi * y) * (1 + 0.2 * np.cos(2 * np.pi * x))
    p = 1.0 + 0.1 * np.sin(2 * np.pi * x + 0.3) * c
    return I.euler_from_primitive(rho, u, v, p)


def test_walls_reproduce_the_mirror_image_flow():
    """R25: a flow that is symmetric about the walls y = 0 and y = 1 of a channel
    evolves, with reflective walls, exactly like the same flow on the doubled
    periodic domain made of the channel and its mirror image, where no
    boundary exists: the wall ghosts carry the mirrored averages and
    derivative averages and the wall flux sees the mirrored Taylor data.  The
    periodic run is the reference (it uses none of the wall code)."""
    ch, full = _channel_and_mirror()
    U_ch = I.initial_state(ch, _symmetric_flow, 4)
    # the mirror half carries exactly the mirrored data: v and d/dy change sign
    Mw = np.array([1.0, 1.0, -1.0, 1.0])[:, None]
    U_full = np.concatenate([U_ch, np.stack([Mw * U_ch[0], Mw * U_ch[1], -Mw * U_ch[2]])], axis=-1)
    walls = oracle.Oracle(ch, "euler")
    torus = oracle.Oracle(full, "euler")
    dt = 0.5 * torus.cfl_dt(U_full)
    for _ in range(4):
        U_ch = walls.step(U_ch, dt)
        U_full = torus.step(U_full, dt)
    ref = U_full[:, :, :ch.nt]
    scale = np.abs(ref).max(axis=-1, keepdims=True)
    err = (np.abs(U_ch - ref) / scale).max()
    assert err < 1e-12, err
    # the wall is felt: transmissive boundaries give a different answer
    ch.edge_bc = None
    U_t = I.initial_state(ch, _symmetric_flow, 4)
    tr = oracle.Oracle(ch, "euler")
    for _ in range(4):
        U_t = tr.step(U_t, dt)
    assert (np.abs(U_t - ref) / scale).max() > 1e-4


def test_free_stream_with_walls_and_inflow():
    """A constant state moving along the walls of a box, with the same state
    imposed at an inflow side and an outflow side, stays constant."""
    mesh = I.jittered_rect(9, 7, 0.0, 1.0, 0.0, 0.6, seed=3)
    mesh.edge_bc = I.side_boundary_types(mesh, left=I.BC_INFLOW, right=I.BC_TRANSMISSIVE,
                                         bottom=I.BC_REFLECTIVE, top=I.BC_REFLECTIVE)
    W = I.euler_from_primitive(np.array(1.3), np.array(0.8), np.array(0.0), np.array(0.9))
    U = np.zeros((3, 4, mesh.nt)); U[0] = W[:, None]
    for pos in (False, True):
        o = oracle.Oracle(mesh, "euler", inflow=W, positivity=pos)
        V = U
        for _ in range(3):
            V = o.step(V, o.cfl_dt(V))
        np.testing.assert_allclose(V[0], U[0], rtol=1e-13, atol=1e-13)
        assert np.abs(V[1:]).max() < 1e-11


def _exact_riemann_density(L, R, xs, t, g=1.4):
    """Density of the exact solution of the 1D Riemann problem (rho, u, p) at
    x / t = xs / t, by Newton on the star pressure (Toro, ch. 4)."""
    rL, uL, pL = L; rR, uR, pR = R
    cL, cR = np.sqrt(g * pL / rL), np.sqrt(g * pR / rR)

    def fk(p, r, pk, ck):
        if p > pk:   # shock
            A, B = 2 / ((g + 1) * r), (g - 1) / (g + 1) * pk
            return (p - pk) * np.sqrt(A / (p + B)), np.sqrt(A / (B + p)) * (1 - (p - pk) / (2 * (B + p)))
        pr = p / pk  # rarefaction
        return 2 * ck / (g - 1) * (pr ** ((g - 1) / (2 * g)) - 1), 1 / (r * ck) * pr ** (-(g + 1) / (2 * g))
    p = 0.5 * (pL + pR)
    for _ in range(100):
        f1, d1 = fk(p, rL, pL, cL); f2, d2 = fk(p, rR, pR, cR)
        dp = (f1 + f2 + uR - uL) / (d1 + d2)
        p = max(p - dp, 1e-12)
        if abs(dp) < 1e-14 * p:
            break
    us = 0.5 * (uL + uR) + 0.5 * (fk(p, rR, pR, cR)[0] - fk(p, rL, pL, cL)[0])
    out = np.empty_like(xs)
    for k, x in enumerate(xs):
        s = x / t
        if s < us:   # left of the contact
            if p > pL:
                SL = uL - cL * np.sqrt((g + 1) / (2 * g) * p / pL + (g - 1) / (2 * g))
                out[k] = rL if s < SL else rL * ((p / pL + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * p / pL + 1))
            else:
                cs = cL * (p / pL) ** ((g - 1) / (2 * g))
                if s < uL - cL:
                    out[k] = rL
                elif s > us - cs:
                    out[k] = rL * (p / pL) ** (1 / g)
                else:
                    out[k] = rL * (2 / (g + 1) + (g - 1) / ((g + 1) * cL) * (uL - s)) ** (2 / (g - 1))
        else:
            if p > pR:
                SR = uR + cR * np.sqrt((g + 1) / (2 * g) * p / pR + (g - 1) / (2 * g))
                out[k] = rR if s > SR else rR * ((p / pR + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * p / pR + 1))
            else:
                cs = cR * (p / pR) ** ((g - 1) / (2 * g))
                if s > uR + cR:
                    out[k] = rR
                elif s < us + cs:
                    out[k] = rR * (p / pR) ** (1 / g)
                else:
                    out[k] = rR * (2 / (g + 1) - (g - 1) / ((g + 1) * cR) * (uR - s)) ** (2 / (g - 1))
    return out


@pytest.mark.slow
def test_lax_tube_against_the_exact_riemann_solution():
    """The Lax problem of Section 3 (inflow on the left, outflow on the right,
    walls at the top and bottom, scale limiter and flux blending) against the
    exact 1D Riemann solution at T = 0.16: the density's L1 error over the
    tube is that of a shock-capturing scheme on 100 cells, and the walls keep
    the flow one-dimensional."""
    mesh, fn, T, win = I.lax_tube()
    o = oracle.Oracle(mesh, "euler", positivity=True, inflow=win)
    U0 = I.initial_state(mesh, fn, 4, nq=4)
    U, dts = o.run_to(U0, T)
    geo = o.cell_geometry()
    exact = _exact_riemann_density((0.445, 0.698, 3.528), (0.5, 0.0, 0.571), geo["cx"], T)
    l1 = float((np.abs(U[0, 0] - exact) * geo["area"]).sum() / geo["area"].sum())
    v = np.abs(U[0, 2] / U[0, 0])
    mean_v = float((v * geo["area"]).sum() / geo["area"].sum())
    print(f"Lax tube: {len(dts)} steps, density L1 error {l1:.3e}, mean |v| {mean_v:.2e}")
    assert l1 < 0.02
    assert mean_v < 0.01     # the jittered cells perturb the flow at the shock; the walls keep it 1D


def test_step_of_a_patch_equals_the_full_step_there():
    """The patch step (used to time the oracle) gives the full step's values on
    its cells; the full step is unchanged by the patch path."""
    mesh = I.jittered_periodic(16, 10.0, 0.15, seed=5)
    U = I.initial_state(mesh, I.vortex, 4)
    o = oracle.Oracle(mesh, "euler")
    dt = o.cfl_dt(U)
    full = o.step(U, dt)
    cells = np.arange(40, 260, 3)
    part = o.step_cells(U, dt, cells)
    np.testing.assert_allclose(part, full[:, :, cells], rtol=1e-13, atol=1e-13 * np.abs(full).max())
    mask = np.zeros(mesh.nt, np.uint8); mask[cells] = 1
    masked = o.step(U, dt, mask=mask)
    np.testing.assert_array_equal(masked[:, :, cells], part)
    others = np.setdiff1d(np.arange(mesh.nt), cells)
    np.testing.assert_array_equal(masked[:, :, others], U[:, :, others])
