"""Seeded synthetic inputs: triangular meshes, initial cell averages, exact solutions.

This module generates the workloads; it holds none of the scheme's arithmetic
and is shared by the CUDA tests, the oracle tests and the benchmark.  Every
generator is deterministic for a given seed (numpy PCG64).

State layout used everywhere on the host: ``U[k, c, i]`` with ``k = 0`` the cell
average of W (Eq. aver, first line), ``k = 1`` the cell average of W_x and
``k = 2`` the cell average of W_y, for component ``c`` of cell ``i``.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

GAMMA_GAS = 1.4


@dataclasses.dataclass
class Mesh:
    """Triangles with counter-clockwise vertex order.

    ``Lx``/``Ly`` > 0 mark a periodic direction (vertex coordinates are taken
    modulo the period); ``bc`` is 0 for periodic and 1 for transmissive
    boundaries."""

    xy: np.ndarray          # float64 [nv, 2]
    tri: np.ndarray         # int32 [nt, 3]
    Lx: float = 0.0
    Ly: float = 0.0
    bc: int = 0
    edge_bc: np.ndarray | None = None   # int32 [nt, 3]: type of local edge j where it is a boundary edge
                                        # (1 transmissive, 2 reflective, 3 inflow); None: all transmissive

    @property
    def nt(self) -> int:
        return int(self.tri.shape[0])

    @property
    def nv(self) -> int:
        return int(self.xy.shape[0])

    def unwrapped(self) -> np.ndarray:
        """Vertex coordinates per triangle [nt, 3, 2], unwrapped around vertex 0."""
        P = self.xy[self.tri]                      # [nt, 3, 2]
        d = P - P[:, :1, :]
        for k, L in enumerate((self.Lx, self.Ly)):
            if L > 0:
                d[..., k] -= L * np.floor(d[..., k] / L + 0.5)
        return P[:, :1, :] + d


# ----------------------------------------------------------------- meshes
def _grid_triangles(n_i: int, n_j: int, vid) -> np.ndarray:
    """Split each square (i, j) by the diagonal from (i, j) to (i+1, j+1)."""
    I, J = np.meshgrid(np.arange(n_i), np.arange(n_j), indexing="ij")
    I = I.ravel(); J = J.ravel()
    a = vid(I, J); b = vid(I + 1, J); c = vid(I + 1, J + 1); d = vid(I, J + 1)
    t1 = np.stack([a, b, c], axis=1)
    t2 = np.stack([a, c, d], axis=1)
    return np.concatenate([t1, t2], axis=0).astype(np.int32)


def structured_periodic(n: int, L: float) -> Mesh:
    """Periodic [0, L)^2, n x n squares each split into two triangles."""
    return jittered_periodic(n, L, jitter=0.0, seed=0)


def jittered_periodic(n: int, L: float, jitter: float = 0.15, seed: int = 0) -> Mesh:
    """Periodic [0, L)^2 grid whose vertices move by U(-jitter*h, +jitter*h) per coordinate."""
    if n < 3:
        raise ValueError("need at least 3 squares per direction on a torus")
    h = L / n
    rng = np.random.default_rng(seed)
    I, J = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    xy = np.stack([I.ravel() * h, J.ravel() * h], axis=1).astype(np.float64)
    if jitter > 0:
        xy += rng.uniform(-jitter * h, jitter * h, size=xy.shape)
    tri = _grid_triangles(n, n, lambda i, j: (i % n) * n + (j % n))
    return Mesh(xy=xy, tri=tri, Lx=L, Ly=L, bc=0)


def jittered_periodic_rect(nx: int, ny: int, h: float, jitter: float = 0.15, seed: int = 0) -> Mesh:
    """Periodic [0, nx h) x [0, ny h) grid of nx x ny squares (2 nx ny
    triangles) whose vertices move by U(-jitter*h, +jitter*h) per coordinate."""
    if nx < 3 or ny < 3:
        raise ValueError("need at least 3 squares per direction on a torus")
    rng = np.random.default_rng(seed)
    I, J = np.meshgrid(np.arange(nx), np.arange(ny), indexing="ij")
    xy = np.stack([I.ravel() * h, J.ravel() * h], axis=1).astype(np.float64)
    if jitter > 0:
        xy += rng.uniform(-jitter * h, jitter * h, size=xy.shape)
    tri = _grid_triangles(nx, ny, lambda i, j: (i % nx) * ny + (j % ny))
    return Mesh(xy=xy, tri=tri, Lx=nx * h, Ly=ny * h, bc=0)


def jittered_box(n: int, L: float = 1.0, jitter: float = 0.15, seed: int = 0) -> Mesh:
    """Non-periodic [0, L]^2 grid (transmissive boundaries).  Interior vertices
    move by U(+-jitter*h) per coordinate, boundary vertices only along the
    boundary, corners stay fixed."""
    h = L / n
    rng = np.random.default_rng(seed)
    I, J = np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="ij")
    I = I.ravel(); J = J.ravel()
    xy = np.stack([I * h, J * h], axis=1).astype(np.float64)
    if jitter > 0:
        dx = rng.uniform(-jitter * h, jitter * h, size=xy.shape)
        dx[(I == 0) | (I == n), 0] = 0.0
        dx[(J == 0) | (J == n), 1] = 0.0
        xy += dx
    tri = _grid_triangles(n, n, lambda i, j: i * (n + 1) + j)
    return Mesh(xy=xy, tri=tri, Lx=0.0, Ly=0.0, bc=1)


BC_TRANSMISSIVE, BC_REFLECTIVE, BC_INFLOW = 1, 2, 3


def jittered_rect(nx: int, ny: int, x0: float, x1: float, y0: float, y1: float, jitter: float = 0.15,
                  seed: int = 0, periodic_x: bool = False) -> Mesh:
    """[x0, x1] x [y0, y1] grid of nx x ny cells split by the "/" diagonal.
    Interior vertices move by U(+-jitter h) per coordinate, boundary vertices
    only along their side (corners stay); periodic_x: the left and right sides
    are identified (x1 - x0 is the period)."""
    hx, hy = (x1 - x0) / nx, (y1 - y0) / ny
    rng = np.random.default_rng(seed)
    ni = nx if periodic_x else nx + 1
    I, J = np.meshgrid(np.arange(ni), np.arange(ny + 1), indexing="ij")
    I = I.ravel(); J = J.ravel()
    xy = np.stack([x0 + I * hx, y0 + J * hy], axis=1).astype(np.float64)
    if jitter > 0:
        d = rng.uniform(-1, 1, size=xy.shape) * jitter * np.array([hx, hy])
        if not periodic_x:
            d[(I == 0) | (I == nx), 0] = 0.0
        d[(J == 0) | (J == ny), 1] = 0.0
        xy += d
    if periodic_x:
        tri = _grid_triangles(nx, ny, lambda i, j: (i % nx) * (ny + 1) + j)
    else:
        tri = _grid_triangles(nx, ny, lambda i, j: i * (ny + 1) + j)
    return Mesh(xy=xy, tri=tri, Lx=(x1 - x0) if periodic_x else 0.0, Ly=0.0, bc=1)


def side_boundary_types(mesh: Mesh, left=BC_TRANSMISSIVE, right=BC_TRANSMISSIVE, bottom=BC_TRANSMISSIVE,
                        top=BC_TRANSMISSIVE) -> np.ndarray:
    """Per-edge boundary types [nt, 3] of an axis-aligned box mesh, each
    boundary edge classified by the side its midpoint lies on."""
    P = mesh.unwrapped()
    lo, hi = P.reshape(-1, 2).min(axis=0), P.reshape(-1, 2).max(axis=0)
    tol = 1e-9 * max(hi - lo)
    ebc = np.full((mesh.nt, 3), BC_TRANSMISSIVE, dtype=np.int32)
    for j in range(3):
        mid = 0.5 * (P[:, j] + P[:, (j + 1) % 3])
        for side, val in ((mid[:, 0] <= lo[0] + tol, left), (mid[:, 0] >= hi[0] - tol, right),
                          (mid[:, 1] <= lo[1] + tol, bottom), (mid[:, 1] >= hi[1] - tol, top)):
            ebc[side, j] = val
    return ebc


def lax_tube(seed: int = 0):
    """The Lax shock tube of Section 3 on (-0.5, 0.5) x (-0.03, 0.03): a jittered
    100 x 6 triangulation, inflow on the left (the left state), outflow on the
    right, walls at the bottom and top; T = 0.16.  Returns (mesh, initial data
    function, T, inflow state)."""
    mesh = jittered_rect(100, 6, -0.5, 0.5, -0.03, 0.03, seed=seed)
    mesh.edge_bc = side_boundary_types(mesh, left=BC_INFLOW, right=BC_TRANSMISSIVE, bottom=BC_REFLECTIVE,
                                       top=BC_REFLECTIVE)
    L, R = (0.445, 0.698, 0.0, 3.528), (0.5, 0.0, 0.0, 0.571)

    def fn(x, y):
        left = x < 0
        return euler_from_primitive(np.where(left, L[0], R[0]), np.where(left, L[1], R[1]),
                                    np.where(left, L[2], R[2]) + 0 * y, np.where(left, L[3], R[3]))
    win = euler_from_primitive(*[np.array(v) for v in L])
    return mesh, fn, 0.16, win


def blast_waves(seed: int = 0):
    """The interacting blast waves of Section 3 on (0, 1) x (-0.0075, 0.0075): a
    jittered 400 x 6 triangulation with walls on all sides; T = 0.038."""
    mesh = jittered_rect(400, 6, 0.0, 1.0, -0.0075, 0.0075, seed=seed)
    mesh.edge_bc = side_boundary_types(mesh, BC_REFLECTIVE, BC_REFLECTIVE, BC_REFLECTIVE, BC_REFLECTIVE)

    def fn(x, y):
        p = np.where(x < 0.1, 1000.0, np.where(x < 0.9, 0.01, 100.0)) + 0 * y
        one = np.ones_like(p)
        return euler_from_primitive(one, 0 * one, 0 * one, p)
    return mesh, fn, 0.038


def poisson_disk_points(L: float, r: float, seed: int, attempts: int = 8) -> np.ndarray:
    """Periodic Poisson-disk sample of [0, L)^2 with minimum distance r.

    Parallel dart throwing on a background grid of cell size <= r/sqrt(2)
    (each cell holds at most one point); cells are visited in 3x3 phases so
    that cells of one phase are at least 2 cells apart and their candidates
    cannot conflict with each other.  A cell is given up after ``attempts``
    rejected candidates (the analogue of Bridson's k)."""
    rng = np.random.default_rng(seed)
    G = 3 * int(math.ceil(L / (r / math.sqrt(2.0)) / 3.0))
    cell = L / G
    grid = -np.ones((G, G), dtype=np.int64)
    fails = np.zeros((G, G), dtype=np.int16)
    px = np.zeros(G * G); py = np.zeros(G * G)
    npts = 0
    offs = [(di, dj) for di in range(-2, 3) for dj in range(-2, 3) if (di, dj) != (0, 0)]
    r2 = r * r
    for _ in range(attempts + 1):
        for pi in range(3):
            for pj in range(3):
                sub = (grid[pi::3, pj::3] < 0) & (fails[pi::3, pj::3] < attempts)
                I, J = np.nonzero(sub)
                if I.size == 0:
                    continue
                I = I * 3 + pi; J = J * 3 + pj
                cx = (I + rng.random(I.size)) * cell
                cy = (J + rng.random(I.size)) * cell
                ok = np.ones(I.size, dtype=bool)
                for di, dj in offs:
                    q = grid[(I + di) % G, (J + dj) % G]
                    has = np.nonzero((q >= 0) & ok)[0]
                    if has.size == 0:
                        continue
                    qq = q[has]
                    dx = cx[has] - px[qq]; dy = cy[has] - py[qq]
                    dx -= L * np.floor(dx / L + 0.5); dy -= L * np.floor(dy / L + 0.5)
                    ok[has[dx * dx + dy * dy < r2]] = False
                k = np.nonzero(ok)[0]
                ids = npts + np.arange(k.size)
                px[ids] = cx[k]; py[ids] = cy[k]
                grid[I[k], J[k]] = ids
                npts += k.size
                bad = np.nonzero(~ok)[0]
                fails[I[bad], J[bad]] += 1
    return np.stack([px[:npts], py[:npts]], axis=1)


def periodic_delaunay(pts: np.ndarray, L: float, margin: float) -> Mesh:
    """Delaunay triangulation of points on the torus [0, L)^2: replicate a margin
    of points around the square, triangulate, keep the triangles whose
    barycenter lies in [0, L)^2 and map their vertices back to the base set."""
    from scipy.spatial import Delaunay

    n = pts.shape[0]
    ext = [pts]; ids = [np.arange(n)]
    for sx in (-1, 0, 1):
        for sy in (-1, 0, 1):
            if sx == 0 and sy == 0:
                continue
            q = pts + np.array([sx * L, sy * L])
            keep = (q[:, 0] > -margin) & (q[:, 0] < L + margin) & (q[:, 1] > -margin) & (q[:, 1] < L + margin)
            ext.append(q[keep]); ids.append(np.nonzero(keep)[0])
    E = np.concatenate(ext); Eid = np.concatenate(ids)
    dt = Delaunay(E)
    S = dt.simplices
    bc = E[S].mean(axis=1)
    keep = (bc[:, 0] >= 0) & (bc[:, 0] < L) & (bc[:, 1] >= 0) & (bc[:, 1] < L)
    S = S[keep]
    P = E[S]
    cross = (P[:, 1, 0] - P[:, 0, 0]) * (P[:, 2, 1] - P[:, 0, 1]) - (P[:, 2, 0] - P[:, 0, 0]) * (P[:, 1, 1] - P[:, 0, 1])
    flip = cross < 0
    S[flip, 1], S[flip, 2] = S[flip, 2].copy(), S[flip, 1].copy()
    tri = Eid[S].astype(np.int32)
    if tri.shape[0] != 2 * n:
        raise RuntimeError(f"periodic Delaunay: {tri.shape[0]} triangles for {n} points (expected {2 * n})")
    return Mesh(xy=pts.astype(np.float64), tri=tri, Lx=L, Ly=L, bc=0)


def poisson_delaunay_periodic(L: float, target_points: int, seed: int) -> Mesh:
    """Periodic Delaunay mesh of a seeded Poisson-disk point set of about
    ``target_points`` points (about twice as many triangles)."""
    # the dart throwing above fills about 0.628 / r^2 points per unit area
    r = math.sqrt(0.628 * L * L / target_points)
    pts = poisson_disk_points(L, r, seed)
    return periodic_delaunay(pts, L, margin=8.0 * r)


def mesh_quality(mesh: Mesh) -> dict:
    P = mesh.unwrapped()
    e = [np.linalg.norm(P[:, (j + 1) % 3] - P[:, j], axis=1) for j in range(3)]
    a, b, c = e
    ang = []
    for (x, y, z) in ((a, b, c), (b, c, a), (c, a, b)):
        ang.append(np.degrees(np.arccos(np.clip((x * x + y * y - z * z) / (2 * x * y), -1, 1))))
    area = 0.5 * ((P[:, 1, 0] - P[:, 0, 0]) * (P[:, 2, 1] - P[:, 0, 1]) - (P[:, 2, 0] - P[:, 0, 0]) * (P[:, 1, 1] - P[:, 0, 1]))
    return {"nt": mesh.nt, "nv": mesh.nv, "min_angle_deg": float(np.min(ang)), "min_area": float(area.min()),
            "max_area": float(area.max())}


# ----------------------------------------------------------------- quadrature
def _tri_rule(nq: int):
    """Collapsed (Duffy) Gauss rule on the reference triangle (0,0),(1,0),(0,1):
    barycentric-free points (u, v) and weights summing to 1."""
    g, w = np.polynomial.legendre.leggauss(nq)
    s = 0.5 * (g + 1); ws = 0.5 * w
    S, T = np.meshgrid(s, s, indexing="ij")
    WS, WT = np.meshgrid(ws, ws, indexing="ij")
    u = S.ravel(); v = (T * (1 - S)).ravel()
    wt = (WS * WT * (1 - S)).ravel() * 2.0
    return u, v, wt


def cell_averages(mesh: Mesh, fn, m: int, nq: int = 6, chunk: int = 1 << 16) -> np.ndarray:
    """(1/|K|) * integral of fn over each triangle -> [m, nt]."""
    P = mesh.unwrapped()
    u, v, wt = _tri_rule(nq)
    out = np.empty((m, mesh.nt))
    for s in range(0, mesh.nt, chunk):
        Q = P[s:s + chunk]
        x = Q[:, 0, 0:1] + u * (Q[:, 1, 0:1] - Q[:, 0, 0:1]) + v * (Q[:, 2, 0:1] - Q[:, 0, 0:1])
        y = Q[:, 0, 1:2] + u * (Q[:, 1, 1:2] - Q[:, 0, 1:2]) + v * (Q[:, 2, 1:2] - Q[:, 0, 1:2])
        val = fn(x, y)                       # [m, n, q]
        out[:, s:s + chunk] = np.einsum("mnq,q->mn", val, wt)
    return out


def derivative_averages(mesh: Mesh, fn, m: int, nq: int = 8, chunk: int = 1 << 16):
    """Cell averages of W_x and W_y by the divergence theorem along the three
    edges with nq-point Gauss-Legendre (valid for discontinuous data too)."""
    P = mesh.unwrapped()
    g, w = np.polynomial.legendre.leggauss(nq)
    s01 = 0.5 * (g + 1); ws = 0.5 * w
    V = np.zeros((m, mesh.nt)); Y = np.zeros((m, mesh.nt))
    for s in range(0, mesh.nt, chunk):
        Q = P[s:s + chunk]
        area = 0.5 * ((Q[:, 1, 0] - Q[:, 0, 0]) * (Q[:, 2, 1] - Q[:, 0, 1]) - (Q[:, 2, 0] - Q[:, 0, 0]) * (Q[:, 1, 1] - Q[:, 0, 1]))
        for j in range(3):
            A = Q[:, j]; B = Q[:, (j + 1) % 3]
            x = A[:, 0:1] + s01 * (B[:, 0:1] - A[:, 0:1])
            y = A[:, 1:2] + s01 * (B[:, 1:2] - A[:, 1:2])
            val = np.einsum("mnq,q->mn", fn(x, y), ws)      # mean along the edge
            nlx = (B[:, 1] - A[:, 1]); nly = -(B[:, 0] - A[:, 0])  # n |e|
            V[:, s:s + chunk] += val * nlx
            Y[:, s:s + chunk] += val * nly
        V[:, s:s + chunk] /= area; Y[:, s:s + chunk] /= area
    return V, Y


def initial_state(mesh: Mesh, fn, m: int, nq: int = 6) -> np.ndarray:
    """U[3, m, nt]: cell averages of W, W_x, W_y of the function fn."""
    W = cell_averages(mesh, fn, m, nq=nq)
    V, Y = derivative_averages(mesh, fn, m)
    return np.stack([W, V, Y], axis=0)


# ----------------------------------------------------------------- problems
def advection_sine(x, y):
    """C1 initial data 1 + 0.2 sin(pi (x + y))."""
    return (1.0 + 0.2 * np.sin(np.pi * (x + y)))[None]


def burgers_sine(x, y):
    """Burgers initial data 0.5 + sin(pi (x + y) / 2) (Example 3.1)."""
    return (0.5 + np.sin(0.5 * np.pi * (x + y)))[None]


def burgers_exact(x, y, t):
    """Exact Burgers solution while smooth: u = u0(x + y - 2 u t) by Newton."""
    s = x + y
    u = 0.5 + np.sin(0.5 * np.pi * s)
    for _ in range(60):
        arg = 0.5 * np.pi * (s - 2 * u * t)
        F = u - 0.5 - np.sin(arg)
        dF = 1 + np.cos(arg) * np.pi * t
        du = F / dF
        u = u - du
        if np.max(np.abs(du)) < 1e-15:
            break
    return u[None]


def euler_from_primitive(rho, u, v, p, gamma=GAMMA_GAS):
    E = p / (gamma - 1) + 0.5 * rho * (u * u + v * v)
    return np.stack([rho, rho * u, rho * v, E], axis=0)


def vortex(x, y, t=0.0, L=10.0, xc=5.0, yc=5.0, gamma=GAMMA_GAS, eps=5.0, bumps=None):
    """Isentropic vortex of Example 3.3 (strength 5, background (1, 1, 1, 1)),
    translated by (t, t) on the periodic square (nearest image), plus optional
    Gaussian density bumps [(cx, cy, amp, sigma), ...]."""
    cx = xc + t; cy = yc + t
    dx = x - cx; dy = y - cy
    dx -= L * np.floor(dx / L + 0.5); dy -= L * np.floor(dy / L + 0.5)
    r2 = dx * dx + dy * dy
    rho = (1 - (gamma - 1) * eps * eps / (8 * gamma * np.pi ** 2) * np.exp(1 - r2)) ** (1 / (gamma - 1))
    u = 1 - eps / (2 * np.pi) * np.exp(0.5 * (1 - r2)) * dy
    v = 1 + eps / (2 * np.pi) * np.exp(0.5 * (1 - r2)) * dx
    p = rho ** gamma
    if bumps is not None:
        for (bx, by, amp, sig) in bumps:
            ex = x - bx; ey = y - by
            ex -= L * np.floor(ex / L + 0.5); ey -= L * np.floor(ey / L + 0.5)
            rho = rho + amp * np.exp(-(ex * ex + ey * ey) / (sig * sig))
    return euler_from_primitive(rho, u, v, p, gamma)


def density_wave(x, y, t=0.0):
    """Euler smooth density wave of Example 3.2 at time t (exact translation)."""
    rho = 1 + 0.2 * np.sin(0.5 * np.pi * (x + y - 2 * t))
    one = np.ones_like(rho)
    return euler_from_primitive(rho, one, one, one)


def quadrant_states(seed: int):
    """Four constant primitive states (rho, u, v, p) for a Riemann-type problem."""
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.1, 1.5, 4)
    p = rng.uniform(0.02, 1.5, 4)
    u = rng.uniform(-1, 1, 4); v = rng.uniform(-1, 1, 4)
    return np.stack([rho, u, v, p], axis=1)


def quadrant_fn(states, xs=0.5, ys=0.5):
    def fn(x, y):
        q = np.where(x >= xs, np.where(y >= ys, 0, 3), np.where(y >= ys, 1, 2))
        st = states[q]                       # [..., 4]
        return euler_from_primitive(st[..., 0], st[..., 1], st[..., 2], st[..., 3])
    return fn


def vortex_bumps(seed: int, n: int = 8, amp: float = 0.01, sigma: float = 0.5, L: float = 10.0):
    rng = np.random.default_rng(seed)
    c = rng.uniform(0, L, size=(n, 2))
    return [(float(a), float(b), amp, sigma) for a, b in c]


# ----------------------------------------------------------------- errors
def cell_areas(mesh: Mesh) -> np.ndarray:
    """|K| of every triangle (counter-clockwise vertices)."""
    P = mesh.unwrapped()
    return 0.5 * ((P[:, 1, 0] - P[:, 0, 0]) * (P[:, 2, 1] - P[:, 0, 1]) - (P[:, 2, 0] - P[:, 0, 0]) * (P[:, 1, 1] - P[:, 0, 1]))


def error_norms(mesh: Mesh, Wh: np.ndarray, We: np.ndarray):
    """L1 (area weighted) and L-infinity errors of cell averages (Section 3)."""
    area = cell_areas(mesh)
    d = np.abs(Wh - We)
    return float((d * area).sum() / area.sum()), float(d.max())


# ----------------------------------------------------------------- configs
def config1_mesh(n: int = 20) -> Mesh:
    """Linear advection u_t + u_x + u_y = 0 on periodic [0, 2]^2."""
    return structured_periodic(n, 2.0)


def config2_mesh(n: int = 316) -> Mesh:
    """Burgers on periodic [0, 4]^2, jittered grid (+-0.15 h), seed 2."""
    return jittered_periodic(n, 4.0, jitter=0.15, seed=2)


def config3_mesh(target_points: int = 1_000_000, seed: int = 3) -> Mesh:
    """Euler vortex on periodic [0, 10]^2, Delaunay mesh of Poisson-disk points."""
    return poisson_delaunay_periodic(10.0, target_points, seed)


def config5_mesh(n: int = 316) -> Mesh:
    """Euler on periodic [0, 10]^2, jittered grid, seed 5."""
    return jittered_periodic(n, 10.0, jitter=0.15, seed=5)


def config5_state(mesh: Mesh, seed: int = 5) -> np.ndarray:
    """Vortex plus 8 seeded Gaussian density bumps (amplitude 0.01, sigma 0.5):
    the initial state of the gradient (adjoint) workload."""
    bumps = vortex_bumps(seed)
    return initial_state(mesh, lambda x, y: vortex(x, y, bumps=bumps), 4)


def config4_batch(count: int = 256):
    """Batched Euler workload: `count` four-quadrant Riemann problems on [0, 1]^2,
    each on its own jittered grid of 2k-40k triangles (transmissive
    boundaries).  Returns (meshes, states)."""
    meshes, states = [], []
    for k, n in enumerate(config4_sizes(count)):
        mesh = jittered_box(n, seed=4000 + k)
        meshes.append(mesh)
        states.append(initial_state(mesh, quadrant_fn(quadrant_states(4 + k)), 4, nq=4))
    return meshes, states


def config4_sizes(count: int = 256, seed: int = 4, lo: int = 2000, hi: int = 40000):
    """Triangle counts of the batched meshes, uniform in [lo, hi], as grid sizes n (2 n^2 triangles)."""
    rng = np.random.default_rng(seed)
    nt = rng.uniform(lo, hi, count)
    return [max(4, int(round(math.sqrt(x / 2.0)))) for x in nt]
