"""GPU path against the FP64 CPU oracle, through the C ABI.

FP64: relative L-infinity error per component, max_K |a - b| / max_K |b|,
at most 1e-12 after the full run.  FP32: L1 / L-infinity error against the
FP64 oracle stated per case and bounded."""
import numpy as np
import pytest

import oracle
from paper_2607_10809_b300 import build as B
from paper_2607_10809_b300 import hweno
from paper_2607_10809_b300 import inputs as I

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    B.build()
    hweno.load()


def rel_linf(a, b):
    """max over cells of |a - b| / max over cells of |b|, per (k, c) plane."""
    num = np.abs(a - b).max(axis=-1)
    den = np.maximum(np.abs(b).max(axis=-1), 1e-300)
    return (num / den).max()


def run_both(mesh, U0, eq, T, precision="fp64"):
    o = oracle.Oracle(mesh, eq)
    Uo, dts = o.run_to(U0, T)
    s = hweno.Solver(mesh, U0, eq=eq, precision=precision)
    n = s.run_to(T)
    Ug, t = s.get_state()
    return Uo, Ug, dts, n, t, s


def test_advection_config1_fp64_full_run():
    mesh = I.config1_mesh(20)
    U0 = I.initial_state(mesh, I.advection_sine, 1)
    Uo, Ug, dts, n, t, _ = run_both(mesh, U0, "advection", 0.5)
    assert n == len(dts) and abs(t - 0.5) < 1e-14
    assert rel_linf(Ug, Uo) < FP64_TOL


def test_step_after_run_to_advances():
    """The target of run_to holds only inside that call: afterwards step()
    takes the CFL step of the state reached (or the given step) and matches
    the oracle's step from it."""
    mesh = I.config1_mesh(10)
    U0 = I.initial_state(mesh, I.advection_sine, 1)
    o = oracle.Oracle(mesh, "advection")
    s = hweno.Solver(mesh, U0, eq="advection", precision="fp64")
    s.run_to(0.1)
    U1, t1 = s.get_state()
    _, dt, _ = s.time()
    assert abs(t1 - 0.1) < 1e-15 and abs(dt - o.cfl_dt(U1)) <= 1e-14 * dt
    s.step()
    U2, t2 = s.get_state()
    assert abs(t2 - (t1 + dt)) < 1e-15
    assert rel_linf(U2, o.step(U1, dt)) < FP64_TOL
    s.step(0.5 * dt)
    U3, t3 = s.get_state()
    assert abs(t3 - (t2 + 0.5 * dt)) < 1e-15
    assert rel_linf(U3, o.step(U2, 0.5 * dt)) < FP64_TOL
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_export_import_continues_the_run_bit_for_bit(precision):
    """An internal state buffer holds the records and (FP32) the compensation
    words: importing an exported state and stepping again repeats the same
    steps bit for bit."""
    mesh = I.poisson_delaunay_periodic(10.0, 1500, seed=4)
    U0 = I.initial_state(mesh, I.vortex, 4)
    s = hweno.Solver(mesh, U0, eq="euler", precision=precision)
    for _ in range(5):
        s.step()
    buf = s.state_buffer()
    s.export_state(buf)
    t5 = s.get_state()[1]
    for _ in range(5):
        s.step()
    X, tx = s.get_state()
    s.import_state(buf, t5)
    for _ in range(5):
        s.step()
    Y, ty = s.get_state()
    assert tx == ty and np.array_equal(X, Y)
    s.close()


@pytest.mark.parametrize("T", [1.5 / np.pi ** 2, 1.5 / np.pi])
def test_burgers_jittered_fp64_smooth_and_shocked(T):
    mesh = I.jittered_periodic(24, 4.0, 0.15, seed=2)
    U0 = I.initial_state(mesh, I.burgers_sine, 1)
    Uo, Ug, dts, n, t, _ = run_both(mesh, U0, "burgers", T)
    assert n == len(dts)
    assert rel_linf(Ug, Uo) < FP64_TOL


@pytest.mark.parametrize("kind", ["jittered", "poisson"])
def test_euler_vortex_fp64(kind):
    if kind == "jittered":
        mesh = I.jittered_periodic(20, 10.0, 0.15, seed=5)
    else:
        mesh = I.poisson_delaunay_periodic(10.0, 700, seed=3)
    U0 = I.initial_state(mesh, I.vortex, 4)
    Uo, Ug, dts, n, t, _ = run_both(mesh, U0, "euler", 0.5)
    assert n == len(dts)
    assert rel_linf(Ug, Uo) < FP64_TOL


def test_euler_riemann_box_transmissive_fp64():
    mesh = I.jittered_box(16, seed=44)
    U0 = I.initial_state(mesh, I.quadrant_fn(I.quadrant_states(44)), 4, nq=4)
    Uo, Ug, dts, n, t, _ = run_both(mesh, U0, "euler", 0.05)
    assert n == len(dts)
    assert rel_linf(Ug, Uo) < FP64_TOL


@pytest.mark.parametrize("eq", ["advection", "burgers", "euler"])
def test_fixed_dt_steps_match_oracle(eq):
    mesh = I.jittered_periodic(7, 10.0 if eq == "euler" else 2.0, seed=61)   # 98 cells: fewer than one block
    m = 4 if eq == "euler" else 1
    fn = I.vortex if eq == "euler" else (I.advection_sine if eq == "advection" else I.burgers_sine)
    U0 = I.initial_state(mesh, fn, m)
    o = oracle.Oracle(mesh, eq)
    dts = [0.5 * o.cfl_dt(U0)] * 5
    Uo = o.run_dts(U0, dts)
    s = hweno.Solver(mesh, U0, eq=eq, precision="fp64")
    for dt in dts:
        s.step(dt)
    Ug, t = s.get_state()
    assert abs(t - sum(dts)) < 1e-14
    assert rel_linf(Ug, Uo) < FP64_TOL


def test_ragged_sizes_and_tiny_meshes():
    for n in (3, 9, 11):   # 18, 162, 242 cells: below, between and above block multiples
        mesh = I.jittered_periodic(n, 2.0, seed=70 + n)
        U0 = I.initial_state(mesh, I.burgers_sine, 1)
        Uo, Ug, dts, k, t, _ = run_both(mesh, U0, "burgers", 0.05)
        assert k == len(dts)
        assert rel_linf(Ug, Uo) < FP64_TOL


def test_conservation_and_free_stream_on_gpu():
    mesh = I.poisson_delaunay_periodic(10.0, 500, seed=9)
    U0 = I.initial_state(mesh, I.vortex, 4)
    s = hweno.Solver(mesh, U0, eq="euler", precision="fp64")
    c0 = s.conservation()
    s.run_to(0.3)
    c1 = s.conservation()
    np.testing.assert_allclose(c1, c0, rtol=1e-14)
    U, _ = s.get_state()
    area = oracle.Oracle(mesh, "euler").cell_geometry()["area"]
    scale = (np.abs(U[1]) * area).sum(axis=1)
    assert np.all(np.abs((U[1] * area).sum(axis=1)) < 1e-13 * scale)
    const = I.euler_from_primitive(1.3, 0.4, -0.7, 0.9)
    Uc = np.zeros_like(U0); Uc[0] = const[:, None]
    for prec, tol in (("fp64", 1e-14), ("fp32", 1e-6)):
        s = hweno.Solver(mesh, Uc, eq="euler", precision=prec)
        for _ in range(3):
            s.step()
        U, _ = s.get_state()
        np.testing.assert_allclose(U[0], Uc[0], rtol=tol)
        assert np.abs(U[1:]).max() < (1e-12 if prec == "fp64" else 1e-4)


def test_deterministic_bitwise():
    mesh = I.jittered_periodic(20, 10.0, 0.15, seed=5)
    U0 = I.initial_state(mesh, I.vortex, 4)
    outs = []
    for _ in range(2):
        s = hweno.Solver(mesh, U0, eq="euler", precision="fp32")
        s.run_to(0.2)
        outs.append(s.get_state()[0])
    assert np.array_equal(outs[0], outs[1])


def test_nonfinite_state_is_reported():
    mesh = I.jittered_periodic(8, 10.0, seed=5)
    U0 = I.initial_state(mesh, I.vortex, 4)
    U0[0, 0, 17] = np.nan
    with pytest.raises(hweno.HwError) as e:
        s = hweno.Solver(mesh, U0, eq="euler", precision="fp64")
        s.run_to(0.2)
    assert e.value.status == hweno.HW_ENONFINITE


@pytest.mark.parametrize("case", ["advection", "burgers", "vortex"])
def test_fp32_error_against_fp64_oracle(case):
    if case == "advection":
        mesh, eq, fn, T, m = I.config1_mesh(20), "advection", I.advection_sine, 0.5, 1
    elif case == "burgers":
        mesh, eq, fn, T, m = I.jittered_periodic(24, 4.0, 0.15, seed=2), "burgers", I.burgers_sine, 1.5 / np.pi ** 2, 1
    else:
        mesh, eq, fn, T, m = I.jittered_periodic(20, 10.0, 0.15, seed=5), "euler", I.vortex, 0.5, 4
    U0 = I.initial_state(mesh, fn, m)
    Uo, Ug, dts, n, t, _ = run_both(mesh, U0, eq, T, precision="fp32")
    area = oracle.Oracle(mesh, eq).cell_geometry()["area"]
    l1 = (np.abs(Ug[0] - Uo[0]) * area).sum(axis=1) / area.sum()
    linf = np.abs(Ug[0] - Uo[0]).max(axis=1)
    print(f"FP32 {case}: L1 {l1} Linf {linf} steps {n}")
    assert np.all(l1 < 1e-5) and np.all(linf < 1e-4)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_euler_riemann_with_scale_limiter(precision):
    mesh = I.jittered_box(20, seed=4)
    U0 = I.initial_state(mesh, I.quadrant_fn(I.quadrant_states(4)), 4, nq=4)
    o = oracle.Oracle(mesh, "euler", positivity=True)
    Uo, dts = o.run_to(U0, 0.05)
    s = hweno.Solver(mesh, U0, eq="euler", precision=precision, positivity=True)
    n = s.run_to(0.05)
    Ug, t = s.get_state()
    rho = Ug[0, 0]; p = 0.4 * (Ug[0, 3] - 0.5 * (Ug[0, 1] ** 2 + Ug[0, 2] ** 2) / rho)
    assert rho.min() > 0 and p.min() > 0
    if precision == "fp64":
        assert n == len(dts)
        assert rel_linf(Ug, Uo) < FP64_TOL
    else:
        err = np.abs(Ug[0] - Uo[0]).max(axis=1) / np.abs(Uo[0]).max(axis=1)
        print("FP32 limited Riemann rel Linf per component", err)
        assert np.all(err < 1e-3)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_euler_riemann_flux_blending(precision):
    """The four-quadrant states of the batched workload's solve 244 on its own
    8,192-triangle mesh: with the scale limiter alone the first step loses
    positivity, so the flux blending is active from the first step.  The
    single-solve kernels against the oracle, 12 steps."""
    k = 244
    mesh = I.jittered_box(I.config4_sizes(256)[k], seed=4000 + k)
    U0 = I.initial_state(mesh, I.quadrant_fn(I.quadrant_states(4 + k)), 4, nq=4)
    o = oracle.Oracle(mesh, "euler", positivity=True)
    dts, U = [], U0
    for _ in range(12):
        dts.append(o.cfl_dt(U))
        U = o.step(U, dts[-1])
    s = hweno.Solver(mesh, U0, eq="euler", precision=precision, positivity=True)
    for dt in dts:
        s.step(dt)
    Ug, t = s.get_state()
    rho = Ug[0, 0]; p = 0.4 * (Ug[0, 3] - 0.5 * (Ug[0, 1] ** 2 + Ug[0, 2] ** 2) / rho)
    assert rho.min() > 0 and p.min() > 0
    err = rel_linf(Ug, U)
    area = I.cell_areas(mesh)
    l1 = ((np.abs(Ug - U) * area).sum(axis=-1) / np.maximum((np.abs(U) * area).sum(axis=-1), 1e-300)).max()
    print(f"{precision} flux-blended Riemann, 12 steps: relative Linf {err:.2e}, relative L1 {l1:.2e}")
    if precision == "fp64":
        # shocked, limited data: the parity norm of R24 (relative L1 1e-12,
        # relative Linf 1e-10); rounding is amplified in a few cells at the jumps
        assert l1 < FP64_TOL and err < 1e-10
    else:
        assert err < 1e-3


@pytest.mark.parametrize("eq", ["advection", "burgers", "euler"])
def test_gauss_legendre_time_rule_matches_oracle(eq):
    """The two-node Gauss-Legendre time rule (a template variant of the edge
    kernel) against the oracle with the same rule: FP64 after the full run at
    1e-12, FP32 within the FP32 bounds of the default rule."""
    L = 10.0 if eq == "euler" else 2.0
    mesh = I.jittered_periodic(13, L, 0.15, seed=81)   # 338 cells: several tiles and a ragged tail
    m = 4 if eq == "euler" else 1
    fn = I.vortex if eq == "euler" else (I.advection_sine if eq == "advection" else I.burgers_sine)
    T = 0.4 if eq == "euler" else 0.1
    U0 = I.initial_state(mesh, fn, m)
    Uo, dts = oracle.Oracle(mesh, eq, time_rule="gauss").run_to(U0, T)
    Ul, _ = oracle.Oracle(mesh, eq).run_to(U0, T)
    if eq == "advection":
        # linear flux of quadratic Taylor data: both rules integrate it exactly
        assert rel_linf(Uo, Ul) < 1e-12
    else:
        # the rules differ (higher-degree integrands): the comparison below is not vacuous
        assert rel_linf(Uo, Ul) > 1e-13
    s = hweno.Solver(mesh, U0, eq=eq, precision="fp64", time_rule="gauss")
    assert s.run_to(T) == len(dts)
    Ug, t = s.get_state()
    assert rel_linf(Ug, Uo) < FP64_TOL
    s32 = hweno.Solver(mesh, U0, eq=eq, precision="fp32", time_rule="gauss")
    s32.run_to(T)
    U32, _ = s32.get_state()
    err = np.abs(U32[0] - Uo[0]).max(axis=1) / np.abs(Uo[0]).max(axis=1)
    print(f"Gauss-Legendre time rule, {eq}: FP64 {rel_linf(Ug, Uo):.2e}, FP32 W {err.max():.2e}")
    assert err.max() < 1e-5


def test_gauss_legendre_time_rule_refused_by_the_adjoint():
    mesh = I.jittered_periodic(5, 10.0, seed=1)
    U0 = I.initial_state(mesh, I.vortex, 4)
    s = hweno.Solver(mesh, U0, eq="euler", precision="fp64", time_rule="gauss")
    a, b = s.state_buffer(), s.state_buffer()
    with pytest.raises(hweno.HwError) as e:
        s.step_adjoint(0.01, a, b, a, s.adjoint_scratch())
    assert e.value.status == hweno.HW_EINVAL
