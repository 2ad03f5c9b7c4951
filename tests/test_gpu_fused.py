"""The fused reconstruct-and-flux kernel (one launch per step, edge-point
records kept in shared memory, the halo of each tile reconstructed by the
tile) against the FP64 CPU oracle and against the two-kernel step, through
the C ABI."""
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
    num = np.abs(a - b).max(axis=-1)
    den = np.maximum(np.abs(b).max(axis=-1), 1e-300)
    return (num / den).max()


CASES = {
    # name: (mesh, equation, initial data, final time, options)
    "advection-structured": (lambda: I.config1_mesh(20), "advection", I.advection_sine, 0.3, {}),
    "burgers-jittered-shock": (lambda: I.jittered_periodic(24, 4.0, 0.15, seed=2), "burgers", I.burgers_sine,
                               1.5 / np.pi, {}),
    "vortex-poisson": (lambda: I.poisson_delaunay_periodic(10.0, 700, seed=3), "euler", I.vortex, 0.4, {}),
    "vortex-jittered-gauss": (lambda: I.jittered_periodic(21, 10.0, 0.15, seed=7), "euler", I.vortex, 0.4,
                              {"time_rule": "gauss"}),
    "riemann-box-transmissive": (lambda: I.jittered_box(16, seed=44), "euler",
                                 I.quadrant_fn(I.quadrant_states(44)), 0.05, {}),
    "tiny-ragged": (lambda: I.jittered_periodic(5, 2.0, seed=75), "burgers", I.burgers_sine, 0.05, {}),
}


@pytest.mark.parametrize("case", list(CASES))
def test_fused_fp64_matches_oracle(case):
    mk, eq, fn, T, opts = CASES[case]
    mesh = mk()
    m = 4 if eq == "euler" else 1
    U0 = I.initial_state(mesh, fn, m, nq=4 if "riemann" in case else 6)
    Uo, dts = oracle.Oracle(mesh, eq, **opts).run_to(U0, T)
    s = hweno.Solver(mesh, U0, eq=eq, precision="fp64", step_kernels="fused", **opts)
    assert s.step_kernels() == "fused"
    n = s.run_to(T)
    Ug, t = s.get_state()
    assert n == len(dts) and abs(t - T) < 1e-14
    err = rel_linf(Ug, Uo)
    print(f"fused FP64 {case} ({mesh.nt} cells, {n} steps): relative Linf {err:.2e}")
    assert err < FP64_TOL


def test_fused_with_scale_limiter_and_flux_blending():
    """Four-quadrant data of the batched workload's solve 244 on its 8,192-cell
    mesh: the limiter and the blending are active from the first step."""
    k = 244
    mesh = I.jittered_box(I.config4_sizes(256)[k], seed=4000 + k)
    U0 = I.initial_state(mesh, I.quadrant_fn(I.quadrant_states(4 + k)), 4, nq=4)
    o = oracle.Oracle(mesh, "euler", positivity=True)
    dts, U = [], U0
    for _ in range(6):
        dts.append(o.cfl_dt(U))
        U = o.step(U, dts[-1])
    out = {}
    for kern in ("fused", "separate"):
        s = hweno.Solver(mesh, U0, eq="euler", precision="fp64", positivity=True, step_kernels=kern)
        for dt in dts:
            s.step(dt)
        out[kern] = s.get_state()[0]
        print(f"{kern} limited FP64, 6 steps: relative Linf to the oracle {rel_linf(out[kern], U):.2e}")
    # the two GPU paths run the same device code on the same data; the compiler
    # may contract multiply-adds differently in the two kernels
    assert rel_linf(out["fused"], out["separate"]) < 1e-12
    area = I.cell_areas(mesh)
    l1 = ((np.abs(out["fused"] - U) * area).sum(axis=-1) / (np.abs(U) * area).sum(axis=-1)).max()
    assert l1 < FP64_TOL and rel_linf(out["fused"], U) < 1e-10   # the parity norm of shocked, limited runs


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_fused_agrees_with_separate_kernels(precision):
    """Many tiles with halos: the fused and the two-kernel step on a 60,000-cell
    Delaunay mesh, 20 CFL steps."""
    mesh = I.poisson_delaunay_periodic(10.0, 30_000, seed=12)
    U0 = I.initial_state(mesh, I.vortex, 4)
    out = {}
    for kern in ("fused", "separate"):
        s = hweno.Solver(mesh, U0, eq="euler", precision=precision, step_kernels=kern)
        assert s.step_kernels() == kern
        for _ in range(20):
            s.step()
        out[kern] = s.get_state()
        s.close()
    assert out["fused"][1] == out["separate"][1]
    err = rel_linf(out["fused"][0], out["separate"][0])
    same = np.array_equal(out["fused"][0], out["separate"][0])
    print(f"{precision}: fused vs separate relative Linf {err:.2e}, bitwise equal: {same}")
    assert err < (FP64_TOL if precision == "fp64" else 1e-5)


def test_default_step_kernels():
    """The default step: the two-sided flux kernel in FP32, the edge-once flux
    phase in FP64 (where the FP64 pipe bounds the step)."""
    mesh = I.jittered_periodic(12, 10.0, 0.15, seed=3)
    U0 = I.initial_state(mesh, I.vortex, 4)
    for prec, path in (("fp32", "separate"), ("fp64", "edge_once")):
        assert hweno.Solver(mesh, U0, eq="euler", precision=prec).step_kernels() == path


def test_fused_conservation_and_steps_past_the_target():
    """run_to replays a graph of several steps per launch; the steps past the
    target keep the state (the kernel's branch for a reached target), so the
    fused run lands on T bitwise equal to the two-kernel run.  After run_to,
    step() advances again."""
    mesh = I.poisson_delaunay_periodic(10.0, 2_000, seed=9)
    U0 = I.initial_state(mesh, I.vortex, 4)
    s = hweno.Solver(mesh, U0, eq="euler", precision="fp64", step_kernels="fused")
    c0 = s.conservation()
    s.run_to(0.2)
    np.testing.assert_allclose(s.conservation(), c0, rtol=1e-14)
    U1, t1 = s.get_state()
    r = hweno.Solver(mesh, U0, eq="euler", precision="fp64", step_kernels="separate")
    r.run_to(0.2)
    Ur, tr = r.get_state()
    r.close()
    assert abs(t1 - 0.2) < 1e-15 and tr == t1 and np.array_equal(U1, Ur)
    s.step()
    U2, t2 = s.get_state()
    assert t2 > t1 and not np.array_equal(U1, U2)
    s.close()
