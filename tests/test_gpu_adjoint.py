"""Adjoint of the step and the differentiable rollout (checkpointed), against
the FP64 oracle's exact directional derivatives (forward-mode dual numbers)
and against central finite differences of the GPU forward."""
import numpy as np
import pytest
import torch

import oracle
from paper_2607_10809_b300 import build as B
from paper_2607_10809_b300 import hweno
from paper_2607_10809_b300 import inputs as I
from paper_2607_10809_b300.adjoint import cfl_steps, rollout

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available()
    B.build()
    hweno.load()


def bumped_vortex(mesh, seed=5):
    bumps = I.vortex_bumps(seed)
    return I.initial_state(mesh, lambda x, y: I.vortex(x, y, bumps=bumps), 4)


def gradient(solver, U0, ubar, dts, every):
    x = torch.from_numpy(U0.copy()).requires_grad_(True)
    UT = rollout(x, solver, dts, every)
    (UT * torch.from_numpy(ubar)).sum().backward()
    return x.grad.numpy(), UT.detach().numpy()


def test_adjoint_matches_oracle_directional_derivatives_fp64():
    mesh = I.jittered_periodic(7, 10.0, 0.15, seed=31)
    U0 = bumped_vortex(mesh)
    o = oracle.Oracle(mesh, "euler")
    dts = [0.5 * o.cfl_dt(U0)] * 4
    rng = np.random.default_rng(55)
    ubar = rng.normal(size=U0.shape)
    s = hweno.Solver(mesh, U0, eq="euler", precision="fp64")
    g, UT = gradient(s, U0, ubar, dts, every=2)
    np.testing.assert_allclose(UT, o.run_dts(U0, dts), rtol=0, atol=1e-12 * np.abs(UT).max())
    for _ in range(4):
        d = rng.normal(size=U0.shape) * np.abs(U0).mean(axis=2, keepdims=True)
        _, dUT = o.run_dual(U0, d, dts)
        lhs = float((ubar * dUT).sum())
        rhs = float((g * d).sum())
        assert abs(lhs - rhs) <= 1e-10 * abs(lhs), (lhs, rhs)


def test_checkpoint_interval_does_not_change_the_gradient():
    mesh = I.jittered_periodic(9, 10.0, 0.15, seed=32)
    U0 = bumped_vortex(mesh)
    s = hweno.Solver(mesh, U0, eq="euler", precision="fp64")
    dts = cfl_steps(s, U0, 12)
    ubar = np.random.default_rng(3).normal(size=U0.shape)
    g1, _ = gradient(s, U0, ubar, dts, every=1)
    g5, _ = gradient(s, U0, ubar, dts, every=5)
    g12, _ = gradient(s, U0, ubar, dts, every=12)
    assert np.array_equal(g1, g5) and np.array_equal(g1, g12)


def misfit_setup(n=24, steps=30, seed=5):
    mesh = I.jittered_periodic(n, 10.0, 0.15, seed=seed)
    U0 = bumped_vortex(mesh, seed)
    area = oracle.Oracle(mesh, "euler").cell_geometry()["area"]
    return mesh, U0, area, steps


def test_misfit_gradient_against_finite_differences_32_directions():
    """J = 1/2 sum_K |K| (rho_K(T) - rho*_K)^2 with rho* the unperturbed
    vortex; the adjoint gradient against central differences of the FP64 GPU
    forward on 32 random directions (relative 1e-6).  The discrete map has
    kinks (|.| in the nonlinear weights, max in the viscosity); a difference
    step h crosses some of them, which adds an error growing like h (measured:
    up to 8e-2 at h = 1e-3, 4e-4 at 1e-4, 2e-5 at 1e-5, 8.4e-7 at 1e-6 over
    these 32 directions), so h = 1e-7; rounding in J (about 1e-16 relative)
    adds only about 1e-10 relative to the quotient at that step."""
    mesh, U0, area, steps = misfit_setup()
    s = hweno.Solver(mesh, U0, eq="euler", precision="fp64")
    dts = cfl_steps(s, U0, steps)
    T = float(np.sum(dts))
    rho_star = I.cell_averages(mesh, lambda x, y: I.vortex(x, y, T), 4)[0]

    def J(U):
        s.set_state(U, 0.0)
        for dt in dts:
            s.step(dt)
        UT, _ = s.get_state()
        return 0.5 * float((area * (UT[0, 0] - rho_star) ** 2).sum()), UT

    J0, UT = J(U0)
    ubar = np.zeros_like(UT); ubar[0, 0] = area * (UT[0, 0] - rho_star)
    g, _ = gradient(s, U0, ubar, dts, every=10)
    rng = np.random.default_rng(55)
    worst = 0.0
    for _ in range(32):
        d = rng.normal(size=U0.shape) * np.abs(U0).mean(axis=2, keepdims=True)
        h = 1e-7
        fd = (J(U0 + h * d)[0] - J(U0 - h * d)[0]) / (2 * h)
        ad = float((g * d).sum())
        worst = max(worst, abs(fd - ad) / abs(fd))
    print(f"adjoint vs central differences, 32 directions: worst relative difference {worst:.2e}")
    assert worst < 1e-6


def test_fp32_adjoint_against_fp64():
    mesh, U0, area, steps = misfit_setup(n=20, steps=20)
    s64 = hweno.Solver(mesh, U0, eq="euler", precision="fp64")
    dts = cfl_steps(s64, U0, steps)
    ubar = np.zeros_like(U0); ubar[0, 0] = area
    g64, _ = gradient(s64, U0, ubar, dts, every=10)
    s32 = hweno.Solver(mesh, U0, eq="euler", precision="fp32")
    g32, _ = gradient(s32, U0, ubar, dts, every=10)
    err = np.abs(g32 - g64).max() / np.abs(g64).max()
    print(f"FP32 adjoint vs FP64 adjoint: relative Linf {err:.2e}")
    assert err < 1e-3


def test_adjoint_rejects_unsupported_configurations():
    mesh = I.jittered_periodic(5, 2.0, seed=1)
    U0 = I.initial_state(mesh, I.burgers_sine, 1)
    s = hweno.Solver(mesh, U0, eq="burgers", precision="fp64")
    a, b = s.state_buffer(), s.state_buffer()
    with pytest.raises(hweno.HwError) as e:
        s.step_adjoint(0.01, a, b, a, s.adjoint_scratch())
    assert e.value.status == hweno.HW_EINVAL


def test_kept_edge_point_data_equals_the_recomputed_one():
    """hw_step_keep leaves the step unchanged and its edge-point data make
    hw_step_adjoint give bit-for-bit the result of the recomputing path."""
    mesh = I.jittered_periodic(11, 10.0, 0.15, seed=33)
    U0 = bumped_vortex(mesh)
    for prec in ("fp64", "fp32"):
        s = hweno.Solver(mesh, U0, eq="euler", precision=prec)
        dt = 0.5 * s.time()[1]
        s.step(dt)
        U1_plain, _ = s.get_state()
        s.set_state(U0, 0.0)
        un, pb = s.state_buffer(), s.pb_buffer()
        s.export_state(un)
        s.step_keep(dt, pb)
        U1_keep, _ = s.get_state()
        assert np.array_equal(U1_plain, U1_keep), prec
        ub, a, b, scratch = s.state_buffer(), s.state_buffer(), s.state_buffer(), s.adjoint_scratch()
        s.host_to_internal(np.random.default_rng(4).normal(size=U0.shape), ub)
        s.step_adjoint(dt, un, ub, a, scratch)
        s.step_adjoint(dt, un, ub, b, scratch, pb)
        assert np.array_equal(s.internal_to_host(a), s.internal_to_host(b)), prec
