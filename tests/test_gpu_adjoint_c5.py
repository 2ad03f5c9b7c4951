"""The gradient workload at its configured size: Euler on the 199,712-triangle
jittered periodic mesh of [0, 10]^2, vortex plus 8 density bumps, 200 steps
with checkpoints every 10; J = 1/2 sum_K |K| (rho_K(T) - rho*_K)^2 with rho*
the unperturbed vortex at T.  The adjoint gradient against central
differences of the FP64 GPU forward on 32 seeded directions, against the
oracle's dual-number directional derivatives on the same mesh (a shortened
rollout, so that the oracle finishes), and the FP32 gradient against FP64."""
import numpy as np
import pytest
import torch

import oracle
from paper_2607_10809_b300 import build as B
from paper_2607_10809_b300 import hweno
from paper_2607_10809_b300 import inputs as I
from paper_2607_10809_b300.adjoint import cfl_steps, rollout

pytestmark = pytest.mark.gpu

STEPS, EVERY = 200, 10


@pytest.fixture(scope="module")
def c5():
    assert torch.cuda.is_available()
    B.build()
    hweno.load()
    mesh = I.config5_mesh()
    U0 = I.config5_state(mesh)
    area = I.cell_areas(mesh)
    s64 = hweno.Solver(mesh, U0, eq="euler", precision="fp64")
    dts = cfl_steps(s64, U0, STEPS)
    T = float(np.sum(dts))
    rho_star = I.cell_averages(mesh, lambda x, y: I.vortex(x, y, T), 4)[0]
    return mesh, U0, area, s64, dts, rho_star


def gradient(solver, U0, dts, area, rho_star):
    x = torch.from_numpy(U0.copy()).requires_grad_(True)
    UT = rollout(x, solver, dts, EVERY)
    J = 0.5 * (torch.from_numpy(area) * (UT[0, 0] - torch.from_numpy(rho_star)) ** 2).sum()
    J.backward()
    return x.grad.numpy()


def test_c5_gradient_against_central_differences_32_directions(c5):
    mesh, U0, area, s, dts, rho_star = c5
    assert mesh.nt == 199_712 and len(dts) == STEPS

    def J(U):
        s.set_state(U, 0.0)
        for dt in dts:
            s.step(dt)
        UT, _ = s.get_state()
        return 0.5 * float((area * (UT[0, 0] - rho_star) ** 2).sum())

    g = gradient(s, U0, dts, area, rho_star)
    rng = np.random.default_rng(55)
    h, worst = 1e-6, 0.0
    for _ in range(32):
        d = rng.normal(size=U0.shape) * np.abs(U0).mean(axis=2, keepdims=True)
        fd = (J(U0 + h * d) - J(U0 - h * d)) / (2 * h)
        ad = float((g * d).sum())
        worst = max(worst, abs(fd - ad) / abs(fd))
    print(f"C5 adjoint vs central differences (h = {h}), 32 directions: worst relative difference {worst:.2e}")
    assert worst < 1e-6


def test_c5_adjoint_against_oracle_dual_numbers(c5):
    """Three steps of the same map: the oracle's forward-mode derivative along
    two seeded directions against <g, d> from the GPU adjoint."""
    mesh, U0, area, s, dts, rho_star = c5
    short = dts[:3]
    rng = np.random.default_rng(7)
    ubar = rng.normal(size=U0.shape)
    x = torch.from_numpy(U0.copy()).requires_grad_(True)
    UT = rollout(x, s, short, 2)
    (UT * torch.from_numpy(ubar)).sum().backward()
    g = x.grad.numpy()
    o = oracle.Oracle(mesh, "euler")
    for _ in range(2):
        d = rng.normal(size=U0.shape) * np.abs(U0).mean(axis=2, keepdims=True)
        _, dUT = o.run_dual(U0, d, short)
        lhs, rhs = float((ubar * dUT).sum()), float((g * d).sum())
        print(f"C5, 3 steps: dual {lhs:.15e} adjoint {rhs:.15e}")
        assert abs(lhs - rhs) <= 1e-10 * abs(lhs)


def test_c5_fp32_gradient_against_fp64(c5):
    mesh, U0, area, s64, dts, rho_star = c5
    g64 = gradient(s64, U0, dts, area, rho_star)
    s32 = hweno.Solver(mesh, U0, eq="euler", precision="fp32")
    g32 = gradient(s32, U0, dts, area, rho_star)
    err = float(np.abs(g32 - g64).max() / np.abs(g64).max())
    print(f"C5 FP32 gradient vs FP64: relative Linf {err:.2e}")
    assert err < 1e-4
