"""Reflective walls and inflow/outflow boundaries (the shock tubes of Section 3)
on the GPU against the FP64 CPU oracle, through the C ABI."""
import os
import sys

import numpy as np
import pytest

import oracle
from paper_2607_10809_b300 import build as B
from paper_2607_10809_b300 import hweno
from paper_2607_10809_b300 import inputs as I

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
from test_oracle_pins import _channel_and_mirror, _symmetric_flow  # noqa: E402

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


def rel_l1(a, b, area):
    """Area-weighted L1 difference over the L1 norm, per plane, maximum."""
    num = (np.abs(a - b) * area).sum(axis=-1)
    den = np.maximum((np.abs(b) * area).sum(axis=-1), 1e-300)
    return (num / den).max()


def pressure(U):
    return 0.4 * (U[0, 3] - 0.5 * (U[0, 1] ** 2 + U[0, 2] ** 2) / U[0, 0])


@pytest.mark.parametrize("kernels", ["separate", "fused"])
def test_wall_channel_fp64(kernels):
    """Smooth flow in a channel with walls at y = 0 and y = 1, 20 CFL steps."""
    ch, _ = _channel_and_mirror(nx=12, ny=8)
    U0 = I.initial_state(ch, _symmetric_flow, 4)
    Uo, dts = oracle.Oracle(ch, "euler").run_to(U0, 0.1)
    s = hweno.Solver(ch, U0, eq="euler", precision="fp64", step_kernels=kernels)
    n = s.run_to(0.1)
    Ug, _ = s.get_state()
    assert n == len(dts)
    err = rel_linf(Ug, Uo)
    print(f"{kernels} wall channel, {n} steps: relative Linf {err:.2e}")
    assert err < FP64_TOL


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_lax_tube(precision):
    """The Lax problem: inflow on the left, outflow on the right, walls at the
    top and bottom, scale limiter and flux blending; 60 steps with the
    oracle's time steps."""
    mesh, fn, T, win = I.lax_tube()
    U0 = I.initial_state(mesh, fn, 4, nq=4)
    o = oracle.Oracle(mesh, "euler", positivity=True, inflow=win)
    dts, U = [], U0
    for _ in range(60):
        dts.append(o.cfl_dt(U))
        U = o.step(U, dts[-1])
    s = hweno.Solver(mesh, U0, eq="euler", precision=precision, positivity=True, inflow=win)
    for dt in dts:
        s.step(dt)
    Ug, _ = s.get_state()
    area = o.cell_geometry()["area"]
    assert Ug[0, 0].min() > 0 and pressure(Ug).min() > 0
    linf, l1 = rel_linf(Ug, U), rel_l1(Ug, U, area)
    print(f"{precision} Lax tube, 60 steps: relative Linf {linf:.2e}, relative L1 {l1:.2e}")
    if precision == "fp64":
        assert l1 < FP64_TOL and linf < 1e-10
    else:
        assert rel_linf(Ug[:1], U[:1]) < 1e-3


def test_blast_waves_keep_positivity_and_match_the_oracle():
    """The interacting blast waves (walls on all sides, pressure ratio 1e5):
    40 steps in FP64 against the oracle, and the FP32 form keeps density and
    pressure positive."""
    mesh, fn, T = I.blast_waves()
    U0 = I.initial_state(mesh, fn, 4, nq=4)
    o = oracle.Oracle(mesh, "euler", positivity=True)
    dts, U = [], U0
    for _ in range(40):
        dts.append(o.cfl_dt(U))
        U = o.step(U, dts[-1])
    area = o.cell_geometry()["area"]
    for prec in ("fp64", "fp32"):
        s = hweno.Solver(mesh, U0, eq="euler", precision=prec, positivity=True)
        for dt in dts:
            s.step(dt)
        Ug, _ = s.get_state()
        assert Ug[0, 0].min() > 0 and pressure(Ug).min() > 0
        l1 = rel_l1(Ug, U, area)
        print(f"{prec} blast waves, 40 steps: relative L1 {l1:.2e}, relative Linf {rel_linf(Ug, U):.2e}")
        assert l1 < (FP64_TOL if prec == "fp64" else 1e-4)
    # the walls conserve mass and energy
    c0 = (U0[0] * area).sum(axis=1)
    np.testing.assert_allclose((U[0] * area).sum(axis=1)[[0, 3]], c0[[0, 3]], rtol=1e-13)


def test_batched_lax_tubes_match_the_single_solve_path():
    meshes, states, wins = [], [], []
    for seed in (1, 2, 3):
        mesh, fn, T, win = I.lax_tube(seed=seed)
        meshes.append(mesh); states.append(I.initial_state(mesh, fn, 4, nq=4)); wins.append(win)
    b = hweno.Batch(meshes, states, eq="euler", precision="fp64", positivity=True, inflow=wins[0])
    b.run_to(0.02)
    for k in range(3):
        s = hweno.Solver(meshes[k], states[k], eq="euler", precision="fp64", positivity=True, inflow=wins[0])
        s.run_to(0.02)
        Us, ts = s.get_state()
        Ub, tb, _, f = b.get_state(k)
        assert not f and abs(tb - ts) < 1e-14
        assert rel_linf(Ub, Us) < FP64_TOL


def test_adjoint_refuses_walls():
    ch, _ = _channel_and_mirror()
    U0 = I.initial_state(ch, _symmetric_flow, 4)
    s = hweno.Solver(ch, U0, eq="euler", precision="fp64")
    buf = [s.state_buffer() for _ in range(3)]
    with pytest.raises(hweno.HwError) as e:
        s.step_adjoint(1e-3, buf[0], buf[1], buf[2], s.adjoint_scratch())
    assert e.value.status == hweno.HW_EINVAL
