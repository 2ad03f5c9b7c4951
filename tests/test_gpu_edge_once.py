"""The edge-once flux phase (step_kernels 3: each edge's flux by its left
cell into a per-point buffer, then the update kernel) against the two-kernel
step (step_kernels 1), which evaluates every edge from both sides with the
same canonical-orientation arithmetic: the states must agree bit for bit, in
FP64 and FP32, on periodic, transmissive, wall and inflow boundaries, with the
scale limiter and flux blending and with the Gauss-Legendre time rule."""
import numpy as np
import pytest

from paper_2607_10809_b300 import build as B
from paper_2607_10809_b300 import hweno
from paper_2607_10809_b300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    B.build()
    hweno.load()


def cases():
    c1 = I.config1_mesh(10)
    yield "advection", c1, I.initial_state(c1, I.advection_sine, 1), "advection", {}
    bm = I.jittered_periodic(12, 4.0, 0.15, seed=2)
    yield "burgers", bm, I.initial_state(bm, I.burgers_sine, 1), "burgers", {}
    vm = I.poisson_delaunay_periodic(10.0, 1500, seed=4)
    vU = I.initial_state(vm, I.vortex, 4)
    yield "vortex", vm, vU, "euler", {}
    yield "vortex-gauss", vm, vU, "euler", {"time_rule": "gauss"}
    box = I.jittered_box(14, seed=4001)
    yield "riemann-limited", box, I.initial_state(box, I.quadrant_fn(I.quadrant_states(5)), 4, nq=4), "euler", \
        {"positivity": True}
    lax, fn, _, win = I.lax_tube(seed=1)
    yield "lax-walls-inflow", lax, I.initial_state(lax, fn, 4), "euler", {"positivity": True, "inflow": win}


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_edge_once_equals_two_sided(precision):
    for name, mesh, U0, eq, kw in cases():
        out = {}
        for mode in ("separate", "edge_once"):
            s = hweno.Solver(mesh, U0, eq=eq, precision=precision, step_kernels=mode, **kw)
            assert s.step_kernels() == mode
            for _ in range(12):
                s.step()
            out[mode] = s.get_state()
            s.close()
        (Ua, ta), (Ub, tb) = out["separate"], out["edge_once"]
        assert ta == tb, name
        assert np.array_equal(Ua, Ub), (name, np.abs(Ua - Ub).max())
        print(f"{precision} {name}: edge-once equals two-sided after 12 steps")


def test_edge_once_run_to_and_static_scratch():
    """run_to (captured graph) and the step without caller scratch take the
    edge-once phase too."""
    mesh = I.poisson_delaunay_periodic(10.0, 1500, seed=4)
    U0 = I.initial_state(mesh, I.vortex, 4)
    ref = hweno.Solver(mesh, U0, eq="euler", precision="fp64", step_kernels="separate")
    ref.run_to(0.3)
    s = hweno.Solver(mesh, U0, eq="euler", precision="fp64", step_kernels="edge_once")
    s.run_to(0.3)
    assert np.array_equal(s.get_state()[0], ref.get_state()[0])
    for _ in range(3):
        ref.step()
        s.step_static_scratch()
    assert np.array_equal(s.get_state()[0], ref.get_state()[0])
    s.close(); ref.close()
