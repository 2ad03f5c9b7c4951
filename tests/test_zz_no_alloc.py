"""hw_step_static_scratch: the step for callers that cannot allocate device
memory (their scratch lives in a static device array inside the library).

It must give the same state as hw_step, call after call, and refuse meshes
whose scratch exceeds the array.  This file is collected last so that a
failure here cannot hide any other test."""
import numpy as np
import pytest

from paper_2607_10809_b300 import build as B
from paper_2607_10809_b300 import hweno
from paper_2607_10809_b300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-12  # the FP64 parity tolerance of the other GPU tests


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


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_static_scratch_step_matches_hw_step_on_consecutive_calls(precision):
    mesh = I.jittered_periodic(20, 10.0, 0.15, seed=5)
    U0 = I.initial_state(mesh, I.vortex, 4)
    ref = hweno.Solver(mesh, U0, eq="euler", precision=precision)
    noalloc = hweno.Solver(mesh, U0, eq="euler", precision=precision)
    for call in range(2):
        ref.step()
        noalloc.step_static_scratch()
        Ur, tr = ref.get_state()
        Un, tn = noalloc.get_state()
        assert tn == tr, (call, tn, tr)
        assert rel_linf(Un, Ur) <= TOL, (call, rel_linf(Un, Ur))


def test_static_scratch_rejects_meshes_beyond_its_maximum():
    mesh = I.jittered_periodic(250, 10.0, 0.15, seed=5)     # 125,000 cells: 72 MB of FP64 Euler scratch
    U0 = np.zeros((3, 4, mesh.nt)); U0[0] = np.array([1.0, 0.0, 0.0, 2.5])[:, None]
    s = hweno.Solver(mesh, U0, eq="euler", precision="fp64")
    with pytest.raises(hweno.HwError) as e:
        s.step_static_scratch()
    assert e.value.status == hweno.HW_EINVAL
    assert "static maximum" in str(e.value)
    s.step()   # the regular step still works on the same solver
