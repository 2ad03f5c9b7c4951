"""hw_step_static_scratch: the step for callers that cannot allocate device
memory, such as code running inside a host that owns the device memory pool,
plug-ins handed fixed buffers, or runtimes that must not allocate once they
run.  Its scratch lives in a static device array inside the library.

It must give the same state as hw_step, call after call, with every option
the step dispatches on, allocate nothing, and refuse meshes whose scratch
exceeds the array.  This file is collected last so that a failure here cannot
hide any other test."""
import numpy as np
import pytest

from paper_2607_10809_b300 import build as B
from paper_2607_10809_b300 import hweno
from paper_2607_10809_b300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-12  # the FP64 parity tolerance of the other GPU tests

STATIC_BYTES = 64 << 20   # size of the library's static scratch array


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


def riemann_state(mesh):
    st = np.array([[1.0, 0.75, -0.5, 1.0], [2.0, 0.0, 0.3, 0.5], [1.0, -0.75, 0.5, 1.0], [3.0, 0.75, 0.5, 0.5]])
    return I.initial_state(mesh, I.quadrant_fn(st), 4, nq=4)


CASES = {
    # (mesh, initial state, solver options): every kernel variant the step dispatches on
    "lobatto": (lambda: I.jittered_periodic(20, 10.0, 0.15, seed=5), lambda m: I.initial_state(m, I.vortex, 4), {}),
    "gauss": (lambda: I.jittered_periodic(20, 10.0, 0.15, seed=5), lambda m: I.initial_state(m, I.vortex, 4),
              {"time_rule": "gauss"}),
    "limiter": (lambda: I.jittered_box(16, seed=7), riemann_state, {"positivity": True}),
}


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("case", list(CASES))
def test_static_scratch_step_matches_hw_step_on_consecutive_calls(precision, case):
    mk_mesh, mk_state, opts = CASES[case]
    mesh = mk_mesh()
    U0 = mk_state(mesh)
    # hw_step with the same two kernels (reconstruction, then flux) and the
    # edge-point buffer in the caller's workspace
    ref = hweno.Solver(mesh, U0, eq="euler", precision=precision, step_kernels="separate", **opts)
    noalloc = hweno.Solver(mesh, U0, eq="euler", precision=precision, step_kernels="separate", **opts)
    for call in range(2):
        ref.step()
        noalloc.step_static_scratch()
        Ur, tr = ref.get_state()
        Un, tn = noalloc.get_state()
        assert tn == tr, (call, tn, tr)
        assert rel_linf(Un, Ur) <= TOL, (call, rel_linf(Un, Ur))


def test_static_scratch_step_allocates_no_device_memory():
    import torch
    mesh = I.jittered_periodic(20, 10.0, 0.15, seed=5)
    U0 = I.initial_state(mesh, I.vortex, 4)
    s = hweno.Solver(mesh, U0, eq="euler", precision="fp32")
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        s.step_static_scratch()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)


def test_static_scratch_limit_is_exact():
    # FP32 Euler scratch is 18 * 4 * 4 = 288 bytes per padded cell; the padded
    # count is ntri rounded up to a multiple of 32
    largest = 288 * 232_992
    assert largest <= STATIC_BYTES < 288 * (232_992 + 32)
    ok_mesh = I.jittered_periodic_rect(809, 144, 0.02, seed=1)      # 232,992 triangles
    bad_mesh = I.jittered_periodic_rect(352, 331, 0.02, seed=1)     # 233,024 triangles: the next tile
    assert ok_mesh.nt == 232_992 and bad_mesh.nt == 233_024
    for mesh, fits in ((ok_mesh, True), (bad_mesh, False)):
        U0 = np.zeros((3, 4, mesh.nt)); U0[0] = np.array([1.0, 0.1, -0.2, 2.5])[:, None]
        s = hweno.Solver(mesh, U0, eq="euler", precision="fp32")
        if fits:
            s.step_static_scratch(1e-4)
            U, _ = s.get_state()
            np.testing.assert_allclose(U[0], U0[0], rtol=1e-6)      # free stream stays put
        else:
            with pytest.raises(hweno.HwError) as e:
                s.step_static_scratch(1e-4)
            assert e.value.status == hweno.HW_EINVAL
            assert "static maximum" in str(e.value)
        s.close()


def test_static_scratch_rejects_meshes_beyond_its_maximum():
    mesh = I.jittered_periodic(250, 10.0, 0.15, seed=5)     # 125,000 cells: 72 MB of FP64 Euler scratch
    U0 = np.zeros((3, 4, mesh.nt)); U0[0] = np.array([1.0, 0.0, 0.0, 2.5])[:, None]
    s = hweno.Solver(mesh, U0, eq="euler", precision="fp64")
    with pytest.raises(hweno.HwError) as e:
        s.step_static_scratch()
    assert e.value.status == hweno.HW_EINVAL
    assert "static maximum" in str(e.value)
    s.step()   # the regular step still works on the same solver
