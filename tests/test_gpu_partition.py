"""The single-mesh partition on the GPU: three parts, each an hweno.Solver on
its local mesh, advanced one after another in one process with the host halo
exchange between steps (no part's kernels wait on another's), against the
single-solver run."""
import numpy as np
import pytest

from paper_2607_10809_b300 import build as B
from paper_2607_10809_b300 import hweno
from paper_2607_10809_b300 import inputs as I
from paper_2607_10809_b300 import partition as PT

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    B.build()
    hweno.load()


# FP32: the exchange passes through host arrays (hw_get_state / hw_set_state),
# which fold each cell average's compensation word into the average every
# step, while the single solver keeps it; that costs FP32 roundings.
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-4)])
def test_three_parts_match_one_solver(precision, tol):
    mesh = I.poisson_delaunay_periodic(10.0, 3000, seed=21)
    U0 = I.initial_state(mesh, I.vortex, 4)
    ref = hweno.Solver(mesh, U0, eq="euler", precision=precision)
    nsteps = 8
    for _ in range(nsteps):
        ref.step()
    Ur, tr = ref.get_state()
    parts = PT.build(mesh, hweno.Mesh(mesh).permutation(), 3)
    steppers = [PT.SolverStepper(hweno.Solver(p.mesh, PT.scatter_state(U0, p), eq="euler", precision=precision))
                for p in parts]
    t = PT.run_local(parts, steppers, nsteps)
    U = PT.gather_state(parts, [s.get() for s in steppers], mesh.nt)
    assert abs(t - tr) <= 1e-14 * tr
    err = (np.abs(U - Ur).max(axis=-1) / np.abs(Ur).max(axis=-1)).max()
    print(f"{precision}: 3 parts vs one solver, {nsteps} steps: relative Linf {err:.2e}")
    assert err < tol


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_three_parts_device_exchange_match_one_solver(precision):
    """The same with the halo rows moved device to device (internal state
    buffers, torch indexing): no host round trip.  A row carries the cell's
    record and, in FP32, its compensation words, so the partitioned run is the
    single run bit for bit in both precisions."""
    mesh = I.poisson_delaunay_periodic(10.0, 3000, seed=21)
    U0 = I.initial_state(mesh, I.vortex, 4)
    ref = hweno.Solver(mesh, U0, eq="euler", precision=precision)
    nsteps = 8
    for _ in range(nsteps):
        ref.step()
    Ur, tr = ref.get_state()
    parts = PT.build(mesh, hweno.Mesh(mesh).permutation(), 3)
    steppers = [PT.DeviceStepper(hweno.Solver(p.mesh, PT.scatter_state(U0, p), eq="euler", precision=precision), p)
                for p in parts]
    t = PT.run_local_device(parts, steppers, nsteps)
    U = PT.gather_state(parts, [s.get() for s in steppers], mesh.nt)
    assert abs(t - tr) <= 1e-14 * tr
    err = (np.abs(U - Ur).max(axis=-1) / np.abs(Ur).max(axis=-1)).max()
    print(f"{precision}: 3 parts (device exchange) vs one solver, {nsteps} steps: relative Linf {err:.2e}")
    assert np.array_equal(U, Ur)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_state_rows_match_the_state_buffer(precision):
    """hw_state_rows_export gives the rows of the internal state buffer
    (record, then FP32 compensation words); hw_state_rows_import writes them
    into another solver's state; an index outside [0, ntri) is skipped and
    raises bit 2 of the status flags."""
    import torch
    mesh = I.poisson_delaunay_periodic(10.0, 800, seed=5)
    U0 = I.initial_state(mesh, I.vortex, 4)
    s = hweno.Solver(mesh, U0, eq="euler", precision=precision)
    for _ in range(3):
        s.step()
    buf = s.state_buffer()
    s.export_state(buf)
    dtype = torch.float32 if precision == "fp32" else torch.float64
    words = s.state_row_words()
    assert words == (16 if precision == "fp32" else 12)
    N = mesh.nt
    flat = buf.view(dtype)
    ld = flat.numel() // words
    table = torch.cat([flat[: ld * 12].view(ld, 12)] +
                      ([flat[ld * 12: ld * 16].view(ld, 4)] if precision == "fp32" else []), dim=1)
    rows = torch.tensor([0, 5, N - 1, 17, 5], dtype=torch.int32, device="cuda")
    out = torch.empty((rows.numel(), words), dtype=dtype, device="cuda")
    s.state_rows_export(rows, out)
    assert torch.equal(out, table[rows.long()])
    r = hweno.Solver(mesh, U0, eq="euler", precision=precision)
    r.state_rows_import(rows[:4], out[:4], refresh=True)
    rb = r.state_buffer()
    r.export_state(rb)
    rflat = rb.view(dtype)
    rtable = torch.cat([rflat[: ld * 12].view(ld, 12)] +
                       ([rflat[ld * 12: ld * 16].view(ld, 4)] if precision == "fp32" else []), dim=1)
    assert torch.equal(rtable[rows[:4].long()], out[:4])
    assert s.status_flags() == 0
    bad = torch.tensor([N, -1], dtype=torch.int32, device="cuda")
    s.state_rows_export(bad, torch.zeros((2, words), dtype=dtype, device="cuda"))
    assert s.status_flags() & 4
    s.close(); r.close()
