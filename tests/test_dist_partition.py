"""The single-mesh partition with a per-step halo exchange (host logic), on CPU:
the CPU oracle stands in for each rank's GPU solver.  Partitioned runs, in
one process and on two gloo ranks (host-array exchange, and the device path's
row exchange with CPU tensors), must reproduce the single-process run to
1e-12; the batch split must balance the solves."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2607_10809_b300 import build as B
from paper_2607_10809_b300 import hweno
from paper_2607_10809_b300 import inputs as I
from paper_2607_10809_b300 import partition as PT

TOL = 1e-12


class OracleStepper:
    """A rank's solver, played by the oracle on the rank's local mesh."""

    def __init__(self, mesh, U, **kw):
        self.o = oracle.Oracle(mesh, "euler", **kw)
        self.U = np.ascontiguousarray(U)

    def cfl_dt(self):
        return self.o.cfl_dt(self.U)

    def step(self, dt):
        self.U = self.o.step(self.U, dt)

    def get(self):
        return self.U.copy()

    def set(self, U, t):
        self.U = np.ascontiguousarray(U)


class OracleRowStepper(OracleStepper):
    """The device stepper's interface (halo rows handed over as tensors, the
    dt minimum as a tensor all-reduce) played by the oracle on CPU tensors, so
    that the NCCL path's exchange logic runs over gloo."""

    def __init__(self, mesh, U, part, **kw):
        import torch
        super().__init__(mesh, U, **kw)
        self.m = self.U.shape[1]
        self.width = 3 * self.m
        self.dtype = torch.float64
        self.device = torch.device("cpu")
        self.send_rows = {q: torch.from_numpy(np.asarray(idx, dtype=np.int64)) for q, idx in part.send.items()}
        self.recv_rows = {q: torch.from_numpy(np.asarray(idx, dtype=np.int64)) for q, idx in part.recv.items()}

    def export(self):
        pass

    def outgoing(self, q):
        import torch
        idx = self.send_rows[q].numpy()
        return torch.from_numpy(np.ascontiguousarray(self.U[:, :, idx].reshape(self.width, idx.size).T))

    def incoming(self, q, data):
        idx = self.recv_rows[q].numpy()
        self.U[:, :, idx] = data.numpy().T.reshape(3, self.m, idx.size)

    def commit(self, t):
        pass


def cases():
    vortex = I.jittered_periodic(14, 10.0, 0.15, seed=5)
    box, fn, _, win = I.lax_tube(seed=4)
    return {
        "vortex-periodic": (vortex, I.initial_state(vortex, I.vortex, 4), {}),
        "lax-walls-inflow": (box, I.initial_state(box, fn, 4, nq=4), {"positivity": True, "inflow": win}),
    }


def order_of(mesh):
    B.build()
    hweno.load()
    return hweno.Mesh(mesh).permutation()


def single_run(mesh, U, kw, nsteps):
    o = oracle.Oracle(mesh, "euler", **kw)
    for _ in range(nsteps):
        U = o.step(U, o.cfl_dt(U))
    return U


def rel_linf(a, b):
    return (np.abs(a - b).max(axis=-1) / np.maximum(np.abs(b).max(axis=-1), 1e-300)).max()


def test_partition_tables():
    mesh = I.jittered_periodic(14, 10.0, 0.15, seed=5)
    parts = PT.build(mesh, order_of(mesh), 3)
    owned = np.concatenate([p.cells[p.owned] for p in parts])
    assert np.array_equal(np.sort(owned), np.arange(mesh.nt))          # every cell owned once
    nbr = PT.neighbours(mesh)
    for p in parts:
        assert np.all(np.diff(p.cells) > 0)                             # ascending global ids
        own = p.cells[p.owned]
        ring1 = np.unique(nbr[own].ravel())
        ring2 = np.unique(nbr[ring1].ravel())
        assert np.isin(ring2, p.cells).all()                            # two rings around the owned cells
        for q, idx in p.send.items():
            assert np.array_equal(p.cells[idx], parts[q].cells[parts[q].recv[p.rank]])
            assert p.owned[idx].all() and not parts[q].owned[parts[q].recv[p.rank]].any()
    # the exchanged halo covers every halo cell exactly once
    for p in parts:
        got = np.concatenate([idx for idx in p.recv.values()]) if p.recv else np.array([], int)
        assert np.array_equal(np.sort(got), np.nonzero(~p.owned)[0])


def test_partition_rim_edges_are_open_whatever_the_interior_edge_types():
    """Boundary types are read only on boundary edges, so the caller may leave
    anything at interior edges; the parts' outer rims are boundary edges of
    their local meshes and must come out transmissive, not the caller's value."""
    mesh, U0, kw = cases()["lax-walls-inflow"]
    nbr = PT.neighbours(mesh)
    mesh.edge_bc = np.where(nbr >= 0, 0, mesh.edge_bc).astype(np.int32)   # 0: not a boundary type
    nsteps = 4
    ref = single_run(mesh, U0, kw, nsteps)
    parts = PT.build(mesh, order_of(mesh), 3)
    for p in parts:
        lnbr = PT.neighbours(p.mesh)
        assert np.isin(p.mesh.edge_bc[lnbr < 0], (I.BC_TRANSMISSIVE, I.BC_REFLECTIVE, I.BC_INFLOW)).all()
    steppers = [OracleStepper(p.mesh, PT.scatter_state(U0, p), **kw) for p in parts]
    PT.run_local(parts, steppers, nsteps)
    U = PT.gather_state(parts, [s.get() for s in steppers], mesh.nt)
    assert rel_linf(U, ref) < TOL


@pytest.mark.parametrize("case", ["vortex-periodic", "lax-walls-inflow"])
def test_partition_in_one_process_matches_the_single_run(case):
    mesh, U0, kw = cases()[case]
    nsteps = 6
    ref = single_run(mesh, U0, kw, nsteps)
    parts = PT.build(mesh, order_of(mesh), 3)
    steppers = [OracleStepper(p.mesh, PT.scatter_state(U0, p), **kw) for p in parts]
    PT.run_local(parts, steppers, nsteps)
    U = PT.gather_state(parts, [s.get() for s in steppers], mesh.nt)
    assert rel_linf(U, ref) < TOL


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, case, nsteps, out):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        mesh, U0, kw = cases()[case]
        parts = PT.build(mesh, order_of(mesh), world)
        p = parts[rank]
        st = OracleStepper(p.mesh, PT.scatter_state(U0, p), **kw)
        t = PT.run_distributed(p, st, nsteps)
        out[rank] = (st.get(), t)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("case", ["vortex-periodic", "lax-walls-inflow"])
def test_partition_on_two_gloo_ranks_matches_the_single_run(case):
    world, nsteps = 2, 5
    mesh, U0, kw = cases()[case]
    ref = single_run(mesh, U0, kw, nsteps)
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(world, _free_port(), case, nsteps, out), nprocs=world, join=True)
    parts = PT.build(mesh, order_of(mesh), world)
    U = PT.gather_state(parts, [out[r][0] for r in range(world)], mesh.nt)
    assert abs(out[0][1] - out[1][1]) == 0.0
    assert rel_linf(U, ref) < TOL


def _worker_rows(rank, world, port, case, nsteps, out):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        mesh, U0, kw = cases()[case]
        parts = PT.build(mesh, order_of(mesh), world)
        p = parts[rank]
        st = OracleRowStepper(p.mesh, PT.scatter_state(U0, p), p, **kw)
        t = PT.run_distributed_device(p, st, nsteps)
        out[rank] = (st.get(), t)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("case", ["vortex-periodic", "lax-walls-inflow"])
def test_row_exchange_path_on_two_gloo_ranks_matches_the_single_run(case):
    """run_distributed_device (halo rows as tensors, isend / irecv, dt by a
    tensor all-reduce) over gloo with CPU tensors."""
    world, nsteps = 2, 5
    mesh, U0, kw = cases()[case]
    ref = single_run(mesh, U0, kw, nsteps)
    out = mp.Manager().dict()
    mp.spawn(_worker_rows, args=(world, _free_port(), case, nsteps, out), nprocs=world, join=True)
    parts = PT.build(mesh, order_of(mesh), world)
    U = PT.gather_state(parts, [out[r][0] for r in range(world)], mesh.nt)
    assert abs(out[0][1] - out[1][1]) == 0.0
    assert rel_linf(U, ref) < TOL


def test_deal_solves_balances_sizes():
    sizes = [int(2 * n * n) for n in I.config4_sizes(256)]     # triangles of the batched solves
    for nranks in (1, 2, 4, 8):
        deal = PT.deal_solves(sizes, nranks)
        assert sorted(k for d in deal for k in d) == list(range(len(sizes)))
        loads = [sum(sizes[k] for k in d) for d in deal]
        assert max(loads) - min(loads) <= max(sizes)
        assert max(loads) <= sum(sizes) / nranks * 1.01 + max(sizes)
