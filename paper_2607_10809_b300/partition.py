"""Partition of one mesh over several ranks (one GPU each) with a halo exchange
per time step, and the split of a batch of independent solves over ranks.

Single mesh.  The cells, in the library's Hilbert order, are cut into P
contiguous ranges.  Rank r holds its owned cells plus two rings of halo cells
around them.  That is what one step needs: the reconstruction of a first-ring
cell reads the averages of its own neighbours (second ring, Section 2.2), and
the flux at an owned cell's edge needs the first-ring cell's time-Taylor data
at that edge (Section 2.1).  A step is then

  1. dt = min over ranks of each rank's CFL step (every cell's state is valid
     on every rank that holds it, so the local minima cover all cells);
  2. every rank advances its local mesh by dt; its owned cells are now right,
     its halo cells are not;
  3. every owned cell that lies in another rank's halo is sent there (one
     point-to-point exchange per neighbouring pair).

The local mesh lists its cells in ascending global index, so that "the cell
with the lower index" (the canonical orientation of an edge) is the same on
every rank and in the single-process run.  Its outer rim is an open boundary;
the cells next to it are second-ring cells, whose updates are overwritten by
the exchange.

Batch.  Independent solves need no exchange: they are dealt to ranks by size
(longest first, to the least loaded rank).

The module holds no arithmetic of the scheme.  The per-rank stepper is passed
in: anything with cfl_dt(), step(dt), get() and set(U, t).
"""
from __future__ import annotations

import dataclasses
from typing import Protocol

import numpy as np

from . import inputs as I


class Stepper(Protocol):
    def cfl_dt(self) -> float: ...              # CFL step of the current local state
    def step(self, dt: float) -> None: ...      # advance every local cell by dt
    def get(self) -> np.ndarray: ...            # local state U[3, m, nloc]
    def set(self, U: np.ndarray, t: float) -> None: ...


@dataclasses.dataclass
class Part:
    rank: int
    cells: np.ndarray          # global ids of the local cells, ascending
    owned: np.ndarray          # bool [nloc]: owned by this rank
    mesh: I.Mesh               # the local mesh (local numbering)
    send: dict                 # rank q -> local indices of owned cells that q holds as halo
    recv: dict                 # rank q -> local indices of halo cells owned by q (same order as q's send)


def neighbours(mesh: I.Mesh) -> np.ndarray:
    """Neighbour across local edge j of every triangle (-1: boundary), by
    matching edge keys; [nt, 3]."""
    nt = mesh.nt
    a = mesh.tri.astype(np.int64)
    b = np.roll(a, -1, axis=1)
    lo, hi = np.minimum(a, b).ravel(), np.maximum(a, b).ravel()
    key = lo * (mesh.nv + 1) + hi
    order = np.argsort(key, kind="stable")
    ks = key[order]
    nbr = -np.ones(3 * nt, dtype=np.int64)
    same = np.nonzero(ks[1:] == ks[:-1])[0]
    i, j = order[same], order[same + 1]
    nbr[i] = j // 3
    nbr[j] = i // 3
    return nbr.reshape(nt, 3)


def _ring(cells: np.ndarray, nbr: np.ndarray) -> np.ndarray:
    nb = nbr[cells].ravel()
    return np.unique(nb[nb >= 0])


def build(mesh: I.Mesh, order: np.ndarray, nparts: int) -> list:
    """Parts of `mesh` for `nparts` ranks; `order` is the cell order whose
    contiguous ranges become the owned sets (the library's Hilbert order,
    hw_mesh_permutation)."""
    nt = mesh.nt
    if not 1 <= nparts <= nt:
        raise ValueError("need 1 <= nparts <= number of cells")
    nbr = neighbours(mesh)
    bounds = np.linspace(0, nt, nparts + 1).round().astype(int)
    owner = np.empty(nt, dtype=np.int64)
    for r in range(nparts):
        owner[order[bounds[r]:bounds[r + 1]]] = r
    parts = []
    for r in range(nparts):
        own = np.sort(order[bounds[r]:bounds[r + 1]])
        ring1 = np.setdiff1d(_ring(own, nbr), own)
        ring2 = np.setdiff1d(_ring(ring1, nbr), np.union1d(own, ring1))
        cells = np.union1d(own, np.union1d(ring1, ring2))
        local = I.Mesh(xy=mesh.xy, tri=mesh.tri[cells], Lx=mesh.Lx, Ly=mesh.Ly, bc=1)
        if mesh.edge_bc is not None:
            # an edge to a cell outside the part is on the local mesh's outer
            # rim: open (transmissive) there, whatever the caller's array holds
            # for that edge, which is interior to the whole mesh
            ebc = np.array(mesh.edge_bc[cells], dtype=np.int32)
            nb = nbr[cells]
            ebc[(nb >= 0) & ~np.isin(nb, cells)] = I.BC_TRANSMISSIVE
            local.edge_bc = ebc
        # keep only the vertices the local cells use
        used = np.unique(local.tri)
        remap = -np.ones(mesh.nv, dtype=np.int64)
        remap[used] = np.arange(used.size)
        local.xy = mesh.xy[used].copy()
        local.tri = remap[local.tri].astype(np.int32)
        owned = owner[cells] == r
        parts.append(Part(rank=r, cells=cells, owned=owned, mesh=local, send={}, recv={}))
    # exchange lists: q's halo cells owned by r, in ascending global id on both sides
    for p in parts:
        for q in parts:
            if p.rank == q.rank:
                continue
            halo_q = q.cells[~q.owned]
            shared = halo_q[owner[halo_q] == p.rank]
            if shared.size:
                p.send[q.rank] = np.searchsorted(p.cells, shared)
                q.recv[p.rank] = np.searchsorted(q.cells, shared)
    return parts


def scatter_state(U: np.ndarray, part: Part) -> np.ndarray:
    """The local state of a part from a global state U[3, m, nt]."""
    return np.ascontiguousarray(U[:, :, part.cells])


def gather_state(parts: list, locals_: list, nt: int) -> np.ndarray:
    """The global state from the parts' local states (owned cells only)."""
    m = locals_[0].shape[1]
    U = np.empty((3, m, nt))
    for p, Ul in zip(parts, locals_):
        U[:, :, p.cells[p.owned]] = Ul[:, :, p.owned]
    return U


def exchange_local(parts: list, states: list) -> None:
    """The halo exchange of one step when all parts live in one process
    (states[r] is part r's local state, updated in place)."""
    for p in parts:
        for q, idx in p.send.items():
            states[q][:, :, parts[q].recv[p.rank]] = states[p.rank][:, :, idx]


def run_local(parts: list, steppers: list, nsteps: int, t0: float = 0.0) -> float:
    """Advance every part by nsteps common CFL steps in one process (parts
    emulated one after another; no part waits on another).  Returns the time."""
    t = t0
    for _ in range(nsteps):
        dt = min(s.cfl_dt() for s in steppers)
        for s in steppers:
            s.step(dt)
        t += dt
        states = [s.get() for s in steppers]
        exchange_local(parts, states)
        for s, U in zip(steppers, states):
            s.set(U, t)
    return t


def run_distributed(part: Part, stepper: Stepper, nsteps: int, t0: float = 0.0, device="cpu") -> float:
    """Advance this rank's part by nsteps steps: a min all-reduce of the CFL
    step and a point-to-point halo exchange per step (torch.distributed; gloo
    on host tensors, NCCL on device tensors)."""
    import torch
    import torch.distributed as dist
    t = t0
    for _ in range(nsteps):
        dt = torch.tensor([stepper.cfl_dt()], dtype=torch.float64, device=device)
        dist.all_reduce(dt, op=dist.ReduceOp.MIN)
        dt = float(dt.item())
        stepper.step(dt)
        t += dt
        U = stepper.get()
        reqs, inbox = [], {}
        for q, idx in sorted(part.send.items()):
            buf = torch.from_numpy(np.ascontiguousarray(U[:, :, idx])).to(device)
            reqs.append(dist.isend(buf, dst=q))
        for q, idx in sorted(part.recv.items()):
            inbox[q] = torch.empty((U.shape[0], U.shape[1], idx.size), dtype=torch.float64, device=device)
            reqs.append(dist.irecv(inbox[q], src=q))
        for r in reqs:
            r.wait()
        for q, idx in part.recv.items():
            U[:, :, idx] = inbox[q].cpu().numpy()
        stepper.set(U, t)
    return t


def deal_solves(sizes, nranks: int) -> list:
    """Independent solves dealt to ranks by size: longest first, each to the
    rank with the fewest cells so far.  Returns the solve indices of every rank."""
    loads = [0] * nranks
    out = [[] for _ in range(nranks)]
    for k in sorted(range(len(sizes)), key=lambda i: (-sizes[i], i)):
        r = min(range(nranks), key=lambda q: (loads[q], q))
        out[r].append(k)
        loads[r] += sizes[k]
    return [sorted(o) for o in out]


class SolverStepper:
    """A part's solver on the GPU: an hweno.Solver on the part's local mesh
    (no target time is set, so its device step is the plain CFL step)."""

    def __init__(self, solver):
        self.s = solver

    def cfl_dt(self) -> float:
        return self.s.time()[1]

    def step(self, dt: float) -> None:
        self.s.step(dt)

    def get(self) -> np.ndarray:
        return self.s.get_state()[0]

    def set(self, U: np.ndarray, t: float) -> None:
        self.s.set_state(U, t)


class DeviceStepper:
    """A part's solver with its halo exchange in device memory: after a step
    the rows of the cells another part holds are gathered from the state
    (hw_state_rows_export: the cell's record and, in FP32, its compensation
    words), the rows of the halo cells are written back into the state
    (hw_state_rows_import), and the CFL step is recomputed from the updated
    state.  Only halo rows move, so the partitioned run is the single run bit
    for bit at a cost set by the halo, not by the part."""

    def __init__(self, solver, part: Part):
        import torch
        self.s = solver
        self.part = part
        perm = solver.mesh.permutation()           # perm[k] = local index of internal cell k
        inv = np.empty_like(perm)
        inv[perm] = np.arange(perm.size)
        self.dtype = torch.float32 if solver.precision == "fp32" else torch.float64
        self.width = solver.state_row_words()
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.send_rows = {q: torch.from_numpy(inv[idx].astype(np.int32)).to(self.device) for q, idx in part.send.items()}
        self.recv_rows = {q: torch.from_numpy(inv[idx].astype(np.int32)).to(self.device) for q, idx in part.recv.items()}

    def cfl_dt(self) -> float:
        return self.s.time()[1]

    def step(self, dt: float) -> None:
        self.s.step(dt)

    def export(self) -> None:
        """Nothing to do: outgoing() reads the rows straight from the state."""

    def outgoing(self, q):
        import torch
        rows = self.send_rows[q]
        out = torch.empty((rows.numel(), self.width), dtype=self.dtype, device=self.device)
        self.s.state_rows_export(rows, out)
        return out

    def incoming(self, q, data) -> None:
        self.s.state_rows_import(self.recv_rows[q], data.contiguous())

    def commit(self, t: float) -> None:
        """The halo rows are in: recompute the CFL step (the time advanced with
        the step on the device)."""
        self.s.state_rows_import(refresh=True)

    def get(self) -> np.ndarray:
        return self.s.get_state()[0]


def run_local_device(parts: list, steppers: list, nsteps: int, t0: float = 0.0) -> float:
    """run_local with DeviceSteppers: the halo rows move device to device."""
    t = t0
    for _ in range(nsteps):
        dt = min(s.cfl_dt() for s in steppers)
        for s in steppers:
            s.step(dt)
            s.export()
        t += dt
        for p in parts:
            for q in p.send:
                steppers[q].incoming(p.rank, steppers[p.rank].outgoing(q))
        for s in steppers:
            s.commit(t)
    return t


def run_distributed_device(part: Part, stepper: "DeviceStepper", nsteps: int, t0: float = 0.0) -> float:
    """run_distributed with a DeviceStepper: the min all-reduce and the halo
    rows as device tensors (NCCL)."""
    import torch
    import torch.distributed as dist
    t = t0
    dev = stepper.device
    for _ in range(nsteps):
        dt = torch.tensor([stepper.cfl_dt()], dtype=torch.float64, device=dev)
        dist.all_reduce(dt, op=dist.ReduceOp.MIN)
        dt = float(dt.item())
        stepper.step(dt)
        stepper.export()
        t += dt
        reqs, inbox = [], {}
        for q in sorted(part.send):
            reqs.append(dist.isend(stepper.outgoing(q), dst=q))
        for q in sorted(part.recv):
            inbox[q] = torch.empty((stepper.recv_rows[q].numel(), stepper.width), dtype=stepper.dtype, device=dev)
            reqs.append(dist.irecv(inbox[q], src=q))
        for r in reqs:
            r.wait()
        for q, data in inbox.items():
            stepper.incoming(q, data)
        stepper.commit(t)
    return t
