"""The FP64 oracle's run to a final time, with each step's cells split over
worker processes (test infrastructure).

Every worker holds the oracle of the whole mesh and computes one contiguous
share of the cells of each step with `step_cells`; the parent computes the
oracle's CFL step, clips the last one to the final time exactly as the
oracle's own `run_to` does, and assembles the new state.  Nothing of the
scheme's arithmetic lives here: the values are the oracle's."""
from __future__ import annotations

import multiprocessing as mp
import os
from multiprocessing import shared_memory

import numpy as np

import oracle


def _worker(conn, mesh, eq, opts, shape, u_name, out_name, lo, hi):
    o = oracle.Oracle(mesh, eq, **opts)
    u_shm = shared_memory.SharedMemory(name=u_name)
    out_shm = shared_memory.SharedMemory(name=out_name)
    U = np.ndarray(shape, dtype=np.float64, buffer=u_shm.buf)
    out = np.ndarray(shape, dtype=np.float64, buffer=out_shm.buf)
    cells = np.arange(lo, hi, dtype=np.int64)
    conn.send("ready")
    try:
        while True:
            msg = conn.recv()
            if msg is None:
                break
            out[:, :, lo:hi] = o.step_cells(U, float(msg), cells)
            conn.send("done")
    finally:
        del U, out
        u_shm.close()
        out_shm.close()


def run_to(mesh, eq, U0, T, workers=None, **opts):
    """(U(T), time steps) of the oracle from U0 [3, m, nt] at t = 0."""
    U0 = np.ascontiguousarray(U0, dtype=np.float64)
    o = oracle.Oracle(mesh, eq, **opts)
    nw = max(1, min(workers or os.cpu_count() or 1, 16, mesh.nt))
    ctx = mp.get_context("spawn")
    u_shm = shared_memory.SharedMemory(create=True, size=U0.nbytes)
    out_shm = shared_memory.SharedMemory(create=True, size=U0.nbytes)
    procs, conns = [], []
    try:
        U = np.ndarray(U0.shape, dtype=np.float64, buffer=u_shm.buf)
        out = np.ndarray(U0.shape, dtype=np.float64, buffer=out_shm.buf)
        U[...] = U0
        bounds = np.linspace(0, mesh.nt, nw + 1).astype(np.int64)
        for w in range(nw):
            a, b = ctx.Pipe()
            p = ctx.Process(target=_worker, args=(b, mesh, eq, opts, U0.shape, u_shm.name, out_shm.name,
                                                  int(bounds[w]), int(bounds[w + 1])), daemon=True)
            p.start()
            procs.append(p)
            conns.append(a)
        for c in conns:
            assert c.recv() == "ready"
        t, dts = 0.0, []
        while t < T * (1.0 - 1e-14):
            dt = o.cfl_dt(U)
            if t + dt > T:
                dt = T - t
            for c in conns:
                c.send(dt)
            for c in conns:
                assert c.recv() == "done"
            U[...] = out
            dts.append(dt)
            t += dt
        result = U.copy()
        del U, out
        return result, np.array(dts)
    finally:
        for c in conns:
            try:
                c.send(None)
            except (BrokenPipeError, OSError):
                pass
        for p in procs:
            p.join(timeout=30)
            if p.is_alive():
                p.kill()
        u_shm.close(); u_shm.unlink()
        out_shm.close(); out_shm.unlink()


def _run_case(args):
    mesh, eq, U0, T, opts = args
    return oracle.Oracle(mesh, eq, **opts).run_to(U0, T)


def run_to_many(cases, workers=None):
    """The oracle's own run_to of each case (mesh, eq, U0, T, options dict),
    one case per worker process; returns [(U(T), time steps)] in order."""
    nw = max(1, min(workers or os.cpu_count() or 1, 16, len(cases)))
    with mp.get_context("spawn").Pool(nw) as pool:
        return pool.map(_run_case, cases)


def _trajectory(args):
    mesh, eq, U0, T, opts = args
    o = oracle.Oracle(mesh, eq, **opts)
    _, dts = o.run_to(U0, T)
    states = [np.asarray(U0, dtype=np.float64).copy()]
    for dt in dts:
        states.append(o.step(states[-1], float(dt)))
    return states, dts


def trajectories_many(cases, workers=None):
    """For each case (mesh, eq, U0, T, options dict): the oracle's states after
    every step of its run to T (the initial state first) and its time steps;
    one case per worker process."""
    nw = max(1, min(workers or os.cpu_count() or 1, 16, len(cases)))
    with mp.get_context("spawn").Pool(nw) as pool:
        return pool.map(_trajectory, cases)
