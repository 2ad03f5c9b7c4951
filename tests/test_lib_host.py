"""Host-side checks of the C-ABI library (no GPU needed): it loads, exports every
declared symbol, and its FP64 mesh precompute matches the oracle bit for bit
on connectivity."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from paper_2607_10809_b300 import build as B
from paper_2607_10809_b300 import hweno
from paper_2607_10809_b300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return hweno.load()


def header_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(hw_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_library_exports_every_declared_symbol(lib):
    names = header_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(hweno.EXPORTED)


MESHES = {
    "structured": lambda: I.config1_mesh(10),
    "jittered": lambda: I.jittered_periodic(9, 4.0, seed=2),
    "poisson": lambda: I.poisson_delaunay_periodic(10.0, 400, seed=3),
    "box": lambda: I.jittered_box(8, seed=4),
}


@pytest.mark.parametrize("name", list(MESHES))
def test_connectivity_bit_exact_against_oracle(lib, name):
    mesh = MESHES[name]()
    m = hweno.Mesh(mesh)
    nbr, nbe = m.neighbors()
    onbr, onbe = oracle.Oracle(mesh).neighbors()
    np.testing.assert_array_equal(nbr, onbr)
    np.testing.assert_array_equal(nbe, onbe)


def test_hilbert_order_is_a_permutation_with_local_neighbours(lib):
    mesh = I.jittered_periodic(64, 4.0, seed=2)
    m = hweno.Mesh(mesh)
    p = m.permutation()
    assert np.array_equal(np.sort(p), np.arange(mesh.nt))
    inv = np.empty_like(p); inv[p] = np.arange(mesh.nt)
    nbr, _ = m.neighbors()
    d = np.abs(inv[nbr] - inv[:, None])
    # most neighbours lie within a few warps of each other in the internal order
    assert np.median(d) < 64
    assert np.mean(d < 1024) > 0.9


def test_mesh_errors_are_reported(lib):
    mesh = I.jittered_periodic(4, 1.0, seed=1)
    bad = mesh.tri.copy(); bad[0, 0] = mesh.nv + 5
    with pytest.raises(hweno.HwError) as e:
        hweno.hw_mesh_create(mesh.xy, bad, 1.0, 1.0, 0)
    assert e.value.status == hweno.HW_EINVAL
    dup = np.concatenate([mesh.tri, mesh.tri[:1]])
    with pytest.raises(hweno.HwError) as e:
        hweno.hw_mesh_create(mesh.xy, dup, 1.0, 1.0, 0)
    assert e.value.status == hweno.HW_EMESH
    cw = mesh.tri.copy(); cw[3] = cw[3, ::-1]
    with pytest.raises(hweno.HwError) as e:
        hweno.hw_mesh_create(mesh.xy, cw, 1.0, 1.0, 0)
    assert e.value.status == hweno.HW_EMESH
    box = I.jittered_box(4)
    with pytest.raises(hweno.HwError) as e:   # open boundary declared periodic
        hweno.hw_mesh_create(box.xy, box.tri, 1.0, 1.0, 0)
    assert e.value.status == hweno.HW_EMESH
    assert "open edge" in str(e.value)


def test_workspace_grows_with_mesh_and_precision(lib):
    a = hweno.Mesh(I.jittered_periodic(8, 1.0, seed=1))
    b = hweno.Mesh(I.jittered_periodic(16, 1.0, seed=1))
    o = hweno.options("euler")
    wa64 = hweno.hw_workspace_bytes(a.h, o, "fp64")
    wb64 = hweno.hw_workspace_bytes(b.h, o, "fp64")
    wb32 = hweno.hw_workspace_bytes(b.h, o, "fp32")
    assert wb64 > 3.5 * wa64 and wb32 < wb64
    with pytest.raises(hweno.HwError):
        hweno.hw_workspace_bytes(a.h, hweno.options("euler", cfl=-1.0), "fp64")


def test_empty_and_degenerate_inputs_are_rejected(lib):
    """Empty meshes and batches, and a triangle of zero area, are refused on
    the host with their status (no device work is attempted)."""
    L = hweno.load()
    h = ctypes.c_void_p()
    xy = np.zeros((3, 2)); tri = np.zeros((0, 3), np.int32)
    rc = L.hw_mesh_create(xy.ctypes.data_as(ctypes.c_void_p), 3, tri.ctypes.data_as(ctypes.c_void_p), 0,
                          1.0, 1.0, 1, ctypes.byref(h))
    assert rc == hweno.HW_EINVAL and b"empty" in L.hw_last_error()
    # collinear vertices: zero area
    xy = np.array([[0.0, 0.0], [1.0, 0.0], [2.0, 0.0], [0.0, 1.0]])
    tri = np.array([[0, 1, 2], [0, 1, 3]], np.int32)
    rc = L.hw_mesh_create(xy.ctypes.data_as(ctypes.c_void_p), 4, tri.ctypes.data_as(ctypes.c_void_p), 2,
                          0.0, 0.0, 1, ctypes.byref(h))
    assert rc == hweno.HW_EMESH and b"degenerate" in L.hw_last_error()
    o = hweno.options("euler")
    n = ctypes.c_size_t()
    assert L.hw_batch_workspace_bytes(None, 0, ctypes.byref(o), 1, ctypes.byref(n)) == hweno.HW_EINVAL
    b = ctypes.c_void_p()
    rc = L.hw_batch_create(None, 0, ctypes.byref(o), 1, None, None, None, None, 0, None, ctypes.byref(b))
    assert rc == hweno.HW_EINVAL and b"empty" in L.hw_last_error()


def test_time_rule_option_is_checked(lib):
    """The Gauss-Legendre time rule is accepted by the single-solve path, and
    refused with the scale limiter, by the batched form, and as an unknown
    value."""
    mesh = hweno.Mesh(I.jittered_periodic(6, 10.0, seed=2))
    assert hweno.hw_workspace_bytes(mesh.h, hweno.options("euler", time_rule="gauss"), "fp32") > 0
    for bad in (hweno.options("euler", time_rule="gauss", positivity=True),):
        with pytest.raises(hweno.HwError) as e:
            hweno.hw_workspace_bytes(mesh.h, bad, "fp32")
        assert e.value.status == hweno.HW_EINVAL
    o = hweno.options("euler"); o.time_rule = 2
    with pytest.raises(hweno.HwError):
        hweno.hw_workspace_bytes(mesh.h, o, "fp32")
    L = hweno.load()
    arr = (ctypes.c_void_p * 1)(mesh.h)
    n = ctypes.c_size_t()
    og = hweno.options("euler", time_rule="gauss")
    assert L.hw_batch_workspace_bytes(arr, 1, ctypes.byref(og), 1, ctypes.byref(n)) == hweno.HW_EINVAL
    assert b"Gauss-Lobatto" in L.hw_last_error()


@pytest.mark.parametrize("weights,why", [
    ((0.94, 0.02, 0.02, 0.0), "a zero linear weight"),
    ((0.98, 0.03, 0.02, -0.03), "a negative linear weight"),
    ((0.94, 0.02, 0.02, 0.03), "weights summing to 1.01"),
    ((0.5, 0.2, 0.2, 0.09), "weights summing to 0.99"),
])
def test_linear_weights_must_be_positive_and_sum_to_one(lib, weights, why):
    # Section 2.2, Step 3: any positive linear weights summing to one
    m = hweno.Mesh(I.config1_mesh(4))
    with pytest.raises(hweno.HwError) as e:
        hweno.hw_workspace_bytes(m.h, hweno.options("advection", gamma_lin=weights), "fp64")
    assert e.value.status == hweno.HW_EINVAL, why
    assert "linear weight" in str(e.value)
    hweno.hw_workspace_bytes(m.h, hweno.options("advection", gamma_lin=(0.7, 0.1, 0.1, 0.1)), "fp64")


def test_connectivity_bit_exact_against_oracle_on_a_mesh_split_over_threads(lib):
    """A mesh large enough that the precompute splits its passes into many
    ranges over the host's cores: connectivity still equals the oracle's."""
    mesh = I.jittered_periodic(160, 10.0, seed=6)   # 51,200 triangles
    m = hweno.Mesh(mesh)
    nbr, nbe = m.neighbors()
    onbr, onbe = oracle.Oracle(mesh).neighbors()
    np.testing.assert_array_equal(nbr, onbr)
    np.testing.assert_array_equal(nbe, onbe)


_ONE_CPU_CHILD = r"""
import os, sys, hashlib
os.sched_setaffinity(0, {sorted(os.sched_getaffinity(0))[0]})
sys.path.insert(0, sys.argv[1])
from paper_2607_10809_b300 import hweno, inputs as I
m = hweno.Mesh(I.jittered_periodic(160, 10.0, seed=6))
nbr, nbe = m.neighbors()
print(hashlib.sha256(nbr.tobytes() + nbe.tobytes() + m.permutation().tobytes()).hexdigest())
"""


def test_mesh_precompute_does_not_depend_on_the_thread_count(lib):
    """The host precompute runs its passes on the CPUs the process may use;
    restricted to one CPU it gives the same neighbours and Hilbert order."""
    import hashlib
    import subprocess
    import sys
    if len(os.sched_getaffinity(0)) < 2:
        pytest.skip("one CPU available: nothing to compare")
    m = hweno.Mesh(I.jittered_periodic(160, 10.0, seed=6))
    nbr, nbe = m.neighbors()
    here = hashlib.sha256(nbr.tobytes() + nbe.tobytes() + m.permutation().tobytes()).hexdigest()
    out = subprocess.run([sys.executable, "-c", _ONE_CPU_CHILD, ROOT], capture_output=True, text=True, check=True)
    assert out.stdout.strip() == here


def test_mesh_faults_are_reported_in_triangle_order(lib):
    """With two faults, the message is the one a scan of the triangles in the
    caller's order meets first."""
    mesh = I.jittered_periodic(4, 1.0, seed=1)
    degen = mesh.tri.copy(); degen[2, 1] = degen[2, 0]
    a = np.concatenate([degen, mesh.tri[:1]])                  # repeated vertex first, duplicate last
    b = np.concatenate([mesh.tri[:1], mesh.tri[:1], degen])    # duplicate first, repeated vertex later
    with pytest.raises(hweno.HwError, match="degenerate"):
        hweno.hw_mesh_create(mesh.xy, a, 1.0, 1.0, 0)
    with pytest.raises(hweno.HwError, match="non-manifold"):
        hweno.hw_mesh_create(mesh.xy, b, 1.0, 1.0, 0)
