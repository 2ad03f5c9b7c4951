"""The process-split oracle run used by the full-size parity tests agrees with
the oracle's own run (same steps; values to the rounding of the edge-term
sums at the split points)."""
import numpy as np

import oracle
import oracle_pool
from paper_2607_10809_b300 import inputs as I


def test_split_run_matches_the_oracle_run():
    mesh = I.jittered_periodic(24, 4.0, 0.15, seed=2)
    U0 = I.initial_state(mesh, I.burgers_sine, 1)
    T = 1.5 / np.pi ** 2
    Ua, da = oracle.Oracle(mesh, "burgers").run_to(U0, T)
    Ub, db = oracle_pool.run_to(mesh, "burgers", U0, T, workers=3)
    assert len(da) == len(db)
    np.testing.assert_allclose(db, da, rtol=1e-13)
    scale = np.abs(Ua).max(axis=-1, keepdims=True)
    assert (np.abs(Ub - Ua) / scale).max() < 1e-13


def test_many_runs_are_the_oracle_runs():
    mesh = I.jittered_periodic(8, 4.0, 0.15, seed=3)
    U0 = I.initial_state(mesh, I.burgers_sine, 1)
    cases = [(mesh, "burgers", U0, T, {}) for T in (0.05, 0.1)]
    for (U, dts), (_, _, _, T, _) in zip(oracle_pool.run_to_many(cases, workers=2), cases):
        Ua, da = oracle.Oracle(mesh, "burgers").run_to(U0, T)
        np.testing.assert_array_equal(U, Ua)
        np.testing.assert_array_equal(dts, da)
