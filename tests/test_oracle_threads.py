"""The oracle's OpenMP build: the per-node loops of a step run over rows in
parallel, and the state and heat grids must be bitwise the same as with one
thread (each value is computed alone, in the same order of operations)."""

import numpy as np
import pytest

import oracle
from paper_1102_1343_gb300 import synth


def run(w, threads, steps):
    oracle.set_threads(threads)
    try:
        f = oracle.OracleFire.from_workload(w)
        hs = hl = None
        for _ in range(steps):
            hs, hl, _ = f.step(w.u, w.v, w.dt)
        return f, hs, hl
    finally:
        oracle.set_threads(1)


def test_thread_count_does_not_change_results(orc):
    if oracle.set_threads(4) == 1:
        pytest.skip("oracle built without OpenMP")
    oracle.set_threads(1)
    w = synth.random_landscape(9, 7, seed=12, ignition="line", steps=1)
    a, hsa, hla = run(w, 1, 25)
    b, hsb, hlb = run(w, 4, 25)
    assert np.isfinite(a.tign).any()
    for x, y in ((a.psi, b.psi), (a.tign, b.tign), (a.frac, b.frac), (hsa, hsb), (hla, hlb)):
        assert np.array_equal(x, y)
    assert a.t == b.t


def test_set_threads_reports_count(orc):
    n = oracle.set_threads(3)
    assert n in (1, 3)
    assert oracle.set_threads(1) == 1
