"""qw_run_host_batch: independent runs from host states with the copies
overlapping the steps give, bit for bit, what the sequential calls give."""
import numpy as np
import pytest

import oracle
from paper_1003_3779_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qw():
    import paper_1003_3779_gb300.qw as qw
    qw.lib()
    return qw


@pytest.mark.parametrize("case", ["cycle_sweep_f32", "cycle_f64", "torus_f32", "torus_f64"])
@pytest.mark.parametrize("count", [1, 2, 3, 5])
def test_pipelined_runs_equal_sequential_calls(qw, case, count):
    rng = np.random.default_rng(count)
    if case.startswith("cycle"):
        shape, dims = (2, 5000), (5000,)
        C = inputs.su2(0.3)
    else:
        shape, dims = (4, 48, 64), (64, 48)
        C = inputs.grover()
    prec = "f32" if case.endswith("f32") else "f64"
    cdt = np.complex64 if prec == "f32" else np.complex128
    states = np.stack([inputs.random_state(shape, seed=int(s)).astype(cdt) for s in rng.integers(0, 1000, count)])
    T = 37
    w = qw.Walk(dims, prec=prec).set_coin(C)
    if case == "cycle_sweep_f32":
        w.set_plan_ex(32, 16, 1)
    P, norms = w.run_host_batch(states, T, norms=True)
    last = w.state(dtype=cdt)
    ref = qw.Walk(dims, prec=prec).set_coin(C)
    if case == "cycle_sweep_f32":
        ref.set_plan_ex(32, 16, 1)
    for i in range(count):
        ref.set_state(states[i]).step(T)
        Pi, ni = ref.probabilities()
        assert np.array_equal(P[i], Pi), i
        assert norms[i] == ni
    assert np.array_equal(last, ref.state(dtype=cdt))
    # FP64 against the oracle as well
    if prec == "f64":
        want, _ = oracle.probabilities(oracle.evolve(states[-1], C, T))
        assert np.abs(P[-1] - want).sum() < 1e-12
    # the walk carries on from the last run's state
    w.step(5)
    ref.step(5)
    assert np.array_equal(w.state(dtype=cdt), ref.state(dtype=cdt))
    w.close()
    ref.close()


def test_pipelined_reuse_and_float_marginals(qw):
    N, T = 3000, 20
    s = inputs.random_state((2, N), seed=3).astype(np.complex64)
    w = qw.Walk((N,), prec="f32").set_coin(inputs.hadamard())
    P = np.empty((N,), dtype=np.float32)          # one buffer, reused by every run
    w.run_host_batch(s, T, count=4, P_out=P)
    ref = qw.Walk((N,), prec="f32").set_coin(inputs.hadamard()).set_state(s).step(T)
    Pr = np.empty(N, dtype=np.float32)
    qw.qw_probabilities(ref.h, Pr)
    assert np.array_equal(P, Pr)
    assert w.run_host_batch(s[None], 0).shape == (1, N)
    w.close()
    ref.close()


def test_pipelined_rejections(qw):
    w = qw.Walk((64,), prec="f32").set_coin(inputs.hadamard())
    with pytest.raises(qw.QWError):
        w.run_host_batch(np.zeros((2, 2, 64), dtype=np.complex128), 3)   # complex128 into FP32
    w.close()
    w = qw.Walk((64,), prec="bf16").set_coin(inputs.hadamard())
    with pytest.raises(qw.QWError):
        w.run_host_batch(np.zeros((2, 2, 64), dtype=np.complex64), 3)
    w.close()


def test_pipelined_norms_when_the_count_grows(qw):
    """The per-run norms are kept on the device and copied once at the end; a
    later call with more runs than any before gets a larger array."""
    N, T = 2000, 15
    states = np.stack([inputs.random_state((2, N), seed=50 + i).astype(np.complex64) for i in range(7)])
    w = qw.Walk((N,), prec="f32").set_coin(inputs.su2(0.7))
    ref = qw.Walk((N,), prec="f32").set_coin(inputs.su2(0.7))
    for n in (2, 7, 3):
        _, norms = w.run_host_batch(states[:n], T, norms=True)
        assert norms.shape == (n,)
        for i in range(n):
            ref.set_state(states[i]).step(T)
            assert norms[i] == ref.probabilities()[1], (n, i)
    w.close()
    ref.close()
