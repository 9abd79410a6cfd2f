"""Warm-started parameter sweeps: a solve may start from a neighbouring sweep
point's steady state (the sweeps over drive strength of the paper's
results).  The answer is the same steady state (the method's fixed point does
not depend on the start), reached in fewer iterations; a guess of zero trace
gives exactly the cold solve."""
import numpy as np
import pytest

from oracle.metrics import trace_distance
from oracle.steady import steady_state_dense
from workloads import jaynes_cummings_rwa

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ss():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import __graft_entry__ as g
    g.build()
    import paper_1504_06768_gb300 as lib
    return lib


def _sweep(count, N=20, E0=0.6, dE=0.02):
    return [jaynes_cummings_rwa(N=N, E=E0 + k * dE) for k in range(count)]


@pytest.mark.parametrize("precision,tol,td", [("fp64", 1e-12, 1e-10), ("mixed", 1e-10, 1e-8)])
def test_batched_warm_start_same_state_fewer_iterations(ss, precision, tol, td):
    systems = _sweep(12)
    pairs = [(s.H, s.c_ops) for s in systems]
    cold, ci = ss.steady_state_batched(pairs, tol=tol, precision=precision)
    # each point starts from its left neighbour's state (the first from its right one)
    guesses = [cold[1]] + cold[:-1]
    warm, wi = ss.steady_state_batched(pairs, tol=tol, precision=precision, rho_init=guesses)
    for s, a, b, info in zip(systems, cold, warm, wi):
        assert info["status"] == 0 and info["resid_Lrho"] <= tol
        assert trace_distance(a, b) <= td
        assert abs(np.trace(b) - 1) < 1e-12
    assert trace_distance(warm[5], steady_state_dense(systems[5].H, systems[5].c_ops)) <= td
    assert np.mean([i["iters"] for i in wi]) < np.mean([i["iters"] for i in ci])


def test_batched_warm_start_zero_trace_is_cold(ss):
    systems = _sweep(3)
    pairs = [(s.H, s.c_ops) for s in systems]
    cold, _ = ss.steady_state_batched(pairs, tol=1e-10, precision="mixed")
    zeros = [np.zeros((s.d, s.d), dtype=complex) for s in systems]
    warm, _ = ss.steady_state_batched(pairs, tol=1e-10, precision="mixed", rho_init=zeros)
    for a, b in zip(cold, warm):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("method", ["iterative-bicgstab", "iterative-lgmres", "inverse-power"])
def test_single_system_warm_start(ss, method):
    a, b = _sweep(2, N=16, dE=0.05)
    ra, _ = ss.steady_state(a.H, a.c_ops, method=method, tol=1e-12)
    cold, ci = ss.steady_state(b.H, b.c_ops, method=method, tol=1e-12)
    warm, wi = ss.steady_state(b.H, b.c_ops, method=method, tol=1e-12, rho_init=ra)
    assert wi["status"] == 0 and wi["resid_Lrho"] <= 1e-12
    assert trace_distance(cold, warm) <= 1e-10
    assert trace_distance(warm, steady_state_dense(b.H, b.c_ops)) <= 1e-10
    if method == "iterative-bicgstab":
        # (restarted GMRES need not gain: its cycles restart from the smaller residual either way)
        assert wi["iters"] < ci["iters"]


def test_single_system_warm_start_device_buffer(ss):
    """The guess may sit in the device output buffer (rho_on_device)."""
    import torch
    a, b = _sweep(2, N=12, dE=0.05)
    ra, _ = ss.steady_state(a.H, a.c_ops, tol=1e-12, precision="mixed")
    out = torch.empty(b.d * b.d, dtype=torch.complex128, device="cuda")
    warm, wi = ss.steady_state(b.H, b.c_ops, tol=1e-12, out=out, rho_init=ra)
    host, _ = ss.steady_state(b.H, b.c_ops, tol=1e-12, rho_init=ra)
    assert wi["status"] == 0
    assert trace_distance(warm.cpu().numpy(), host) <= 1e-12
