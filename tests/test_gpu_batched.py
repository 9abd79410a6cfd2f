"""GPU parity of the per-system persistent solver (steady_state_batched):
against the CPU oracle, against the single-system path, and alone versus in
a mixed batch."""
import numpy as np
import pytest

from oracle.metrics import trace_distance
from oracle.steady import steady_state_dense
from workloads import driven_cavity, jaynes_cummings_rwa, kerr_sweep, thermal_cavity, two_level_atom

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


def _mix():
    systems = [driven_cavity(n_th=0.0), driven_cavity(n_th=0.2), thermal_cavity(n_th=0.2), two_level_atom()]
    systems += kerr_sweep(6, seed=3)
    systems += [jaynes_cummings_rwa(seed=s, N=12) for s in range(3)]      # shared pattern
    return systems


@pytest.mark.parametrize("precision,tol,td", [("fp64", 1e-12, 1e-10), ("mixed", 1e-10, 1e-8)])
def test_batched_matches_oracle(ss, precision, tol, td):
    systems = _mix()
    rhos, infos = ss.steady_state_batched([(s.H, s.c_ops) for s in systems], tol=tol, precision=precision)
    for s, rho, info in zip(systems, rhos, infos):
        assert info["status"] == 0, (s.name, info)
        assert info["resid_Lrho"] <= tol
        assert trace_distance(rho, steady_state_dense(s.H, s.c_ops)) <= td, s.name
        assert abs(np.trace(rho) - 1) < 1e-12


def test_batched_alone_equals_in_mix(ss):
    """Each system's result is the same alone and inside a mixed batch."""
    systems = _mix()
    rhos, _ = ss.steady_state_batched([(s.H, s.c_ops) for s in systems], tol=1e-10, precision="mixed")
    for k in (0, 5, len(systems) - 1):
        alone, _ = ss.steady_state_batched([(systems[k].H, systems[k].c_ops)], tol=1e-10, precision="mixed")
        assert np.array_equal(alone[0], rhos[k])


def test_batched_agrees_with_single_system_path(ss):
    systems = [jaynes_cummings_rwa(seed=s, N=16) for s in range(4)]
    rhos, infos = ss.steady_state_batched([(s.H, s.c_ops) for s in systems], tol=1e-12)
    for s, rho in zip(systems, rhos):
        single, _ = ss.steady_state(s.H, s.c_ops, tol=1e-12)
        assert trace_distance(rho, single) <= 1e-10


def test_batched_jc40_full_size(ss):
    systems = [jaynes_cummings_rwa(seed=s) for s in (0, 5)]
    rhos, infos = ss.steady_state_batched([(s.H, s.c_ops) for s in systems], tol=1e-12)
    for s, rho, info in zip(systems, rhos, infos):
        assert info["n"] == 6400 and info["status"] == 0
        assert trace_distance(rho, steady_state_dense(s.H, s.c_ops)) <= 1e-10


def test_batched_kerr_sweep_uneven(ss):
    """The uneven Kerr sweep (cutoffs 8..64, n = 64..4096), mixed precision,
    against FP64 single-system solves on a sample."""
    systems = kerr_sweep(48, seed=0)
    rhos, infos = ss.steady_state_batched([(s.H, s.c_ops) for s in systems], tol=1e-10, precision="mixed")
    assert all(i["status"] == 0 and i["resid_Lrho"] <= 1e-10 for i in infos)
    for k in range(0, 48, 8):
        ref = steady_state_dense(systems[k].H, systems[k].c_ops)
        assert trace_distance(rhos[k], ref) <= 1e-8


def test_batched_falls_back_for_other_methods(ss):
    systems = [driven_cavity(n_th=0.2), thermal_cavity()]
    rhos, infos = ss.steady_state_batched([(s.H, s.c_ops) for s in systems], method="iterative-lgmres",
                                          tol=1e-12)
    for s, rho, info in zip(systems, rhos, infos):
        assert info["status"] == 0
        assert trace_distance(rho, steady_state_dense(s.H, s.c_ops)) <= 1e-10
