"""The serving loop (ss_server_*): requests submitted while others are on the
device are admitted by memory footprint into waves of the persistent solver
(or into the single-system lane), and each result is the one the same system
gets alone."""
import time

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
    systems += kerr_sweep(8, seed=11)
    systems += [jaynes_cummings_rwa(seed=s, N=12) for s in range(3)]     # shared pattern
    return systems


def test_served_results_equal_alone(ss):
    systems = _mix()
    large = jaynes_cummings_rwa(seed=1, N=80)                           # n = 25,600: the single-system lane
    with ss.Server(precision="mixed", tol=1e-10, max_waves=3, max_wave_systems=4) as srv:
        tickets = [srv.submit(s.H, s.c_ops) for s in systems]
        t_large = srv.submit(large.H, large.c_ops)
        served = [srv.wait(t, timeout_s=120) for t in tickets]
        rho_large, info_large, _ = srv.wait(t_large, timeout_s=300)
        stats = srv.stats()
    assert stats["completed"] == len(systems) + 1 and stats["waves"] >= 2
    for s, (rho, info, lat) in zip(systems, served):
        assert info["status"] == 0 and info["resid_Lrho"] <= 1e-10, s.name
        alone, _ = ss.steady_state_batched([(s.H, s.c_ops)], tol=1e-10, precision="mixed")
        assert np.array_equal(rho, alone[0]), s.name                    # same arithmetic alone and in the mix
        assert lat > 0
    ref, _ = ss.steady_state(large.H, large.c_ops, tol=1e-10, precision="fp64")   # the lane solves in FP64
    assert info_large["status"] == 0 and info_large["resid_Lrho"] <= 1e-10
    assert trace_distance(rho_large, ref) <= 1e-12
    for s, (rho, _, _) in zip(systems[:4], served[:4]):               # and against the oracle
        assert trace_distance(rho, steady_state_dense(s.H, s.c_ops)) <= 1e-8


def test_budget_limits_admission(ss):
    """A budget of a few requests: the rest wait in the queue, every request
    still completes, in several waves."""
    systems = kerr_sweep(24, seed=5)
    budget_mb = 12.0                                                  # a few of these requests at a time
    with ss.Server(precision="mixed", hbm_budget_mb=budget_mb, max_waves=4, max_wave_systems=8) as srv:
        tickets = [srv.submit(s.H, s.c_ops) for s in systems]
        out = [srv.wait(t, timeout_s=300) for t in tickets]
        stats = srv.stats()
        assert stats["in_use_mb"] == 0.0 and stats["budget_mb"] == pytest.approx(budget_mb)
    assert stats["waves"] >= 4
    for s, (rho, info, _) in zip(systems, out):
        assert info["status"] == 0 and info["resid_Lrho"] <= 1e-10
        assert abs(np.trace(rho) - 1) < 1e-12


def test_poisson_arrivals_report_latency(ss):
    rng = np.random.default_rng(0)
    systems = kerr_sweep(40, seed=2) + [jaynes_cummings_rwa(seed=s, N=16) for s in range(10)]
    order = rng.permutation(len(systems))
    with ss.Server(precision="mixed") as srv:
        tickets = []
        for k in order:
            time.sleep(rng.exponential(1.0 / 400.0))                   # 400 requests/s
            tickets.append(srv.submit(systems[k].H, systems[k].c_ops))
        lat = [srv.wait(t, timeout_s=120)[2] for t in tickets]
    lat = np.array(lat)
    assert np.all(lat > 0)
    p50, p99 = np.percentile(lat, [50, 99])
    assert p50 <= p99 < 60_000


def test_oversized_request_rejected(ss):
    s = jaynes_cummings_rwa(seed=0, N=12)
    with ss.Server(precision="mixed", hbm_budget_mb=0.1) as srv:
        with pytest.raises(ss.SolverError) as e:
            srv.submit(s.H, s.c_ops)
        assert e.value.status == 2


def test_wait_timeout_leaves_request_queryable(ss):
    s = jaynes_cummings_rwa(seed=2, N=80)
    with ss.Server(precision="mixed") as srv:
        t = srv.submit(s.H, s.c_ops)
        with pytest.raises(TimeoutError):
            srv.wait(t, timeout_s=0.0)
        rho, info, lat = srv.wait(t, timeout_s=300)
        assert info["status"] == 0 and lat > 0


def test_served_sweep_warm_starts_from_earlier_requests(ss):
    """With warm_start, a request starts from the stored state of the closest
    earlier request with the same pattern: a drive sweep served point after
    point reaches the same states (against the cold server and the oracle)
    in fewer iterations, and a repeated request needs almost none."""
    sweep = [jaynes_cummings_rwa(N=12, E=0.5 + 0.005 * k) for k in range(8)]

    def serve(warm):
        out = []
        with ss.Server(precision="mixed", tol=1e-10, warm_start=warm) as srv:
            for s in sweep + sweep[3:4]:                   # the last request repeats an earlier one
                out.append(srv.wait(srv.submit(s.H, s.c_ops), timeout_s=120))
        return out

    cold, warm = serve(False), serve(True)
    for s, (rc, ic, _), (rw, iw, _) in zip(sweep + sweep[3:4], cold, warm):
        assert ic["status"] == 0 and iw["status"] == 0 and iw["resid_Lrho"] <= 1e-10
        assert trace_distance(rc, rw) <= 1e-8
    assert trace_distance(warm[5][0], steady_state_dense(sweep[5].H, sweep[5].c_ops)) <= 1e-8
    assert sum(i["iters"] for _, i, _ in warm[1:8]) < sum(i["iters"] for _, i, _ in cold[1:8])
    assert warm[8][1]["iters"] <= 2 < cold[8][1]["iters"]
