"""Serving: requests admitted by device memory and stepped together give the
same result as the same request run alone."""
import numpy as np
import pytest

import workloads
from tests.test_gpu_parity import _fq

pytestmark = pytest.mark.gpu


def _mix():
    h, eri = workloads.synthetic_abinitio(8, 24, 77)
    ab = dict(kind="abinitio", norb=8, n_alpha=3, n_beta=3, h1=h, eri=eri, ecore=0.0)
    return [
        (workloads.hubbard_1d(8, 1.0, 4.0), dict(tau=0.01, target_walkers=2000, seed=11, shift_damping=0.5,
                                                 shift_interval=5)),
        (workloads.hubbard_2d(3, 4, 2.0), dict(tau=0.0, target_walkers=5000, seed=12, initiator_threshold=3.0,
                                               shift_damping=0.5, shift_interval=5)),
        (ab, dict(tau=0.0, target_walkers=3000, seed=13, initiator_threshold=3.0, shift_damping=0.5,
                  shift_interval=5)),
        (workloads.hubbard_1d(10, 1.0, 2.0), dict(tau=0.0, target_walkers=4000, seed=14, shift_damping=0.5,
                                                  shift_interval=5)),
    ]


def test_requests_in_the_mix_equal_alone():
    fq = _fq()
    mix = _mix()
    srv = fq.fciqmc_server_create(8 << 30, max_active=3)
    ids = [fq.fciqmc_server_submit(srv, s, p, target_sigma=1e-12, max_iters=300) for s, p in mix]
    while fq.fciqmc_server_tick(srv, 50) > 0:
        pass
    for (s, p), rid in zip(mix, ids):
        st = fq.fciqmc_server_poll(srv, rid)
        assert st["state_name"] == "max_iters", st
        assert st["iterations"] == 300
        alone = fq.fciqmc_create(s, p)
        fq.fciqmc_step(alone, 300)
        en = fq.fciqmc_energy(alone)
        assert st["tau"] == fq.fciqmc_tau(alone)
        # the walker dynamics, the shift and every statistics row (E_num an
        # exact sum, R12) are bit-identical, and so are E_proj and its error
        assert st["shift"] == en["shift"]
        for k_srv, k_alone in [("energy", "e_proj_mean"), ("sigma", "e_proj_sigma")]:
            a, b = st[k_srv], en[k_alone]
            assert (np.isnan(a) and np.isnan(b)) or a == b, (k_srv, a, b)
        assert st["attempts"] == en["attempts_total"]
        assert st["t_done"] >= st["t_start"] >= st["t_submit"] == st["t_arrival"]


def test_admission_respects_the_memory_budget():
    fq = _fq()
    mix = _mix()
    # a budget that fits roughly one request at a time
    srv = fq.fciqmc_server_create(1, max_active=8)
    ids = [fq.fciqmc_server_submit(srv, s, p, target_sigma=1e-12, max_iters=50) for s, p in mix[:3]]
    fq.fciqmc_server_tick(srv, 50)
    states = [fq.fciqmc_server_poll(srv, i)["state_name"] for i in ids]
    assert states.count("queued") == 2
    while fq.fciqmc_server_tick(srv, 50) > 0:
        pass
    assert all(fq.fciqmc_server_poll(srv, i)["state_name"] == "max_iters" for i in ids)


def test_request_that_cannot_grow_is_retired():
    """A request whose spawn regions must grow past its own device-memory cap
    fails with OUT_OF_MEMORY; the server retires it as failed and the tick
    loop ends, while the other request in the batch still finishes."""
    fq = _fq()
    mix = _mix()
    s, p = mix[0]
    p = dict(p, initial_walkers=2e4, target_walkers=1e5)
    alone = fq.fciqmc_create(s, p)
    cap = fq.fciqmc_layout(alone)["device_bytes"] + (64 << 10)  # no room for larger spawn buffers
    del alone
    srv = fq.fciqmc_server_create(8 << 30, max_active=4)
    bad = fq.fciqmc_server_submit(srv, s, dict(p, max_device_bytes=cap), target_sigma=1e-12, max_iters=100)
    good = fq.fciqmc_server_submit(srv, *mix[1], target_sigma=1e-12, max_iters=100)
    for _ in range(50):  # a handful of ticks; never unbounded
        if fq.fciqmc_server_tick(srv, 20) == 0:
            break
    st = fq.fciqmc_server_poll(srv, bad)
    assert st["state_name"] == "failed" and st["error"] == fq.FCIQMC_ERR_OUT_OF_MEMORY, st
    assert fq.fciqmc_server_poll(srv, good)["state_name"] == "max_iters"
    assert fq.fciqmc_server_tick(srv, 20) == 0


def test_auto_time_step_bounds_spawning():
    fq = _fq()
    s, p = _mix()[2]
    h = fq.fciqmc_create(s, p)
    sm = fq.fciqmc_ref_offdiag_sum(h)
    assert sm > 0 and fq.fciqmc_tau(h) == 0.5 / sm


def test_arrival_while_others_run_is_admitted_at_the_next_tick():
    """Continuous batching: a request that arrives while another is on the
    GPU joins the running batch at the next scheduling round, without waiting
    for the running request to finish, and its latency counts from its
    arrival time; a request with a future arrival time is not admitted early."""
    fq = _fq()
    mix = _mix()
    srv = fq.fciqmc_server_create(8 << 30, max_active=8)
    first = fq.fciqmc_server_submit(srv, *mix[0], target_sigma=1e-12, max_iters=2000)
    fq.fciqmc_server_tick(srv, 20)
    assert fq.fciqmc_server_poll(srv, first)["state_name"] == "running"
    now = fq.fciqmc_server_clock(srv)
    second = fq.fciqmc_server_submit(srv, *mix[1], target_sigma=1e-12, max_iters=100, t_arrival=now)
    later = fq.fciqmc_server_submit(srv, *mix[2], target_sigma=1e-12, max_iters=100, t_arrival=now + 3600.0)
    fq.fciqmc_server_tick(srv, 20)
    s1, s2, s3 = (fq.fciqmc_server_poll(srv, i) for i in (first, second, later))
    assert s1["state_name"] == "running" and s2["state_name"] == "running", (s1, s2)
    assert s3["state_name"] == "queued"
    assert s2["t_arrival"] == now and s2["t_start"] >= now
    assert s1["iterations"] == 40 and s2["iterations"] == 20
    for _ in range(10):
        fq.fciqmc_server_tick(srv, 20)
    s2 = fq.fciqmc_server_poll(srv, second)
    assert s2["state_name"] == "max_iters" and s2["iterations"] == 100
    assert s2["t_done"] > s2["t_start"] >= s2["t_arrival"]
    assert fq.fciqmc_server_poll(srv, first)["state_name"] == "running"
    assert fq.fciqmc_server_poll(srv, later)["state_name"] == "queued"
