"""Many runs per launch (fciqmc_step_batch): every run's walker list and
statistics are bit-identical to the same run stepped alone, and to the oracle."""
import numpy as np
import pytest

import oracle
import workloads
from tests.test_gpu_parity import DAMP, assert_states_equal, assert_stats_equal, _fq

pytestmark = pytest.mark.gpu

RUNS = [
    (workloads.hubbard_2d(3, 4, 4.0), dict(DAMP, tau=0.005, target_walkers=2000, initiator_threshold=3.0, seed=1000)),
    (workloads.hubbard_2d(4, 4, 2.0), dict(DAMP, tau=0.005, target_walkers=8000, initiator_threshold=3.0, seed=1001,
                                           max_dets=16)),
    (workloads.hubbard_2d(4, 5, 8.0), dict(DAMP, tau=0.005, target_walkers=3000, initiator_threshold=3.0, seed=1002)),
    (workloads.small_abinitio(8, 3, 3, seed=5), dict(DAMP, tau=0.005, target_walkers=3000, initiator_threshold=3.0,
                                                     seed=11, semistoch_size=40, semistoch_start=5)),
    (workloads.hubbard_1d(8, 1.0, 4.0), dict(DAMP, tau=0.01, target_walkers=1000, seed=3)),
]


def test_batch_equals_alone_and_oracle():
    fq = _fq()
    batch = [fq.fciqmc_create(s, p) for s, p in RUNS]
    fq.fciqmc_step_batch(batch, 120)
    fq.fciqmc_step_batch(batch, 80)
    for (s, p), hb in zip(RUNS, batch):
        ha = fq.fciqmc_create(s, p)
        fq.fciqmc_step(ha, 200)
        assert_states_equal(fq.fciqmc_export_state(hb), fq.fciqmc_export_state(ha))
        sb, sa = fq.fciqmc_iter_stats_get(hb), fq.fciqmc_iter_stats_get(ha)
        for k in ["nw", "shift", "ndet", "attempts", "spawns", "rejected", "annihilated", "e_den"]:
            np.testing.assert_array_equal(np.asarray(sb[k]), np.asarray(sa[k]), err_msg=k)
    # and the batch against the oracle for two of the runs
    for idx in (0, 3):
        s, p = RUNS[idx]
        o = oracle.Run(oracle.system_from_workload(s), **p)
        o.step(200)
        assert_states_equal(fq.fciqmc_export_state(batch[idx]), o.export())
        assert_stats_equal(fq.fciqmc_iter_stats_get(batch[idx]), o.stats())


def test_batch_runs_with_different_targets_stop_on_time():
    fq = _fq()
    a = fq.fciqmc_create(*RUNS[0])
    b = fq.fciqmc_create(*RUNS[2])
    fq.fciqmc_step(a, 30)          # a is ahead by 30 iterations
    fq.fciqmc_step_batch([a, b], 50)
    assert fq.fciqmc_export_shift(a)["iteration"] == 80
    assert fq.fciqmc_export_shift(b)["iteration"] == 50
    fq.fciqmc_step(b, 30)          # single stepping still works after a batch
    assert fq.fciqmc_export_shift(b)["iteration"] == 80
    c = fq.fciqmc_create(*RUNS[2])
    fq.fciqmc_step(c, 80)
    assert_states_equal(fq.fciqmc_export_state(b), fq.fciqmc_export_state(c))


def test_autotuned_geometry_changes_no_result():
    fq = _fq()
    runs = RUNS[:3]
    a = [fq.fciqmc_create(s, p) for s, p in runs]
    b = [fq.fciqmc_create(s, p) for s, p in runs]
    fq.fciqmc_step_batch(a, 60)
    tuned = fq.fciqmc_autotune(b, 6)      # advances b by 13 sweeps of 6 iterations
    assert tuned["spawn_blocks_per_sm"] in (0, 1, 2, 4, 8, 16)
    assert tuned["annihilate_blocks_per_sm"] in (0, 3, 9, 24)
    fq.fciqmc_step_batch(a, 0)
    done = fq.fciqmc_export_shift(b[0])["iteration"]
    fq.fciqmc_step_batch(a, done - 60)
    fq.fciqmc_step_batch(a, 20)
    fq.fciqmc_step_batch(b, 20)
    for x, y in zip(a, b):
        assert_states_equal(fq.fciqmc_export_state(x), fq.fciqmc_export_state(y))


def test_all_64_batched_hubbard_runs_equal_alone():
    """The batched set (64 uneven 2D Hubbard runs: 3x4, 4x4, 4x5, U/t 2/4/8,
    targets 1e4 .. 1e6): after 150 iterations in one batch every run's
    walker list, shift and counters equal the same run stepped alone."""
    fq = _fq()
    runs = [(s, dict(p, shift_damping=0.5, shift_interval=5)) for s, p in workloads.batched_hubbard_instances(64)]
    batch = [fq.fciqmc_create(s, p) for s, p in runs]
    fq.fciqmc_step_batch(batch, 150)
    for (s, p), hb in zip(runs, batch):
        ha = fq.fciqmc_create(s, p)
        fq.fciqmc_step(ha, 150)
        assert_states_equal(fq.fciqmc_export_state(hb), fq.fciqmc_export_state(ha))
        sb, sa = fq.fciqmc_iter_stats_get(hb), fq.fciqmc_iter_stats_get(ha)
        for k in ["nw", "shift", "ndet", "attempts", "spawns", "rejected", "annihilated", "e_den"]:
            np.testing.assert_array_equal(np.asarray(sb[k]), np.asarray(sa[k]), err_msg=k)
        del ha
