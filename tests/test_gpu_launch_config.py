"""Every launch configuration gives the same runs: the staged and plain-load
spawning and annihilation kernels, and split spawning (attempts queued in
global memory by class and evaluated by a flat kernel), against the oracle and
against each other, including capacity growth of the attempt queues, heavy
determinants, a semi-stochastic space, batches and the adaptive shift."""
import pytest

import oracle
import workloads
from tests.test_gpu_parity import DAMP, _fq, assert_states_equal, assert_stats_equal

pytestmark = pytest.mark.gpu

CONFIGS = [(0, 2, 0), (1, 2, 9), (4, 2, 3), (0, 2, 24)]


@pytest.fixture
def config():
    fq = _fq()
    saved = fq.fciqmc_get_launch_config()
    yield fq
    fq.fciqmc_set_launch_config(saved["spawn"], saved["heavy"], saved["annihilate"])


CASES = {
    "hubbard_4x4_initiator": (workloads.hubbard_2d(4, 4, 4.0),
                              dict(tau=0.005, target_walkers=5000, initiator_threshold=3.0, seed=7), 200),
    "abinitio_8_3_3_semistoch": (workloads.small_abinitio(8, 3, 3, seed=5),
                                 dict(tau=0.005, target_walkers=3000, initiator_threshold=3.0, seed=11,
                                      semistoch_size=60, semistoch_start=5), 200),
    "abinitio_8_heavy": (workloads.small_abinitio(8, 3, 3, seed=21),
                         dict(tau=0.002, target_walkers=1e9, initial_walkers=3e5, initiator_threshold=3.0, seed=4),
                         6),
    "abinitio_7_adaptive": (workloads.small_abinitio(7, 2, 2, seed=13),
                            dict(tau=0.004, target_walkers=1500, initiator_threshold=3.0, seed=8, adaptive_shift=1),
                            150),
}


@pytest.mark.parametrize("cfg", CONFIGS)
@pytest.mark.parametrize("name", sorted(CASES))
def test_launch_configuration_matches_oracle(config, cfg, name):
    fq = config
    fq.fciqmc_set_launch_config(*cfg)
    sysd, params, n = CASES[name]
    params = dict(DAMP, **params)
    g = fq.fciqmc_create(sysd, params)
    o = oracle.Run(oracle.system_from_workload(sysd), **params)
    for _ in range(2):
        fq.fciqmc_step(g, n // 2)
        o.step(n // 2)
    assert_states_equal(fq.fciqmc_export_state(g), o.export())
    assert_stats_equal(fq.fciqmc_iter_stats_get(g), o.stats())


def test_split_spawning_queue_growth_and_batch(config):
    """Split spawning from one bucket and the smallest queues: the walker list
    and the attempt queues grow several times (each overflowing iteration
    repeated bit-identically), alone and in a batch."""
    fq = config
    fq.fciqmc_set_launch_config(1, 2, 0)
    sysd = workloads.hubbard_2d(4, 4, 2.0)
    params = dict(DAMP, tau=0.005, target_walkers=6e4, initiator_threshold=3.0, seed=17, max_dets=16)
    g = fq.fciqmc_create(sysd, params)
    fq.fciqmc_step(g, 250)
    o = oracle.Run(oracle.system_from_workload(sysd), **{k: v for k, v in params.items() if k != "max_dets"})
    o.step(250)
    assert_states_equal(fq.fciqmc_export_state(g), o.export())
    assert_stats_equal(fq.fciqmc_iter_stats_get(g), o.stats())
    runs = [(workloads.hubbard_2d(3, 4, 4.0), dict(DAMP, tau=0.005, target_walkers=2000, initiator_threshold=3.0,
                                                   seed=1000)),
            (sysd, params)]
    batch = [fq.fciqmc_create(s, p) for s, p in runs]
    fq.fciqmc_step_batch(batch, 250)
    assert_states_equal(fq.fciqmc_export_state(batch[1]), o.export())
    fq.fciqmc_set_launch_config(0, 2, 0)  # and back: the next step recaptures the graph
    fq.fciqmc_step(g, 20)
    o.step(20)
    assert_states_equal(fq.fciqmc_export_state(g), o.export())


@pytest.mark.gpu
def test_device_memory_interface_is_reported():
    """fciqmc_device_memory: the peak memory clock (kHz) and bus width (bits)
    the nominal HBM bandwidth of the bench line is computed from."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2006_14956_gb300 as fq
    clk, bus = fq.fciqmc_device_memory(0)
    assert clk > 0 and bus > 0 and bus % 64 == 0
    assert 1e2 < 2.0 * clk * 1e3 * bus / 8 / 1e9 < 1e5  # GB/s
