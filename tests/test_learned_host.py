"""Host logic of the learned start that needs no GPU: the training draws and the refusal to
run the network without CUDA (there is no CPU fallback)."""
import math

import numpy as np
import pytest
import torch

from paper_2206_13164_gb300 import learned


def test_training_draws_keep_out_of_the_held_out_box():
    rng = np.random.default_rng(2206)
    hold = (0.03, 0.35)
    draws = learned.draw_problems(3000, rng, holdout=hold)
    kn = np.array([d[0] for d in draws])
    u = np.array([d[1] for d in draws])
    assert len(draws) == 3000
    assert kn.min() >= 0.01 and kn.max() <= 1.0 and u.min() >= 0.05 and u.max() <= 0.5
    near = (np.abs(np.log10(kn) - math.log10(hold[0])) < 0.08) & (np.abs(u - hold[1]) < 0.03)
    assert not near.any()
    # log-uniform in Kn: each decade gets about half of the draws
    assert abs(np.mean(kn < 0.1) - 0.5) < 0.05


def test_solver_grids_of_a_learned_solve_are_powers_of_two_above_the_start():
    with pytest.raises(ValueError):
        learned.lid_solver(48, 5, 0.1, 0.2)  # not 8 * 2^k


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the behaviour without a GPU")
def test_network_refuses_to_run_without_cuda():
    with pytest.raises(RuntimeError):
        learned.Net()


def test_committed_weights_describe_their_training():
    import os

    assert os.path.exists(learned.WEIGHTS)
    z = np.load(learned.WEIGHTS)
    import json

    meta = json.loads(str(z["meta"]))
    assert int(z["cin"]) == learned.CIN and int(z["cout"]) == learned.COUT and int(z["hidden"]) == 64
    assert sum(meta["n_pairs"]) == 2000 and meta["sizes"] == [64, 128] and meta["M"] == 8
    assert meta["holdout"] == [0.03, 0.35]
    from oracle import net_ref

    assert z["params"].size == net_ref.n_params(learned.CIN, 64, learned.COUT)
    assert np.all(np.isfinite(z["params"]))


def test_committed_correction_weights_describe_their_training():
    import json
    import os

    assert os.path.exists(learned.CORR_WEIGHTS)
    z = np.load(learned.CORR_WEIGHTS)
    meta = json.loads(str(z["meta"]))
    assert int(z["cin"]) == learned.CORR_CIN and int(z["cout"]) == learned.COUT and int(z["hidden"]) == 64
    assert meta["sizes"] == [64] and meta["M"] == 8 and meta["holdout"] == [0.03, 0.35]
    assert meta["n_pairs"][0] > meta["problems"]  # several cycles of every training cavity
    from oracle import net_ref

    assert z["params"].size == net_ref.n_params(learned.CORR_CIN, 64, learned.COUT)
    assert np.all(np.isfinite(z["params"]))
    # training lowered the loss
    assert meta["loss_history"][-1] < 0.2 * meta["loss_history"][0]


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the behaviour without a GPU")
def test_learned_cycle_refuses_to_run_without_cuda():
    with pytest.raises(RuntimeError):
        learned.lid_solver(16, 5, 0.1, 0.2)
