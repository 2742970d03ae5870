"""State in and out of host memory through the C ABI (nrmg_set_state_host /
nrmg_get_state_host): the same state, checks and cycle as the device-pointer calls."""
import numpy as np
import pytest
import torch

from inputs import lid_cavity, random_state
from paper_2206_13164_gb300 import nrmg

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def test_host_state_round_trip_and_cycle():
    torch.cuda.set_device(0)
    prob = lid_cavity(32, 7, 0.1, 0.3, order=2, slope=2, levels=3)
    rng = np.random.default_rng(210)
    P, F = random_state(rng, 32, 32, prob.M, amp=0.05)
    A = nrmg.from_problem(prob, device=DEV)
    B = nrmg.from_problem(prob, device=DEV)
    A.set_state(torch.tensor(P, device=DEV), torch.tensor(F, device=DEV))
    hP = torch.tensor(P).pin_memory()
    hF = torch.tensor(F).pin_memory()
    B.set_state_host(hP, hF)
    oP, oF = torch.empty_like(hP).pin_memory(), torch.empty_like(hF).pin_memory()
    B.get_state_host(oP, oF)
    assert torch.equal(oP, hP) and torch.equal(oF, hF)
    ra, rb = A.fas_cycle(), B.fas_cycle()
    assert ra == rb
    Pa, Fa = A.get_state()
    B.get_state_host(oP, oF)
    assert torch.equal(Pa.cpu(), oP) and torch.equal(Fa.cpu(), oF)
    # plain numpy (pageable) arrays work too
    nP, nF = np.zeros_like(P), np.zeros_like(F)
    B.get_state_host(nP, nF)
    assert np.array_equal(nP, oP.numpy()) and np.array_equal(nF, oF.numpy())


def test_host_state_rejects_a_non_physical_state():
    prob = lid_cavity(16, 4, 0.1, 0.3)
    rng = np.random.default_rng(211)
    P, F = random_state(rng, 16, 16, prob.M)
    F[5, 0] = -1.0  # negative density
    S = nrmg.from_problem(prob, device=DEV)
    with pytest.raises(nrmg.NrmgError) as e:
        S.set_state_host(P, F)
    assert e.value.status == nrmg.ERR_NONPHYSICAL
