"""The learned sampling proposal against the plain uniform method, paired, on held-out
environments.

Plain PUMP plans 10^4 seeded training environments (4000 uniform samples, N = 128, CP 1 %); the
BF16 network is trained on the certified plans' states with the device loop; then each of 200
held-out environments (seeds 1,000,000 on) is planned with 4000 uniform samples and with the same
first 3000 uniform samples plus 1000 proposals kept clear of the boxes (the fraction and the
clearance were chosen on separate validation environments).  Everything is seeded, so the outcome
is reproducible.  The test asserts what the network gains: at least the uniform method's success
rate, and a median certified-cost ratio (mixed / uniform, on pairs both solve) below 1.  It takes
about two minutes on one GB300."""
import numpy as np
import pytest

from paper_1607_06886_gb300 import inputs, proposal, pump

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    pump.load()
    pump.use_torch_allocator()
    yield


def test_learned_proposal_gains_over_uniform_sampling():
    data = proposal.collect(list(range(10000)))
    assert data.stats["kept"] > 5000
    m = proposal.make_model(0, proposal.PATH_INDEXED)
    tr = proposal.train(m, data, 5000)
    assert tr["loss_last"] < tr["loss_first"]
    held = list(range(proposal.HELDOUT_SEED0, proposal.HELDOUT_SEED0 + 200))
    ev = proposal.evaluate(m, held)
    m.close()
    assert ev["learned"] == proposal.LEARNED and ev["clearance"] == proposal.CLEARANCE
    assert not ev["errors_uniform"] and not ev["errors_mixed"], (ev["errors_uniform"], ev["errors_mixed"])
    assert ev["paired"] >= 100
    assert ev["success_mixed"] >= ev["success_uniform"], ev
    assert ev["median_cost_ratio"] < 1.0, ev
    assert ev["mixed_cheaper"] > ev["mixed_dearer"], ev
