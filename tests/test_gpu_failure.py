"""Failure detection without a GPU fault: every wait in the library's kernels is
bounded (mbarrier waits give up after a limit, set a device error word and let
the kernel return).  gtb_selftest_wait makes such a wait run out on purpose (an
mbarrier nobody arrives at, a 20 ms limit); the host reads the error through
gtb_device_status, the word is cleared, and the context keeps working."""
import time

import numpy as np
import pytest

from helpers import region, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import torch
    from paper_2311_08322_b300 import build, gtb
    assert torch.cuda.is_available()
    build.build()
    return gtb


def test_expired_wait_is_reported_and_cleared(G, orc):
    G.device_status()  # nothing pending
    t0 = time.perf_counter()
    G.selftest_wait(20_000_000, arrive=False)
    with pytest.raises(G.GtbError) as e:
        G.device_status()
    assert e.value.code == -7
    assert time.perf_counter() - t0 < 5.0  # the wait gave up near its limit, not after the default 2 s
    G.device_status()  # cleared by the read above
    # the context is still usable: a stencil call right after matches the oracle
    rng = np.random.default_rng(0)
    inp, coeff = rng.uniform(-1, 1, (3, 20, 24)), rng.uniform(0, 0.025, (3, 20, 24))
    sin, scf = G.storage_from(inp, (2, 2, 0)), G.storage_from(coeff, (2, 2, 0))
    sout = G.storage_from(np.zeros_like(coeff), (2, 2, 0))
    G.hdiff(sin, scf, sout)
    G.device_status()
    ref = region(orc.hdiff(inp, coeff), (2, 2, 0), (20, 16, 3))
    assert rel_err(region(sout.numpy(), (2, 2, 0), (20, 16, 3)), ref) <= 1e-12


def test_completed_wait_reports_nothing(G):
    G.selftest_wait(20_000_000, arrive=True)
    G.device_status()


def test_selftest_arguments(G):
    for limit, arrive in ((0, 0), (-5, 0), (3_000_000_000, 0), (1000, 2)):
        assert G.lib().gtb_selftest_wait(limit, arrive, None) == -9
