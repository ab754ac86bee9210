"""Failure detection without a GPU fault: the bounded device-side wait of the tensor-core
contractions gives up on a barrier that nothing completes, the host reads NTF_ERR_TIMEOUT from
the context's status word, and the context keeps working afterwards."""
import time

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ntf():
    from paper_1409_2383_gb300 import build, ntf as binding
    build.build()
    binding.lib()
    return binding


def _context(ntf):
    rng = np.random.default_rng(3)
    X = torch.as_tensor(rng.random((64, 48, 40), dtype=np.float32)).cuda()
    fs = [torch.as_tensor(rng.random((d, 8), dtype=np.float32)).cuda() for d in X.shape]
    ctx = ntf.Context(X, 8, ntf.default_params(contraction=ntf.NTF_CONTRACT_TENSOR))
    return ctx, fs


def test_wait_that_runs_out_is_reported_and_the_context_stays_usable(ntf):
    ctx, fs = _context(ntf)
    with ctx:
        before = [ctx.mttkrp(n, fs).cpu() for n in range(3)]
        t0 = time.perf_counter()
        with pytest.raises(ntf.NTFError) as e:
            ctx.watchdog_check(50.0)
        waited = time.perf_counter() - t0
        assert e.value.status == 7                 # NTF_ERR_TIMEOUT
        assert waited >= 0.05                      # it waited out its limit ...
        assert waited < 1.5                        # ... and no longer than the limit needs
        ctx.sync()                                 # the status was cleared
        after = [ctx.mttkrp(n, fs).cpu() for n in range(3)]
        for a, b in zip(before, after):
            assert torch.equal(a, b)               # the contractions still run, unchanged
        with pytest.raises(ntf.NTFError):
            ctx.watchdog_check(5.0)                # and the check can be repeated


def test_watchdog_limit_out_of_range(ntf):
    ctx, _ = _context(ntf)
    with ctx:
        for bad in (0.0, -1.0, 2500.0):
            with pytest.raises(ntf.NTFError) as e:
                ctx.watchdog_check(bad)
            assert e.value.status == 1
