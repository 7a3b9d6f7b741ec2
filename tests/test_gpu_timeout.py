"""Failure detection on the GPU without a fault: the tensor-core prune waits on
an mbarrier for its MMAs with a time limit.  A test-only switch withholds the
completion signal (a flag nothing sets), so every wait runs out; the kernel
records the timeout in the device error word, frees its tensor memory and
returns, the call reports RNSM_ETIMEOUT, and the context stays usable."""
import numpy as np
import pytest
import torch

from workloads import generators as gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rn():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_17099_gb300 import build as b
    b.build()
    from paper_2602_17099_gb300 import rnsm
    return rnsm


# L2 at d = 64 with pools of 40: the two-owner pair tile (BF16 and FP8); inner
# product: the general tile (one owner per CTA)
@pytest.mark.parametrize("metric,prec", [(0, 1), (1, 1), (0, 2)])
def test_tile_wait_runs_out_and_the_context_stays_usable(rn, monkeypatch, metric, prec):
    n = 2000
    X = torch.from_numpy(gen.gaussian(n, 64, 5)).cuda()
    if metric == 1:
        X = X / X.norm(dim=1, keepdim=True)
    rng = np.random.default_rng(3)
    owners = torch.from_numpy(rng.choice(n, 300, replace=False).astype(np.int32)).cuda()
    pool = torch.from_numpy(rng.integers(-1, n, size=(300, 40)).astype(np.int32)).cuda()
    want = rn.prune(X, owners, pool, 16, 1.2, metric=metric)
    monkeypatch.setenv("RNSM_TEST_WITHHOLD_COMMIT", "1")
    with pytest.raises(rn.RnsmError) as ei:
        rn.prune(X, owners, pool, 16, 1.2, metric=metric, prec=prec)
    assert ei.value.status == rn.ETIMEOUT
    monkeypatch.delenv("RNSM_TEST_WITHHOLD_COMMIT")
    torch.cuda.synchronize()          # no sticky error: the context still works
    got = rn.prune(X, owners, pool, 16, 1.2, metric=metric, prec=prec)
    assert torch.equal(got, want)
