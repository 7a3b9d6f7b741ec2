"""rnsm_prune_noalloc: the prune entry point for callers that cannot let the
library allocate device memory (their HBM is all handed to their own pool
allocator, or their path cannot afford cudaMalloc/cudaFree).  Its scratch is
a static device array of the library; the caller passes inputs and outputs.

Checked through the C ABI against rnsm_prune on two calls in a row (the
static scratch keeps the previous call's contents, so the second call shows
that each call resets what must start at zero).  This file is collected last
on purpose; it also passes on its own in a fresh process."""
import ctypes as C

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


def _case(seed, n, d, nv, w):
    X = gen.sift_like(n, seed, d=d)
    rng = np.random.default_rng(seed)
    owners = rng.choice(n, nv, replace=False).astype(np.int32)
    pool = rng.integers(-1, n, size=(nv, w)).astype(np.int32)
    pool[:, 0] = owners                      # the owner must be dropped
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return t(X), t(owners), t(pool)


def _noalloc(rn, X, owners, pool, R, alpha, keep_all=False):
    """Direct C-ABI call; the output buffer belongs to the caller."""
    out = torch.full((owners.shape[0], R), -7, dtype=torch.int32, device=X.device)
    st = rn.lib().rnsm_prune_noalloc(C.c_void_p(X.data_ptr()), X.shape[0], X.shape[1],
                                     C.c_void_p(owners.data_ptr()), owners.shape[0],
                                     C.c_void_p(pool.data_ptr()), pool.shape[1], R, alpha, 0,
                                     int(keep_all), C.c_void_p(out.data_ptr()),
                                     C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == rn.OK, rn.lib().rnsm_last_error()
    return out


def test_noalloc_prune_matches_prune_on_consecutive_calls(rn):
    # first call: a larger batch with wide pools (general kernel); second call:
    # a smaller batch with narrow pools (small-pool kernel) on other data
    X1, o1, p1 = _case(5, 6000, 128, 4000, 96)
    X2, o2, p2 = _case(6, 3000, 32, 1500, 40)
    got1 = _noalloc(rn, X1, o1, p1, 32, 1.2)
    got2 = _noalloc(rn, X2, o2, p2, 16, 1.2, keep_all=True)
    want1 = rn.prune(X1, o1, p1, 32, 1.2)
    want2 = rn.prune(X2, o2, p2, 16, 1.2, keep_all_if_fit=True)
    assert torch.equal(got1, want1)
    assert torch.equal(got2, want2)
    # and again on the first input, after the second call used the scratch
    assert torch.equal(_noalloc(rn, X1, o1, p1, 32, 1.2), want1)


def test_noalloc_prune_rejects_batches_over_its_limit(rn):
    X, o, p = _case(7, 1000, 32, 10, 8)
    big = torch.zeros(rn.NOALLOC_MAX_OWNERS + 1, dtype=torch.int32, device="cuda")
    pool = torch.zeros((big.shape[0], 1), dtype=torch.int32, device="cuda")
    out = torch.empty((big.shape[0], 4), dtype=torch.int32, device="cuda")
    st = rn.lib().rnsm_prune_noalloc(C.c_void_p(X.data_ptr()), X.shape[0], X.shape[1],
                                     C.c_void_p(big.data_ptr()), big.shape[0],
                                     C.c_void_p(pool.data_ptr()), 1, 4, 1.2, 0, 0,
                                     C.c_void_p(out.data_ptr()), None)
    assert st == rn.EINVAL
    assert b"static scratch limit" in rn.lib().rnsm_last_error()


def test_noalloc_prune_leaves_device_memory_unchanged(rn):
    # The point of this entry point: no device allocation inside the call.
    # Warm-up calls load the kernels first (lazy module loading may map code
    # memory); then the library workspace is released and the free device
    # memory is read around calls that reach the general kernel (pools of
    # 96) and the small-pool kernel (pools of 40).
    X1, o1, p1 = _case(8, 6000, 128, 4000, 96)
    X2, o2, p2 = _case(9, 3000, 32, 1500, 40)
    out1 = torch.empty((o1.shape[0], 32), dtype=torch.int32, device="cuda")
    out2 = torch.empty((o2.shape[0], 16), dtype=torch.int32, device="cuda")
    for _ in range(2):
        rn.prune_noalloc(X1, o1, p1, 32, 1.2, out=out1)
        rn.prune_noalloc(X2, o2, p2, 16, 1.2, out=out2)
    rn.release_workspace()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    rn.prune_noalloc(X1, o1, p1, 32, 1.2, out=out1)
    rn.prune_noalloc(X2, o2, p2, 16, 1.2, out=out2)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.equal(out1, rn.prune(X1, o1, p1, 32, 1.2))


def test_noalloc_prune_rejects_a_wrong_output_buffer(rn):
    X, o, p = _case(10, 1000, 32, 10, 8)
    with pytest.raises(ValueError):
        rn.prune_noalloc(X, o, p, 16, 1.2, out=torch.empty((10, 15), dtype=torch.int32,
                                                            device="cuda"))
    with pytest.raises(ValueError):
        rn.prune_noalloc(X, o, p, 16, 1.2, out=torch.empty((10, 16), dtype=torch.int32))
