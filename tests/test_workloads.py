"""The seeded input recipes (workloads/generators.py) on the CPU: the GPU
drawer's stream partition (incremental workload) and cluster partition hold
the same rows, the stream's segments are consecutive views in arrival order,
and every row is unit-norm."""
import numpy as np
import pytest

from workloads import generators as gen

torch = pytest.importorskip("torch")


def test_stream_and_cluster_partitions_hold_the_same_rows():
    sizes = [300, 500, 200, 400]
    n = sum(sizes)
    segs_s, q_s, all_s = gen.deep_like_gpu_segments(n, 16, 11, sizes, 3, device="cpu",
                                                    stream=True, return_all=True, n_comp=40)
    segs_c, q_c = gen.deep_like_gpu_segments(n, 16, 11, sizes, 3, device="cpu", n_comp=40)
    assert [len(s) for s in segs_s] == sizes and [len(s) for s in segs_c] == sizes
    # stream: consecutive views of one tensor, in the order the rows are drawn
    off = 0
    for s in segs_s:
        assert s.data_ptr() == all_s[off:].data_ptr()
        off += len(s)
    # same draw, another partition: the same multiset of rows, the same queries
    a = np.sort(np.ascontiguousarray(torch.cat(segs_s).numpy()).view(f"V{4 * 96}").ravel())
    b = np.sort(np.ascontiguousarray(torch.cat(segs_c).numpy()).view(f"V{4 * 96}").ravel())
    assert (a == b).all()
    assert torch.equal(q_s, q_c)
    norms = torch.cat(segs_s).norm(dim=1)
    assert torch.allclose(norms, torch.ones_like(norms), atol=1e-5)
