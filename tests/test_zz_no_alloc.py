"""The allocation-free dense product (collected last on purpose).

imq_dense_matvec_noalloc serves callers that may not allocate device memory:
code under a memory manager that owns the whole device, or latency-critical
loops that cannot afford an allocation.  It keeps its scratch in one fixed
device array inside the library, so two calls in a row must both agree with
the FP64 oracle's dense product and with imq_dense_matvec (the second call
reuses the array the first one left behind), imq_sync_check must then report
no failed wait, and sizes beyond the fixed capacity must be refused.
"""
import numpy as np
import pytest

from gpu_util import cuda, host, need_gpu, rel2
from oracle import dense
from paper_2205_04194_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_noalloc_matches_oracle_and_dense_on_two_calls_in_a_row():
    import torch
    need_gpu()
    from paper_2205_04194_gb300 import imq
    c = 0.05
    for seed, n in ((1, 3000), (2, 1777)):   # the second call is smaller than the first
        pts = W.uniform_points(n, seed)
        v = W.random_vector(n, seed)
        d_pts = cuda(pts)
        d_v = cuda(v, torch.float32)
        ref = dense.matvec(pts, c, v.astype(np.float32).astype(np.float64))
        lib_ref = host(imq.dense_matvec(d_pts, c, d_v))
        out = torch.full_like(d_v, float("nan"))
        imq.dense_matvec_noalloc(d_pts, c, d_v, out)
        imq.sync_check()             # no bounded wait ran out (reads the scratch array's error word)
        got = host(out)
        assert np.all(np.isfinite(got))
        assert rel2(got, ref) < 1e-6
        assert rel2(got, lib_ref) < 1e-6


def test_noalloc_rejects_sizes_beyond_capacity_and_host_memory():
    import torch
    need_gpu()
    from paper_2205_04194_gb300 import imq
    n = 262144 + 1
    d_pts = torch.zeros((n, 2), dtype=torch.float64, device="cuda")
    d_v = torch.zeros(n, dtype=torch.float32, device="cuda")
    with pytest.raises(imq.ImqError) as e:
        imq.dense_matvec_noalloc(d_pts, 0.1, d_v, torch.empty_like(d_v))
    assert e.value.status == 1 and "capacity" in str(e.value)
    pts = W.uniform_points(10, 3)
    with pytest.raises(imq.ImqError):
        imq.dense_matvec_noalloc(torch.from_numpy(pts), 0.1, torch.zeros(10), torch.zeros(10))
