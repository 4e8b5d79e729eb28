"""A plan's own device buffers can come from the caller's allocator (imq_options.alloc /
free): here torch's caching allocator, through the Python binding's allocator="torch"."""
import numpy as np
import pytest

from gpu_util import cuda, host, need_gpu
from paper_2205_04194_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_plan_buffers_from_the_callers_allocator():
    import torch
    need_gpu()
    from paper_2205_04194_gb300 import imq
    pts = W.uniform_points(20000, 51)
    c = 2.0 * W.mean_nn_spacing(pts)
    d_pts, d_v, d_f = cuda(pts), cuda(W.random_vector(20000, 51), torch.float32), cuda(W.franke(pts))
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    pa = imq.Plan(d_pts, c, 12, 32, allocator="torch")
    torch.cuda.synchronize()
    held = torch.cuda.memory_allocated() - base
    assert held > 1 << 20                                   # the tree, lists and operators
    p0 = imq.Plan(d_pts, c, 12, 32)                         # cudaMalloc: not torch's
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() - base == held
    a = host(pa.matvec(d_v))
    b = host(p0.matvec(d_v))
    assert np.array_equal(a, b)                             # same plan, other memory
    coef, info = pa.solve(d_f, rtol=1e-6, maxit=500)        # solver work arrays through torch too
    assert info["status"] == "IMQ_OK", info
    del coef
    pa.close()
    p0.close()
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == base            # every block handed back
