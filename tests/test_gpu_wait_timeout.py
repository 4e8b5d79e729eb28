"""Failure detection without a GPU fault: a bounded kernel wait that runs out is
reported as IMQ_TIMEOUT, and the context stays usable afterwards."""
import time

import numpy as np
import pytest

from gpu_util import cuda, host, need_gpu, rel2
from oracle import dense
from paper_2205_04194_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_wait_that_never_completes_reports_timeout_and_context_survives():
    import torch
    need_gpu()
    from paper_2205_04194_gb300 import _lib, imq
    L = _lib.load()
    t0 = time.perf_counter()
    st = L.imq_selftest_wait_timeout(None)
    dt = time.perf_counter() - t0
    assert _lib.status_name(st) == "IMQ_TIMEOUT", L.imq_last_error()
    assert dt < 10.0
    imq.sync_check()                       # the word was cleared by the failing call
    pts = W.uniform_points(3000, 41)
    v = W.random_vector(3000, 41)
    plan = imq.Plan(cuda(pts), 0.05, 10, 32)
    b = host(plan.matvec(cuda(v, torch.float32)))
    imq.sync_check()
    assert rel2(b, dense.matvec(pts, 0.05, v)) < 1e-6
    plan.close()
