"""Batched plans: the flattened multi-problem product equals the per-problem products."""
import numpy as np
import pytest

from gpu_util import cuda, host, need_gpu, rel2
from oracle import dense
from paper_2205_04194_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _problems(seed=4, n_problems=6):
    g = np.random.default_rng(seed)
    sizes = [int(v) for v in np.rint(np.exp(g.uniform(np.log(300), np.log(6000), n_problems)))]
    cs = g.uniform(0.01, 0.2, n_problems)
    pts = [W.uniform_points(n, seed, stream=100 + b) for b, n in enumerate(sizes)]
    return pts, cs


def test_batched_product_matches_single_problem_plans():
    import torch
    need_gpu()
    from paper_2205_04194_gb300 import imq
    pts, cs = _problems()
    bp = imq.BatchedPlan([cuda(x) for x in pts], cs, 12, 32, domain=(0.0, 0.0, 1.0))
    info = bp.info()
    assert info["n_problems"] == len(pts)
    offs = bp.offsets
    v = W.random_vector(int(offs[-1]), 9, nrhs=2)
    b32 = host(bp.matvec(cuda(v, torch.float32)))
    b64 = host(bp.matvec(cuda(v)))
    for b, (x, c) in enumerate(zip(pts, cs)):
        sl = slice(offs[b], offs[b + 1])
        sp = imq.Plan(cuda(x), c, 12, 32, domain=(0.0, 0.0, 1.0))
        for r in range(2):
            s32 = host(sp.matvec(cuda(v[r, sl], torch.float32)))
            s64 = host(sp.matvec(cuda(v[r, sl])))
            ref = dense.matvec(x, c, v[r, sl])
            assert rel2(b32[r, sl], s32) < 1e-6     # same tree, same operators: rounding only
            assert rel2(b64[r, sl], s64) < 1e-11
            # the method's own accuracy at p = 12 (these c span 0.01..0.2): a few 1e-6
            assert rel2(b64[r, sl], ref) < 5e-6 and rel2(b32[r, sl], ref) < 5e-6
        sp.close()


def test_batched_default_domain_and_single_problem():
    import torch
    need_gpu()
    from paper_2205_04194_gb300 import imq
    pts, cs = _problems(5, 1)
    bp = imq.BatchedPlan([cuda(pts[0])], cs, 10, 32)
    v = W.random_vector(pts[0].shape[0], 3)
    assert rel2(host(bp.matvec(cuda(v, torch.float32))), dense.matvec(pts[0], cs[0], v)) < 1e-6


def _solve_problems(seed=6, n_problems=5):
    g = np.random.default_rng(seed)
    sizes = [int(v) for v in np.rint(np.exp(g.uniform(np.log(400), np.log(4000), n_problems)))]
    pts = [W.uniform_points(n, seed, stream=200 + b) for b, n in enumerate(sizes)]
    cs = [2.0 * W.mean_nn_spacing(x) for x in pts]    # moderate conditioning, as in the single-plan CG tests
    fs = [W.franke(x) for x in pts]
    return pts, cs, fs


def test_batched_cg_per_problem_residuals_and_zero_rhs():
    need_gpu()
    from paper_2205_04194_gb300 import imq
    from oracle import solve as OS
    pts, cs, fs = _solve_problems()
    fs[2] = np.zeros_like(fs[2])     # converged before the first iteration: coef stays 0
    bp = imq.BatchedPlan([cuda(x) for x in pts], cs, 12, 32, domain=(0.0, 0.0, 1.0))
    f = np.concatenate(fs)
    coef, info = bp.solve(cuda(f), rtol=1e-6, maxit=2000, precond="schwarz", residual="dense")
    assert info["status"] == "IMQ_OK", info
    x = host(coef)
    offs = bp.offsets
    rel = info["problem_rel_residual"][0]
    its = info["problem_iterations"][0]
    assert its[2] == 0 and np.all(x[offs[2]:offs[3]] == 0) and rel[2] == 0
    for b, (xb, c, fb) in enumerate(zip(pts, cs, fs)):
        if b == 2:
            continue
        sl = slice(offs[b], offs[b + 1])
        assert rel[b] <= 1e-6
        assert OS.true_relres(xb, c, x[sl], fb) <= 1e-6
        # the same system alone takes about as many iterations
        sp = imq.Plan(cuda(xb), c, 12, 32, domain=(0.0, 0.0, 1.0))
        _, i1 = sp.solve(cuda(fb), rtol=1e-6, maxit=2000, precond="schwarz", residual="dense")
        assert abs(i1["iterations"] - its[b]) <= max(3, 0.2 * i1["iterations"])
        sp.close()
    assert info["iterations"] == its.max()


def test_batched_cg_refinement_and_dense_modes():
    need_gpu()
    from paper_2205_04194_gb300 import imq
    from oracle import solve as OS
    pts, cs, fs = _solve_problems(7, 3)
    bp = imq.BatchedPlan([cuda(x) for x in pts], cs, 16, 32, domain=(0.0, 0.0, 1.0))
    f = np.stack([np.concatenate(fs), np.concatenate([2.0 * v for v in fs])])
    # the residual of each problem is certified with its own dense FP64 product
    coef, info = bp.solve(cuda(f), rtol=1e-9, maxit=4000, precond="schwarz", refine_steps=6, inner_rtol=1e-5,
                          residual="dense")
    assert info["status"] == "IMQ_OK", info
    assert info["outer_steps"] >= 2
    assert np.all(info["problem_rel_residual"] <= 1e-9)
    x = host(coef)
    offs = bp.offsets
    for b, (xb, c, fb) in enumerate(zip(pts, cs, fs)):
        sl = slice(offs[b], offs[b + 1])
        assert OS.true_relres(xb, c, x[0, sl], fb) <= 1e-9
        assert OS.true_relres(xb, c, x[1, sl], 2.0 * fb) <= 1e-9
    # the dense FP64 inner operator is block diagonal too: every problem with itself
    coef2, info2 = bp.solve(cuda(f[0]), rtol=1e-8, maxit=4000, precond="schwarz", operator="dense_f64",
                            residual="dense")
    assert info2["status"] == "IMQ_OK", info2
    x2 = host(coef2)
    for b, (xb, c, fb) in enumerate(zip(pts, cs, fs)):
        sl = slice(offs[b], offs[b + 1])
        assert OS.true_relres(xb, c, x2[sl], fb) <= 1e-8
