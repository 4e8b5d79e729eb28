"""GPU products vs the FP64 oracle.

Tolerances (relative 2-norm):
* FP32 paths vs FP64 dense (O1): 1e-6 at the chosen p -- the accuracy target of
  the method; each term is one FP32 rsqrt (<= 2 ulp) and the sums are FP32
  within one leaf / tile, so rounding stays near 1e-7 and the rest of the
  budget is expansion truncation.
* FP32 fast path vs the FP64 FMM reference on the same tree and p (O3b): 1e-6.
* FP64 fast path vs O3b: 1e-11 (same truncation, only rounding differs).
* FP64 dense vs O1: 1e-13.
"""
import numpy as np
import pytest

from gpu_util import cuda, host, need_gpu, rel2
from oracle import dense, fmm
from paper_2205_04194_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _imq():
    need_gpu()
    from paper_2205_04194_gb300 import imq
    return imq


@pytest.mark.parametrize("n", [1, 1025, 3000])
def test_dense_f32_f64(n):
    import torch
    imq = _imq()
    pts = W.uniform_points(n, 7)
    v = W.random_vector(n, 7, nrhs=2)
    c = 0.05
    ref = dense.matvec(pts, c, v)
    b32 = host(imq.dense_matvec(cuda(pts), c, cuda(v, torch.float32)))
    b64 = host(imq.dense_matvec(cuda(pts), c, cuda(v)))
    for r in range(2):
        assert rel2(b32[r], ref[r]) < 1e-6
        assert rel2(b64[r], ref[r]) < 1e-13
    # host buffers go through the same call
    bh = imq.dense_matvec(pts, c, v.astype(np.float32))
    assert isinstance(bh, np.ndarray) and rel2(bh[0], ref[0]) < 1e-6


def _fast_case(pts, c, p, leaf, domain=None, nrhs=1, tol_dense=1e-6):
    import torch
    imq = _imq()
    n = pts.shape[0]
    v = W.random_vector(n, 11, nrhs=nrhs)
    ref = dense.matvec(pts, c, v)
    plan = imq.Plan(cuda(pts), c, p, leaf, domain=domain)
    b32 = host(plan.matvec(cuda(v, torch.float32)))
    b64 = host(plan.matvec(cuda(v)))
    vv = v if nrhs > 1 else v[None]
    b32 = b32 if nrhs > 1 else b32[None]
    b64 = b64 if nrhs > 1 else b64[None]
    rr = ref if nrhs > 1 else ref[None]
    for r in range(nrhs):
        ofmm = fmm.fmm_matvec(pts, c, vv[r], p, leaf, domain)
        assert rel2(b64[r], ofmm) < 1e-11, "FP64 fast path vs FP64 FMM reference"
        assert rel2(b32[r], ofmm) < 1e-6, "FP32 fast path vs FP64 FMM reference"
        assert rel2(b32[r], rr[r]) < tol_dense, "FP32 fast path vs FP64 dense"
    plan.close()


def test_fast_plain_2k():
    wl = W.plain_2k()
    _fast_case(wl.points, wl.c, wl.p, wl.leaf, wl.domain)


def test_fast_host_buffers_replay_the_same_product():
    """Host input / output buffers run the plan's cached graph of the product: pinned and pageable
    buffers, repeated calls and a change of nrhs give the bits of the device-buffer product."""
    import torch
    imq = _imq()
    pts = W.clustered_points(1500, 8, 6000, 0.03, 4)
    plan = imq.Plan(cuda(pts), 0.01, 12, 64, domain=(0.0, 0.0, 1.0))
    n = pts.shape[0]
    v2 = np.random.default_rng(7).uniform(-1, 1, (2, n)).astype(np.float32)
    ref1 = host(plan.matvec(cuda(v2[0])))
    ref2 = host(plan.matvec(cuda(v2)))
    for _ in range(2):
        pinned = torch.from_numpy(v2[0].copy()).pin_memory()
        out = torch.empty(n, dtype=torch.float32).pin_memory()
        plan.matvec(pinned, out)
        assert np.array_equal(out.numpy(), ref1)
        out2 = np.empty((2, n), dtype=np.float32)
        plan.matvec(v2, out2)                      # pageable numpy buffers, nrhs = 2
        assert np.array_equal(out2, ref2)
    assert rel2(ref1, dense.matvec(pts, 0.01, v2[0].astype(np.float64))) <= 1e-6
    plan.close()


def test_fast_clustered_small_c():
    pts = W.clustered_points(1500, 8, 6000, 0.03, 3)
    _fast_case(pts, 0.01, 12, 64, nrhs=2)


def test_fast_uniform_ragged_leaf():
    pts = W.uniform_points(4321, 8)
    _fast_case(pts, 0.02, 12, 17, (0.0, 0.0, 1.0))


def test_fast_large_leaves_stage_sources_in_chunks():
    # leaf 200: U-list sources exceed one shared-memory stage (1024 records) and
    # leaves hold several 32-target chunks
    pts = W.uniform_points(12000, 12)
    _fast_case(pts, 0.02, 10, 200, (0.0, 0.0, 1.0))


def test_fast_degenerate_single_leaf_and_single_point():
    imq = _imq()
    pts = W.uniform_points(90, 9)
    v = W.random_vector(90, 9)
    ref = dense.matvec(pts, 0.2, v)
    plan = imq.Plan(cuda(pts), 0.2, 4, 1000)     # one leaf: pure P2P
    assert rel2(host(plan.matvec(cuda(v))), ref) < 1e-13
    one = imq.Plan(cuda(np.array([[0.4, 0.1]])), 0.5, 4, 8)
    assert host(one.matvec(cuda(np.array([3.0]))))[0] == pytest.approx(6.0, rel=1e-14)


def test_fast_full_size_clustered_1m_sampled_rows():
    import torch
    imq = _imq()
    wl = W.clustered_1m(p=12)
    plan = imq.Plan(cuda(wl.points), wl.c, wl.p, wl.leaf, domain=wl.domain)
    b = host(plan.matvec(cuda(wl.v, torch.float32)))
    rows = np.random.default_rng(0).choice(wl.n, 2048, replace=False)
    ref = dense.matvec_rows(wl.points, wl.c, wl.v, rows)
    assert rel2(b[rows], ref) < 1e-6


@pytest.mark.parametrize("p,leaf", [(8, 32), (12, 64), (16, 40), (18, 64)])
def test_tensor_core_m2l_matches_cuda_core_m2l_and_oracle(p, leaf):
    """The tcgen05 M2L (fp16 hi/lo split, power-of-two scaled rows) against the register-tiled FP32
    M2L and the FP64 FMM reference on the same tree.  p = 16 (K = 153) and p = 18 (K = 190) use
    five and six accumulator column groups; at p = 18 the row scale fills the last two padding
    halfs of the packed row (K = 190 of KP = 192)."""
    import torch
    imq = _imq()
    pts = W.clustered_points(2000, 6, 4000, 0.04, 5)
    c = 0.005
    v = W.random_vector(pts.shape[0], 13, nrhs=2)
    tc = imq.Plan(cuda(pts), c, p, leaf, domain=(0.0, 0.0, 1.0), m2l_kernel="tensor")
    # the register-tiled CUDA-core M2L stages the whole operator in shared memory: up to p = 16
    cc = imq.Plan(cuda(pts), c, p, leaf, domain=(0.0, 0.0, 1.0), m2l_kernel="cuda_cores") if p <= 16 else None
    assert tc.info()["m2l_pairs"] > 1000
    bt = host(tc.matvec(cuda(v, torch.float32)))
    bc = host(cc.matvec(cuda(v, torch.float32))) if cc else None
    for r in range(2):
        ofmm = fmm.fmm_matvec(pts, c, v[r], p, leaf, (0.0, 0.0, 1.0))
        if cc:
            assert rel2(bt[r], bc[r]) < 5e-7
        assert rel2(bt[r], ofmm) < 1e-6
    tc.close()
    if cc:
        cc.close()


def test_tensor_core_m2l_batched_matches_cuda_cores():
    import torch
    imq = _imq()
    pts = [W.uniform_points(n, 21, stream=s) for s, n in enumerate((700, 5000, 2300))]
    cs = [0.02, 0.15, 0.05]
    a = imq.BatchedPlan([cuda(x) for x in pts], cs, 12, 32, domain=(0.0, 0.0, 1.0), m2l_kernel="tensor")
    b = imq.BatchedPlan([cuda(x) for x in pts], cs, 12, 32, domain=(0.0, 0.0, 1.0), m2l_kernel="cuda_cores")
    v = W.random_vector(a.n, 5)
    ref = host(a.matvec(cuda(v)))      # FP64 product, same tree and truncation: the rounding reference
    et = rel2(host(a.matvec(cuda(v, torch.float32))), ref)
    ec = rel2(host(b.matvec(cuda(v, torch.float32))), ref)
    # c = 0.15 on 5000 points cancels strongly in M2L: both FP32 paths sit near 1e-6 here
    assert et < 2e-6 and et < 1.5 * ec + 2e-7, (et, ec)


@pytest.mark.parametrize("p", [1, 3, 6, 9, 14])
def test_fixed_order_far_field_every_p(p):
    """The far-field kernel is compiled per order p; odd and even p against the FP64
    FMM reference on an adaptive tree (W lists present)."""
    import torch
    imq = _imq()
    pts = W.clustered_points(800, 4, 1500, 0.03, 8)
    c = 0.01
    v = W.random_vector(pts.shape[0], 17)
    plan = imq.Plan(cuda(pts), c, p, 24, domain=(0.0, 0.0, 1.0))
    assert plan.info()["n_w"] > 0
    b32 = host(plan.matvec(cuda(v, torch.float32)))
    ofmm = fmm.fmm_matvec(pts, c, v, p, 24, (0.0, 0.0, 1.0))
    assert rel2(b32, ofmm) < 1e-6
    plan.close()


def test_fast_full_size_uniform_100k_sampled_rows():
    """The 100k configuration at its own p and leaf (12, 64), c = 2 x mean NN spacing."""
    import torch
    imq = _imq()
    wl = W.uniform_100k()
    v = W.random_vector(wl.n, 2)
    plan = imq.Plan(cuda(wl.points), wl.c, wl.p, wl.leaf, domain=wl.domain)
    b = host(plan.matvec(cuda(v, torch.float32)))
    rows = np.random.default_rng(1).choice(wl.n, 2048, replace=False)
    ref = dense.matvec_rows(wl.points, wl.c, v, rows)
    assert rel2(b[rows], ref) < 1e-6
    plan.close()


def test_batched_256_full_size_sampled_rows():
    """All 256 problems (3.7M points) in one batched plan at p = 14, leaf 128, 4 right-hand
    sides; 64 sampled rows of 16 problems against the FP64 oracle, 1e-6 for every
    right-hand side.  The trig sums cancel in the far field (c up to 0.2, several sign
    changes over the square), so the FP32 rounding of the translated coefficients is above
    1e-6 there: the plan translates in FP64 (P2M, P2P, M2P and L2P stay FP32).  With FP32
    translations the Franke data (no cancellation) still meet 1e-6."""
    import torch
    imq = _imq()
    probs = W.batched_256()
    pts = [cuda(x) for x, _, _ in probs]
    cs = [c for _, c, _ in probs]
    f = np.concatenate([r for _, _, r in probs], axis=1)
    d_f = cuda(f, torch.float32)
    bp = imq.BatchedPlan(pts, cs, 14, 128, domain=(0.0, 0.0, 1.0), translations="fp64")
    b = host(bp.matvec(d_f))
    bp.close()
    b32 = imq.BatchedPlan(pts, cs, 14, 128, domain=(0.0, 0.0, 1.0))
    bf = host(b32.matvec(d_f))
    offs = b32.offsets
    b32.close()
    g = np.random.default_rng(3)
    for q in np.linspace(0, len(probs) - 1, 16).astype(int):
        x, c, rhs = probs[q]
        rows = g.choice(x.shape[0], min(64, x.shape[0]), replace=False)
        for r in range(4):
            ref = dense.matvec_rows(x, c, rhs[r], rows)
            got = b[r, offs[q]:offs[q + 1]][rows]
            assert rel2(got, ref) <= 1e-6, (q, r, rel2(got, ref))
        ref = dense.matvec_rows(x, c, rhs[0], rows)
        assert rel2(bf[0, offs[q]:offs[q + 1]][rows], ref) <= 1e-6, q


def test_fp64_translations_remove_the_fp32_cancellation_floor():
    """One of the batched workload's largest problems (N = 46,994, c = 0.18) with a trig-sum
    vector: the FP32 product stays above 1e-6, the same plan with FP64 translations meets it,
    and both agree with the all-FP64 product to their own error.  Mixed translations (FP64 M2M
    and L2L around the tensor-core M2L) land between the two: most of the FP32 floor comes from
    the M2L's FP32 sums."""
    import torch
    imq = _imq()
    x, c, rhs = W.batched_256()[14]
    rows = np.random.default_rng(5).choice(x.shape[0], 512, replace=False)
    v = rhs[3]
    ref = dense.matvec_rows(x, c, v, rows)
    p32 = imq.Plan(cuda(x), c, 14, 128, domain=(0.0, 0.0, 1.0))
    p64t = imq.Plan(cuda(x), c, 14, 128, domain=(0.0, 0.0, 1.0), translations="fp64")
    e32 = rel2(host(p32.matvec(cuda(v, torch.float32)))[rows], ref)
    e64t = rel2(host(p64t.matvec(cuda(v, torch.float32)))[rows], ref)
    e64 = rel2(host(p32.matvec(cuda(v)))[rows], ref)
    pmx = imq.Plan(cuda(x), c, 14, 128, domain=(0.0, 0.0, 1.0), translations="mixed")
    emx = rel2(host(pmx.matvec(cuda(v, torch.float32)))[rows], ref)
    assert e64 < 1e-7
    assert e64t <= 1e-6 < e32, (e64t, e32)
    assert e64t < 0.5 * e32
    assert e64t < emx < e32, (e64t, emx, e32)
    p32.close()
    p64t.close()
    pmx.close()
