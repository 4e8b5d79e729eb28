// C ABI entry points (include/imq.h): argument checks, host/device pointer
// handling, and translation of internal errors into imq_status codes.
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <string>

#include "imq_internal.h"
#include "util.cuh"

struct imq_plan_s {
    imq::Plan P;
};

namespace imq {
namespace {

thread_local std::string g_last_error;

template <class F>
imq_status guard(F &&f) {
    try {
        f();
        g_last_error.clear();
        return IMQ_OK;
    } catch (const Error &e) {
        g_last_error = e.msg;
        return e.status;
    } catch (const std::bad_alloc &) {
        g_last_error = "host allocation failed";
        return IMQ_OOM;
    } catch (...) {
        g_last_error = "unexpected internal error";
        return IMQ_CUDA_ERROR;
    }
}

bool is_device_ptr(const void *p) {
    cudaPointerAttributes a;
    const cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Device view of a caller buffer: in place for device memory, a stream-ordered
// copy for host memory.
struct DevIn {
    const void *ptr = nullptr;
    AsyncMem *tmp = nullptr;
    DevIn(const void *p, size_t bytes, cudaStream_t s) {
        if (is_device_ptr(p)) {
            ptr = p;
        } else {
            tmp = new AsyncMem(bytes, s);
            IMQ_CUDA(cudaMemcpyAsync(tmp->ptr, p, bytes, cudaMemcpyHostToDevice, s));
            ptr = tmp->ptr;
        }
    }
    DevIn(const DevIn &) = delete;
    ~DevIn() { delete tmp; }
};

struct DevOut {
    void *user = nullptr;
    void *ptr = nullptr;
    size_t bytes = 0;
    cudaStream_t stream = nullptr;
    AsyncMem *tmp = nullptr;
    DevOut(void *p, size_t b, cudaStream_t s) : user(p), bytes(b), stream(s) {
        if (is_device_ptr(p)) {
            ptr = p;
        } else {
            tmp = new AsyncMem(b, s);
            ptr = tmp->ptr;
        }
    }
    DevOut(const DevOut &) = delete;
    void finish() {   // copy a host-destined result back and wait for it
        if (tmp) {
            IMQ_CUDA(cudaMemcpyAsync(user, ptr, bytes, cudaMemcpyDeviceToHost, stream));
            IMQ_CUDA(cudaStreamSynchronize(stream));
        }
    }
    ~DevOut() { delete tmp; }
};

std::mutex g_dev_mu;
int g_dev_ok[64] = {0};   // 0 unknown, 1 ok, -1 unsupported

}  // namespace

void set_last_error(const std::string &msg) { g_last_error = msg; }

void check_device() {
    int dev = 0;
    IMQ_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_dev_mu);
    if (dev >= 0 && dev < 64 && g_dev_ok[dev] == 1) return;
    cudaDeviceProp prop;
    IMQ_CUDA(cudaGetDeviceProperties(&prop, dev));
    if (!(prop.major == 10 && prop.minor == 3)) {
        if (dev >= 0 && dev < 64) g_dev_ok[dev] = -1;
        fail(IMQ_UNSUPPORTED, std::string("this library is built for sm_103a; device is ") + prop.name +
                                  " (sm_" + std::to_string(prop.major) + std::to_string(prop.minor) + ")");
    }
    if (dev >= 0 && dev < 64) g_dev_ok[dev] = 1;
}

}  // namespace imq

using namespace imq;

extern "C" {

const char *imq_status_string(imq_status s) {
    switch (s) {
        case IMQ_OK: return "IMQ_OK";
        case IMQ_INVALID_ARG: return "IMQ_INVALID_ARG";
        case IMQ_DUPLICATE_POINTS: return "IMQ_DUPLICATE_POINTS";
        case IMQ_CUDA_ERROR: return "IMQ_CUDA_ERROR";
        case IMQ_OOM: return "IMQ_OOM";
        case IMQ_NOT_CONVERGED: return "IMQ_NOT_CONVERGED";
        case IMQ_NUMERICAL: return "IMQ_NUMERICAL";
        case IMQ_UNSUPPORTED: return "IMQ_UNSUPPORTED";
        case IMQ_TIMEOUT: return "IMQ_TIMEOUT";
    }
    return "IMQ_UNKNOWN";
}

const char *imq_last_error(void) { return g_last_error.c_str(); }

const char *imq_version(void) { return "imq-gb300 0.1 (sm_103a)"; }

}  // extern "C"

namespace {

Allocator plan_allocator(const imq_options *opt) {
    Allocator a;
    if (opt && opt->struct_size >= (int)(offsetof(imq_options, alloc_ctx) + sizeof(void *))) {
        if ((opt->alloc == nullptr) != (opt->free == nullptr))
            fail(IMQ_INVALID_ARG, "imq_plan: imq_options.alloc and free must be given together");
        a.alloc = opt->alloc;
        a.free = opt->free;
        a.ctx = opt->alloc_ctx;
    }
    return a;
}

void parse_plan_args(int64_t N, double c, int p, int leaf, const imq_options *opt, double &x0, double &y0,
                     double &side, bool &dups, int *m2l_kernel = nullptr, int *algorithm = nullptr,
                     int *tc_depth = nullptr, int *trans_mode = nullptr) {
    if (N < 1 || N > 0x7FFFFFFF) fail(IMQ_INVALID_ARG, "imq_plan: N must be in [1, 2^31-1]");
    if (!std::isfinite(c) || c <= 0) fail(IMQ_INVALID_ARG, "imq_plan: c must be finite and > 0");
    if (p < 1 || p > IMQ_MAX_P) fail(IMQ_UNSUPPORTED, "imq_plan: p must be in [1, IMQ_MAX_P]");
    if (leaf < 1 && !(opt && opt->algorithm == IMQ_ALG_TREECODE))   // the treecode ignores leaf
        fail(IMQ_INVALID_ARG, "imq_plan: leaf must be >= 1");
    dups = false;
    x0 = 0;
    y0 = 0;
    side = -1;
    if (opt) {
        if (opt->struct_size < (int)offsetof(imq_options, translations))
            fail(IMQ_INVALID_ARG, "imq_plan: imq_options.struct_size too small");
        if (opt->has_domain) {
            if (!std::isfinite(opt->x0) || !std::isfinite(opt->y0) || !std::isfinite(opt->side) || opt->side <= 0)
                fail(IMQ_INVALID_ARG, "imq_plan: domain must be finite with side > 0");
            x0 = opt->x0;
            y0 = opt->y0;
            side = opt->side;
        }
        dups = opt->check_duplicates != 0;
        if (opt->m2l_kernel < IMQ_M2L_AUTO || opt->m2l_kernel > IMQ_M2L_TENSOR)
            fail(IMQ_INVALID_ARG, "imq_plan: unknown m2l_kernel");
        if (m2l_kernel) *m2l_kernel = opt->m2l_kernel;
        if (opt->algorithm != IMQ_ALG_FMM && opt->algorithm != IMQ_ALG_TREECODE)
            fail(IMQ_INVALID_ARG, "imq_plan: unknown algorithm");
        if (opt->algorithm == IMQ_ALG_TREECODE && (opt->levels < 1 || opt->levels > IMQ_MAX_LEVEL - 1))
            fail(IMQ_INVALID_ARG, "imq_plan: the treecode needs levels in [1, IMQ_MAX_LEVEL - 1]");
        if (algorithm) *algorithm = opt->algorithm;
        if (tc_depth) *tc_depth = opt->algorithm == IMQ_ALG_TREECODE ? opt->levels + 1 : 0;
        if (opt->struct_size >= (int)(offsetof(imq_options, translations) + sizeof(int32_t))) {
            if (opt->translations != IMQ_TRANS_FP32 && opt->translations != IMQ_TRANS_FP64 &&
                opt->translations != IMQ_TRANS_MIXED)
                fail(IMQ_INVALID_ARG, "imq_plan: unknown translations precision");
            if (opt->translations != IMQ_TRANS_FP32 && (p > 16 || opt->algorithm != IMQ_ALG_FMM))
                fail(IMQ_UNSUPPORTED, "imq_plan: FP64 or mixed translations need the fast multipole form and p <= 16");
            if (trans_mode) *trans_mode = opt->translations;
        }
        if (opt->struct_size >= (int)(offsetof(imq_options, m2l_split) + sizeof(int32_t))) {
            if (opt->p2p_warps != 0 && opt->p2p_warps != 2 && opt->p2p_warps != 4 && opt->p2p_warps != 8)
                fail(IMQ_INVALID_ARG, "imq_plan: p2p_warps must be 0, 2, 4 or 8");
            if (opt->p2p_chunk != 0 && opt->p2p_chunk != 8 && opt->p2p_chunk != 16 && opt->p2p_chunk != 32)
                fail(IMQ_INVALID_ARG, "imq_plan: p2p_chunk must be 0, 8, 16 or 32");
            if (opt->m2l_stages != 0 && (opt->m2l_stages < 2 || opt->m2l_stages > 6))
                fail(IMQ_INVALID_ARG, "imq_plan: m2l_stages must be 0 or 2..6");
            if (opt->m2l_split < 0 || opt->m2l_split > 4) fail(IMQ_INVALID_ARG, "imq_plan: m2l_split must be 0..4");
        }
    }
}

// tile shapes of the FP32 product from the options (0: default)
void plan_tiles(Plan &P, const imq_options *opt) {
    if (opt && opt->struct_size >= (int)(offsetof(imq_options, m2l_split) + sizeof(int32_t))) {
        P.p2p_warps = opt->p2p_warps;
        P.p2p_chunk = opt->p2p_chunk;
        P.m2l_stages = opt->m2l_stages;
        P.m2l_split = opt->m2l_split;
    }
}

imq_plan_s *plan_create(const double *d_points, int64_t N, int64_t n_nodes, double c, int p, int leaf,
                        const imq_options *opt, cudaStream_t s) {
    double x0, y0, side;
    bool dups;
    int m2lk = IMQ_M2L_AUTO, alg = IMQ_ALG_FMM, depth = 0;
    int tmode = IMQ_TRANS_FP32;
    parse_plan_args(N, c, p, leaf, opt, x0, y0, side, dups, &m2lk, &alg, &depth, &tmode);
    const Allocator al = plan_allocator(opt);
    check_device();
    auto *h = new imq_plan_s;
    h->P.allocator = al;
    UseAllocator use(&h->P.allocator);
    try {
        Plan &P = h->P;
        IMQ_CUDA(cudaGetDevice(&P.device));
        P.N = N;
        P.n_nodes = n_nodes;
        P.c = c;
        P.p = p;
        P.leaf = leaf;
        P.x0 = x0;
        P.y0 = y0;
        P.side = side;
        P.m2l_kernel = m2lk;
        P.algorithm = alg;
        P.tc_depth = depth;
        P.trans64 = tmode == IMQ_TRANS_FP64;
        P.trans_mixed = tmode == IMQ_TRANS_MIXED;
        plan_tiles(P, opt);
        P.layout.build(p, 0);
        build_tree(P, d_points, s, dups);
        ensure_ops(P, false, s);
        if (tmode != IMQ_TRANS_FP32) ensure_ops(P, true, s);
        IMQ_CUDA(cudaStreamSynchronize(s));
    } catch (...) {
        delete h;
        throw;
    }
    return h;
}

}  // namespace

extern "C" {

imq_status imq_plan(const double *points, int64_t N, double c, int p, int leaf, const imq_options *opt,
                    void *stream, imq_plan_t *out) {
    if (out) *out = nullptr;
    return guard([&] {
        if (!out || !points) fail(IMQ_INVALID_ARG, "imq_plan: NULL pointer");
        double x0, y0, side;
        bool dups;
        parse_plan_args(N, c, p, leaf, opt, x0, y0, side, dups);   // argument errors before any GPU work
        (void)plan_allocator(opt);
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        check_device();
        DevIn pts(points, sizeof(double) * 2 * (size_t)N, s);
        *out = plan_create(static_cast<const double *>(pts.ptr), N, 0, c, p, leaf, opt, s);
    });
}

imq_status imq_plan_eval(const double *nodes, int64_t n_nodes, const double *targets, int64_t n_targets, double c,
                         int p, int leaf, const imq_options *opt, void *stream, imq_plan_t *out) {
    if (out) *out = nullptr;
    return guard([&] {
        if (!out || !nodes || !targets) fail(IMQ_INVALID_ARG, "imq_plan_eval: NULL pointer");
        if (n_nodes < 1 || n_targets < 1 || n_nodes + n_targets > 0x7FFFFFFF)
            fail(IMQ_INVALID_ARG, "imq_plan_eval: need n_nodes >= 1, n_targets >= 1, total < 2^31");
        if (opt && opt->check_duplicates) fail(IMQ_INVALID_ARG, "imq_plan_eval: targets may coincide with nodes");
        double x0, y0, side;
        bool dups;
        parse_plan_args(n_nodes + n_targets, c, p, leaf, opt, x0, y0, side, dups);
        (void)plan_allocator(opt);
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        check_device();
        const int64_t N = n_nodes + n_targets;
        DevIn a(nodes, sizeof(double) * 2 * (size_t)n_nodes, s), b(targets, sizeof(double) * 2 * (size_t)n_targets, s);
        AsyncMem all(sizeof(double) * 2 * (size_t)N, s);
        IMQ_CUDA(cudaMemcpyAsync(all.ptr, a.ptr, sizeof(double) * 2 * n_nodes, cudaMemcpyDeviceToDevice, s));
        IMQ_CUDA(cudaMemcpyAsync(all.as<double>() + 2 * n_nodes, b.ptr, sizeof(double) * 2 * n_targets,
                                 cudaMemcpyDeviceToDevice, s));
        *out = plan_create(all.as<double>(), N, n_nodes, c, p, leaf, opt, s);
    });
}

imq_status imq_plan_batched(const double *points, const int64_t *offsets, int nprob, const double *cvals, int p,
                            int leaf, const imq_options *opt, void *stream, imq_plan_t *out) {
    if (out) *out = nullptr;
    return guard([&] {
        if (!out || !points || !offsets || !cvals) fail(IMQ_INVALID_ARG, "imq_plan_batched: NULL pointer");
        if (nprob < 1) fail(IMQ_INVALID_ARG, "imq_plan_batched: nprob must be >= 1");
        std::vector<int64_t> offs(offsets, offsets + nprob + 1);
        std::vector<double> cs(cvals, cvals + nprob);
        if (offs[0] != 0) fail(IMQ_INVALID_ARG, "imq_plan_batched: offsets[0] must be 0");
        for (int b = 0; b < nprob; ++b) {
            if (offs[b + 1] <= offs[b]) fail(IMQ_INVALID_ARG, "imq_plan_batched: every problem needs >= 1 point");
            if (!std::isfinite(cs[b]) || cs[b] <= 0) fail(IMQ_INVALID_ARG, "imq_plan_batched: c must be finite and > 0");
        }
        const int64_t N = offs[nprob];
        double x0, y0, side;
        bool dups;
        int m2lk = IMQ_M2L_AUTO, alg = IMQ_ALG_FMM;
        int tmode = IMQ_TRANS_FP32;
        parse_plan_args(N, cs[0], p, leaf, opt, x0, y0, side, dups, &m2lk, &alg, nullptr, &tmode);
        (void)plan_allocator(opt);
        if (alg != IMQ_ALG_FMM) fail(IMQ_UNSUPPORTED, "imq_plan_batched: the treecode is built for single plans only");
        check_device();
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        DevIn pts(points, sizeof(double) * 2 * (size_t)N, s);
        if (side <= 0) {   // one square containing every problem's points
            std::vector<double> h(2 * (size_t)N);
            IMQ_CUDA(cudaMemcpyAsync(h.data(), pts.ptr, sizeof(double) * 2 * N, cudaMemcpyDefault, s));
            IMQ_CUDA(cudaStreamSynchronize(s));
            double mnx = INFINITY, mny = INFINITY, mxx = -INFINITY, mxy = -INFINITY;
            for (int64_t i = 0; i < N; ++i) {
                if (!std::isfinite(h[2 * i]) || !std::isfinite(h[2 * i + 1]))
                    fail(IMQ_INVALID_ARG, "imq_plan_batched: a coordinate is NaN or infinite");
                mnx = std::min(mnx, h[2 * i]); mxx = std::max(mxx, h[2 * i]);
                mny = std::min(mny, h[2 * i + 1]); mxy = std::max(mxy, h[2 * i + 1]);
            }
            x0 = mnx;
            y0 = mny;
            side = std::max(mxx - mnx, mxy - mny);
            if (!(side > 0)) side = 1.0;
        }
        auto *hp = new imq_plan_s;
        hp->P.allocator = plan_allocator(opt);
        UseAllocator use(&hp->P.allocator);
        try {
            Plan &P = hp->P;
            IMQ_CUDA(cudaGetDevice(&P.device));
            P.N = N;
            P.c = cs[0];
            P.p = p;
            P.leaf = leaf;
            P.x0 = x0;
            P.y0 = y0;
            P.side = side;
            P.m2l_kernel = m2lk;
            P.trans64 = tmode == IMQ_TRANS_FP64;
            P.trans_mixed = tmode == IMQ_TRANS_MIXED;
            plan_tiles(P, opt);
            P.layout.build(p, 0);
            build_batched_plan(P, static_cast<const double *>(pts.ptr), offs, cs, dups, s);
            ensure_ops(P, false, s);
            if (tmode != IMQ_TRANS_FP32) ensure_ops(P, true, s);
            IMQ_CUDA(cudaStreamSynchronize(s));
        } catch (...) {
            delete hp;
            throw;
        }
        *out = hp;
    });
}

void imq_plan_destroy(imq_plan_t plan) {
    if (!plan) return;
    cudaDeviceSynchronize();
    delete plan;
}

// FP32 product through the plan's cached graph: copy v in, replay, copy the result out, synchronise.
// The graph is captured on the first such call (and again when nrhs changes), after one direct
// product that makes every lazily created buffer and kernel attribute exist.
static void matvec_graph(Plan &P, const void *v, void *out, int nrhs, cudaStream_t s) {
    Plan::ProductGraph &G = P.pgraph;
    const size_t bytes = sizeof(float) * (size_t)nrhs * P.N;
    if (!G.exec || G.nrhs != nrhs) {
        G.exec = nullptr;
        G.cap.reset();
        G.in.alloc(bytes);
        G.out.alloc(bytes);
        G.us.alloc(bytes);
        G.bs.alloc(bytes);
        IMQ_CUDA(cudaMemsetAsync(G.in.ptr, 0, bytes, s));
        gather_sorted<float, float>(P, G.in.as<float>(), G.us.as<float>(), nrhs, s);
        fmm_apply<float>(P, G.us.as<float>(), G.bs.as<float>(), nrhs, s);
        scatter_sorted<float, float>(P, G.bs.as<float>(), G.out.as<float>(), nrhs, s);
        IMQ_CUDA(cudaStreamSynchronize(s));
        G.cap = std::make_unique<GraphCapture>();
        cudaStream_t cs = G.cap->begin();
        gather_sorted<float, float>(P, G.in.as<float>(), G.us.as<float>(), nrhs, cs);
        fmm_apply<float>(P, G.us.as<float>(), G.bs.as<float>(), nrhs, cs);
        scatter_sorted<float, float>(P, G.bs.as<float>(), G.out.as<float>(), nrhs, cs);
        G.exec = G.cap->instantiate();
        G.nrhs = nrhs;
    }
    IMQ_CUDA(cudaMemcpyAsync(G.in.ptr, v, bytes, cudaMemcpyDefault, s));
    IMQ_CUDA(cudaGraphLaunch(G.exec, s));
    IMQ_CUDA(cudaMemcpyAsync(out, G.out.ptr, bytes, cudaMemcpyDefault, s));
    check_device_errors(s);   // synchronises
}

static void matvec_impl(imq_plan_t plan, const void *v, void *out, int nrhs, imq_dtype dt, void *stream,
                        PhaseTimer *tm, bool dz = false) {
    if (!plan || !v || !out) fail(IMQ_INVALID_ARG, "imq_matvec: NULL pointer");
    if (nrhs < 1) fail(IMQ_INVALID_ARG, "imq_matvec: nrhs must be >= 1");
    if (dt != IMQ_F32 && dt != IMQ_F64) fail(IMQ_INVALID_ARG, "imq_matvec: unknown dtype");
    Plan &P = plan->P;
    UseAllocator use(&P.allocator);   // buffers the plan creates lazily
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // a call with a host buffer synchronises anyway: replay the cached graph of the product
    if (!tm && !dz && dt == IMQ_F32 && (!is_device_ptr(v) || !is_device_ptr(out))) {
        matvec_graph(P, v, out, nrhs, s);
        return;
    }
    const size_t es = dt == IMQ_F32 ? 4 : 8;
    const size_t bytes = es * (size_t)nrhs * P.N;
    DevIn dv(v, bytes, s);
    DevOut dout(out, bytes, s);
    AsyncMem us(bytes, s), bs(bytes, s);
    if (tm) tm->start(kPhGather, s);
    if (dt == IMQ_F32) gather_sorted<float, float>(P, static_cast<const float *>(dv.ptr), us.as<float>(), nrhs, s);
    else gather_sorted<double, double>(P, static_cast<const double *>(dv.ptr), us.as<double>(), nrhs, s);
    if (tm) { tm->stop(s); tm->launches += nrhs; }
    if (dz) {
        if (dt == IMQ_F32) fmm_apply_dz<float>(P, us.as<float>(), bs.as<float>(), nrhs, s);
        else fmm_apply_dz<double>(P, us.as<double>(), bs.as<double>(), nrhs, s);
    } else {
        if (dt == IMQ_F32) fmm_apply<float>(P, us.as<float>(), bs.as<float>(), nrhs, s, tm);
        else fmm_apply<double>(P, us.as<double>(), bs.as<double>(), nrhs, s, tm);
    }
    if (tm) tm->start(kPhScatter, s);
    if (dt == IMQ_F32) scatter_sorted<float, float>(P, bs.as<float>(), static_cast<float *>(dout.ptr), nrhs, s);
    else scatter_sorted<double, double>(P, bs.as<double>(), static_cast<double *>(dout.ptr), nrhs, s);
    if (tm) { tm->stop(s); tm->launches += nrhs; }
    dout.finish();
    if (dout.tmp || tm) check_device_errors(s);   // the call synchronises anyway
}

imq_status imq_matvec(imq_plan_t plan, const void *v, void *out, int nrhs, imq_dtype dt, void *stream) {
    return guard([&] { matvec_impl(plan, v, out, nrhs, dt, stream, nullptr); });
}

imq_status imq_matvec_dc(imq_plan_t plan, const void *v, void *out, int nrhs, imq_dtype dt, void *stream) {
    return guard([&] { matvec_impl(plan, v, out, nrhs, dt, stream, nullptr, true); });
}

// mode 0: evaluate, 1: transpose, 2: evaluate with dphi/dc
static void eval_impl(imq_plan_t plan, const void *in, void *out, int nrhs, imq_dtype dt, void *stream, int mode) {
    if (!plan || !in || !out) fail(IMQ_INVALID_ARG, "imq_evaluate: NULL pointer");
    if (nrhs < 1) fail(IMQ_INVALID_ARG, "imq_evaluate: nrhs must be >= 1");
    if (dt != IMQ_F32 && dt != IMQ_F64) fail(IMQ_INVALID_ARG, "imq_evaluate: unknown dtype");
    Plan &P = plan->P;
    UseAllocator use(&P.allocator);
    if (P.n_nodes <= 0) fail(IMQ_INVALID_ARG, "imq_evaluate: the plan was not made by imq_plan_eval");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t N = P.N, Nn = P.n_nodes, Nt = N - Nn;
    const int64_t in_len = mode == 1 ? Nt : Nn, out_len = mode == 1 ? Nn : Nt;
    const int64_t in_off = mode == 1 ? Nn : 0, out_off = mode == 1 ? 0 : Nn;
    const size_t es = dt == IMQ_F32 ? 4 : 8;
    DevIn din(in, es * (size_t)nrhs * in_len, s);
    DevOut dout(out, es * (size_t)nrhs * out_len, s);
    AsyncMem fu(es * (size_t)nrhs * N, s), fb(es * (size_t)nrhs * N, s);
    IMQ_CUDA(cudaMemsetAsync(fu.ptr, 0, es * (size_t)nrhs * N, s));
    for (int r = 0; r < nrhs; ++r)
        IMQ_CUDA(cudaMemcpyAsync(static_cast<char *>(fu.ptr) + es * ((size_t)r * N + in_off),
                                 static_cast<const char *>(din.ptr) + es * (size_t)r * in_len, es * in_len,
                                 cudaMemcpyDeviceToDevice, s));
    imq_plan_s *hp = plan;
    matvec_impl(hp, fu.ptr, fb.ptr, nrhs, dt, s, nullptr, mode == 2);
    for (int r = 0; r < nrhs; ++r)
        IMQ_CUDA(cudaMemcpyAsync(static_cast<char *>(dout.ptr) + es * (size_t)r * out_len,
                                 static_cast<const char *>(fb.ptr) + es * ((size_t)r * N + out_off), es * out_len,
                                 cudaMemcpyDeviceToDevice, s));
    dout.finish();
}

imq_status imq_evaluate(imq_plan_t eplan, const void *coef, void *out, int nrhs, imq_dtype dt, void *stream) {
    return guard([&] { eval_impl(eplan, coef, out, nrhs, dt, stream, 0); });
}

imq_status imq_evaluate_transpose(imq_plan_t eplan, const void *r, void *out, int nrhs, imq_dtype dt, void *stream) {
    return guard([&] { eval_impl(eplan, r, out, nrhs, dt, stream, 1); });
}

imq_status imq_evaluate_dc(imq_plan_t eplan, const void *coef, void *out, int nrhs, imq_dtype dt, void *stream) {
    return guard([&] { eval_impl(eplan, coef, out, nrhs, dt, stream, 2); });
}

imq_status imq_matvec_timed(imq_plan_t plan, const void *v, void *out, int nrhs, imq_dtype dt, void *stream,
                            float *phase_ms, int n_phases, int32_t *launches) {
    return guard([&] {
        if (!phase_ms || n_phases < 1) fail(IMQ_INVALID_ARG, "imq_matvec_timed: phase_ms required");
        PhaseTimer tm;
        matvec_impl(plan, v, out, nrhs, dt, stream, &tm);
        tm.collect(phase_ms, n_phases);
        if (launches) *launches = tm.launches;
    });
}

static void autotune_entry(const double *points, const int64_t *offsets, int nprob, const double *cvals,
                           double target, const int32_t *p_cand, int n_p, const int32_t *leaf_cand, int n_leaf,
                           int nrhs, const float *v, const imq_options *opt, void *stream, imq_tune_result *out) {
    {
        if (!points || !offsets || !cvals || !p_cand || !leaf_cand || !out)
            fail(IMQ_INVALID_ARG, "imq_autotune: NULL pointer");
        if (nprob < 1) fail(IMQ_INVALID_ARG, "imq_autotune: nprob must be >= 1");
        if (!(target > 0) || !std::isfinite(target)) fail(IMQ_INVALID_ARG, "imq_autotune: target must be > 0");
        if (n_p < 1 || n_p > 16 || n_leaf < 1 || n_leaf > 16)
            fail(IMQ_INVALID_ARG, "imq_autotune: need 1..16 candidates of p and of leaf");
        if (nrhs < 1 || nrhs > 16) fail(IMQ_INVALID_ARG, "imq_autotune: nrhs must be in [1, 16]");
        for (int k = 0; k < n_p; ++k)
            if (p_cand[k] < 1 || p_cand[k] > IMQ_MAX_P) fail(IMQ_INVALID_ARG, "imq_autotune: p out of [1, IMQ_MAX_P]");
        for (int k = 0; k < n_leaf; ++k)
            if (leaf_cand[k] < 1) fail(IMQ_INVALID_ARG, "imq_autotune: leaf must be >= 1");
        if (offsets[0] != 0) fail(IMQ_INVALID_ARG, "imq_autotune: offsets[0] must be 0");
        for (int q = 0; q < nprob; ++q) {
            if (offsets[q + 1] <= offsets[q]) fail(IMQ_INVALID_ARG, "imq_autotune: every problem needs >= 1 point");
            if (!std::isfinite(cvals[q]) || cvals[q] <= 0) fail(IMQ_INVALID_ARG, "imq_autotune: c must be finite and > 0");
        }
        if (offsets[nprob] > 0x7FFFFFFF) fail(IMQ_INVALID_ARG, "imq_autotune: too many points");
        check_device();
        autotune(points, offsets, nprob, cvals, target, p_cand, n_p, leaf_cand, n_leaf, nrhs, v, opt,
                 static_cast<cudaStream_t>(stream), out);
    }
}

imq_status imq_autotune(const double *points, const int64_t *offsets, int nprob, const double *cvals, double target,
                        const int32_t *p_cand, int n_p, const int32_t *leaf_cand, int n_leaf, int nrhs,
                        const imq_options *opt, void *stream, imq_tune_result *out) {
    return guard([&] {
        autotune_entry(points, offsets, nprob, cvals, target, p_cand, n_p, leaf_cand, n_leaf, nrhs, nullptr, opt,
                       stream, out);
    });
}

imq_status imq_autotune_v(const double *points, const int64_t *offsets, int nprob, const double *cvals,
                          double target, const int32_t *p_cand, int n_p, const int32_t *leaf_cand, int n_leaf,
                          int nrhs, const float *v, const imq_options *opt, void *stream, imq_tune_result *out) {
    return guard([&] {
        if (!v) fail(IMQ_INVALID_ARG, "imq_autotune_v: NULL test vectors");
        autotune_entry(points, offsets, nprob, cvals, target, p_cand, n_p, leaf_cand, n_leaf, nrhs, v, opt, stream,
                       out);
    });
}

imq_status imq_sync_check(void *stream) {
    return guard([&] { check_device_errors(static_cast<cudaStream_t>(stream)); });
}

imq_status imq_selftest_wait_timeout(void *stream) {
    return guard([&] {
        check_device();
        selftest_wait_timeout(static_cast<cudaStream_t>(stream));
    });
}

void imq_cg_default_options(imq_cg_options *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->struct_size = sizeof(imq_cg_options);
    o->rtol = 1e-6;
    o->maxit = 1000;
    o->precond = IMQ_PRECOND_SCHWARZ;
    o->schwarz_nmax = 0;   // 224 points (FP32 patches), 160 (FP64)
    o->schwarz_shift = 0.0;
    o->refine_steps = 0;
    o->inner_rtol = 1e-4;
    o->residual = IMQ_RESIDUAL_PLAN_F64;
}

namespace {

imq_status cg_entry(imq_plan_t plan, const double *f, double *coef, int nrhs, const imq_cg_options *opt,
                    imq_cg_info *info, double *rel_out, int32_t *iters_out, bool batched_call, void *stream) {
    if (info) {
        std::memset(info, 0, sizeof(*info));
        info->status = IMQ_CUDA_ERROR;
    }
    const imq_status st = guard([&] {
        if (!plan || !f || !coef) fail(IMQ_INVALID_ARG, "imq_cg_solve: NULL pointer");
        if (nrhs < 1) fail(IMQ_INVALID_ARG, "imq_cg_solve: nrhs must be >= 1");
        UseAllocator use(&plan->P.allocator);   // preconditioner factors and solver work arrays
        imq_cg_options o;
        imq_cg_default_options(&o);
        if (opt) {
            if (opt->struct_size < (int)offsetof(imq_cg_options, coarse_points))
                fail(IMQ_INVALID_ARG, "imq_cg_solve: imq_cg_options.struct_size too small");
            std::memcpy(&o, opt, std::min(sizeof(o), (size_t)opt->struct_size));
        }
        if (!(o.rtol > 0) || !std::isfinite(o.rtol)) fail(IMQ_INVALID_ARG, "imq_cg_solve: rtol must be > 0");
        if (o.maxit < 1) fail(IMQ_INVALID_ARG, "imq_cg_solve: maxit must be >= 1");
        if (o.precond != IMQ_PRECOND_NONE && o.precond != IMQ_PRECOND_SCHWARZ && o.precond != IMQ_PRECOND_SCHWARZ_2L)
            fail(IMQ_INVALID_ARG, "imq_cg_solve: unknown preconditioner");
        if (o.coarse_points < 0 || o.coarse_points > 1024)
            fail(IMQ_INVALID_ARG, "imq_cg_solve: coarse_points must be in [0, 1024]");
        if (o.coarse_gram < 0 || o.coarse_gram > 2) fail(IMQ_INVALID_ARG, "imq_cg_solve: unknown coarse_gram");
        if (o.krylov != IMQ_KRYLOV_CG && o.krylov != IMQ_KRYLOV_GMRES)
            fail(IMQ_INVALID_ARG, "imq_cg_solve: unknown krylov method");
        if (o.gmres_m < 0 || o.gmres_m > 200) fail(IMQ_INVALID_ARG, "imq_cg_solve: gmres_m must be in [0, 200]");
        if (o.schwarz_nmax < 0 || o.schwarz_nmax > 224) fail(IMQ_INVALID_ARG, "imq_cg_solve: schwarz_nmax must be in [0, 224]");
        if (o.inner_operator < IMQ_OPERATOR_FAST_F32 || o.inner_operator > IMQ_OPERATOR_DENSE_F64)
            fail(IMQ_INVALID_ARG, "imq_cg_solve: unknown inner operator");
        if (o.schwarz_fp64 && o.schwarz_nmax > 160)
            fail(IMQ_INVALID_ARG, "imq_cg_solve: schwarz_nmax must be <= 160 with FP64 patches");
        if (o.residual != IMQ_RESIDUAL_PLAN_F64 && o.residual != IMQ_RESIDUAL_DENSE_F64)
            fail(IMQ_INVALID_ARG, "imq_cg_solve: unknown residual mode");
        Plan &P = plan->P;
        if (batched_call && P.prob_off.empty())
            fail(IMQ_INVALID_ARG, "imq_cg_solve_batched: plan was not made by imq_plan_batched");
        Plan *RP = o.residual_plan ? &o.residual_plan->P : nullptr;
        if (RP && RP->N != P.N) fail(IMQ_INVALID_ARG, "imq_cg_solve: residual_plan has a different N");
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        const size_t bytes = sizeof(double) * (size_t)nrhs * P.N;
        DevIn df(f, bytes, s);
        DevOut dx(coef, bytes, s);
        if (o.x0_given && dx.tmp) IMQ_CUDA(cudaMemcpyAsync(dx.ptr, coef, bytes, cudaMemcpyHostToDevice, s));
        try {
            if (!P.prob_off.empty() && o.precond == IMQ_PRECOND_SCHWARZ_2L && o.krylov != IMQ_KRYLOV_GMRES)
                fail(IMQ_UNSUPPORTED, "imq_cg_solve: on batched plans the two-level preconditioner runs with GMRES");
            if (!P.prob_off.empty())
                cg_solve_batched(P, static_cast<const double *>(df.ptr), static_cast<double *>(dx.ptr), nrhs, o,
                                 info, rel_out, iters_out, s);
            else
                cg_solve(P, static_cast<const double *>(df.ptr), static_cast<double *>(dx.ptr), nrhs, o, RP, info, s);
        } catch (const Error &e) {
            if (e.status == IMQ_NOT_CONVERGED || e.status == IMQ_NUMERICAL) dx.finish();
            throw;
        }
        dx.finish();
    });
    if (info) info->status = st;
    return st;
}

}  // namespace

imq_status imq_cg_solve(imq_plan_t plan, const double *f, double *coef, int nrhs, const imq_cg_options *opt,
                        imq_cg_info *info, void *stream) {
    return cg_entry(plan, f, coef, nrhs, opt, info, nullptr, nullptr, false, stream);
}

imq_status imq_cg_solve_batched(imq_plan_t plan, const double *f, double *coef, int nrhs, const imq_cg_options *opt,
                                imq_cg_info *info, double *rel_residual, int32_t *iterations, void *stream) {
    return cg_entry(plan, f, coef, nrhs, opt, info, rel_residual, iterations, true, stream);
}

imq_status imq_dense_matvec(const double *points, int64_t N, double c, const void *v, void *out, int nrhs,
                            imq_dtype dt, void *stream) {
    return guard([&] {
        if (!points || !v || !out) fail(IMQ_INVALID_ARG, "imq_dense_matvec: NULL pointer");
        if (N < 1 || N > 0x7FFFFFFF) fail(IMQ_INVALID_ARG, "imq_dense_matvec: N must be in [1, 2^31-1]");
        if (!std::isfinite(c) || c <= 0) fail(IMQ_INVALID_ARG, "imq_dense_matvec: c must be finite and > 0");
        if (nrhs < 1) fail(IMQ_INVALID_ARG, "imq_dense_matvec: nrhs must be >= 1");
        if (dt != IMQ_F32 && dt != IMQ_F64) fail(IMQ_INVALID_ARG, "imq_dense_matvec: unknown dtype");
        check_device();
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        const size_t es = dt == IMQ_F32 ? 4 : 8;
        DevIn pts(points, sizeof(double) * 2 * (size_t)N, s);
        DevIn dv(v, es * (size_t)nrhs * N, s);
        DevOut dout(out, es * (size_t)nrhs * N, s);
        dense_matvec_dev(static_cast<const double *>(pts.ptr), N, c, dv.ptr, dout.ptr, nrhs, dt, s);
        dout.finish();
    });
}

imq_status imq_plan_get_info(imq_plan_t plan, imq_plan_info *info) {
    return guard([&] {
        if (!plan || !info) fail(IMQ_INVALID_ARG, "imq_plan_get_info: NULL pointer");
        const Plan &P = plan->P;
        std::memset(info, 0, sizeof(*info));
        info->n_points = P.N;
        info->n_nodes = P.n_nodes;
        info->n_problems = P.nprob;
        info->algorithm = P.algorithm;
        info->n_boxes = P.nbox;
        info->n_leaves = P.nleaf;
        info->max_level = P.max_level;
        info->p = P.p;
        info->leaf = P.leaf;
        info->k_real = P.layout.K;
        info->x0 = P.x0;
        info->y0 = P.y0;
        info->side = P.side;
        info->c = P.c;
        info->n_u = P.U.total;
        info->n_v = P.V.total;
        info->n_w = P.W.total;
        info->n_x = P.X.total;
        info->p2p_pairs = P.p2p_pairs;
        info->m2l_pairs = P.m2l_pairs;
        info->device_bytes = P.device_bytes();
    });
}

imq_status imq_plan_export_tree(imq_plan_t plan, uint32_t *codes, int64_t *perm, int32_t *level, uint32_t *prefix,
                                int64_t *begin, int64_t *end, int32_t *parent, int32_t *child) {
    return guard([&] {
        if (!plan) fail(IMQ_INVALID_ARG, "imq_plan_export_tree: NULL plan");
        const Plan &P = plan->P;
        auto d2h = [](void *dst, const DevMem &src, size_t bytes) {
            if (dst) IMQ_CUDA(cudaMemcpy(dst, src.ptr, bytes, cudaMemcpyDeviceToHost));
        };
        d2h(codes, P.codes, sizeof(uint32_t) * P.N);
        d2h(level, P.level, sizeof(int32_t) * P.nbox);
        d2h(prefix, P.prefix, sizeof(uint32_t) * P.nbox);
        d2h(parent, P.parent, sizeof(int32_t) * P.nbox);
        d2h(child, P.child, sizeof(int32_t) * 4 * P.nbox);
        if (perm) {
            std::vector<int32_t> t(P.N);
            d2h(t.data(), P.perm, sizeof(int32_t) * P.N);
            for (int64_t i = 0; i < P.N; ++i) perm[i] = t[i];
        }
        if (begin || end) {
            std::vector<int32_t> b(P.nbox), e(P.nbox);
            d2h(b.data(), P.begin, sizeof(int32_t) * P.nbox);
            d2h(e.data(), P.end, sizeof(int32_t) * P.nbox);
            for (int i = 0; i < P.nbox; ++i) {
                if (begin) begin[i] = b[i];
                if (end) end[i] = e[i];
            }
        }
    });
}

imq_status imq_plan_export_list(imq_plan_t plan, char which, int32_t *offsets, int32_t *items) {
    return guard([&] {
        if (!plan) fail(IMQ_INVALID_ARG, "imq_plan_export_list: NULL plan");
        const Plan &P = plan->P;
        const ListCSR *L = nullptr;
        switch (which) {
            case 'U': L = &P.U; break;
            case 'V': L = &P.V; break;
            case 'W': L = &P.W; break;
            case 'X': L = &P.X; break;
            default: fail(IMQ_INVALID_ARG, "imq_plan_export_list: which must be U, V, W or X");
        }
        if (offsets) IMQ_CUDA(cudaMemcpy(offsets, L->off.ptr, sizeof(int32_t) * (P.nbox + 1), cudaMemcpyDeviceToHost));
        if (items && L->total > 0)
            IMQ_CUDA(cudaMemcpy(items, L->items.ptr, sizeof(int32_t) * L->total, cudaMemcpyDeviceToHost));
    });
}

}  // extern "C"
