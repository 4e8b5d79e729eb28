// The plain ("standard row-column") IMQ product of the paper's Section 3,
// computed matrix-free on all N^2 pairs:
//     b_i = sum_j v_j / sqrt(|x_i - x_j|^2 + c^2)            (Eq. (4)-(5))
//
// FP32 form: each thread owns kTPT targets held in registers; source tiles of
// kTile (x, y, v, 0) float4 records are staged in shared memory by a 1-D TMA
// bulk copy (cp.async.bulk + mbarrier), double-buffered, and read back as
// warp-wide broadcasts.  Per pair: 2 FADD + 2 FFMA + 1 MUFU rsqrt + 1 FFMA.
// Partial sums over one tile are FP32 and are folded into FP64 accumulators
// once per tile, which keeps the rounding error of a 10^6-term sum at the
// level of one tile.
// FP64 form: the same loop in double with 1/sqrt, plain cooperative loads.
#include <mutex>

#include "imq_internal.h"
#include "ptx.cuh"
#include "util.cuh"

namespace imq {
namespace {

constexpr int kThreads = 256;
constexpr int kTPT = 4;            // targets per thread
constexpr int kTile = 1024;        // sources per shared-memory tile (16 KB)

template <class Tin>
__global__ void pack_sources(const double *__restrict__ pts, const Tin *__restrict__ v, int64_t n,
                             float4 *__restrict__ src) {
    int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j < n) src[j] = make_float4((float)pts[2 * j], (float)pts[2 * j + 1], (float)v[j], 0.f);
}

template <class Tout>
__global__ void __launch_bounds__(kThreads) dense_f32(const float4 *__restrict__ src, int64_t n, float c2,
                                                      Tout *__restrict__ out, int *err) {
    __shared__ __align__(128) float4 buf[2][kTile];
    __shared__ __align__(8) uint64_t bar[2];
    const int tid = threadIdx.x;
    const int64_t t0 = (int64_t)blockIdx.x * (kThreads * kTPT);
    float xt[kTPT], yt[kTPT];
    double acc[kTPT];
#pragma unroll
    for (int k = 0; k < kTPT; ++k) {
        int64_t t = t0 + k * kThreads + tid;
        float4 q = t < n ? src[t] : make_float4(0.f, 0.f, 0.f, 0.f);
        xt[k] = q.x;
        yt[k] = q.y;
        acc[k] = 0.0;
    }
    const int ntiles = (int)((n + kTile - 1) / kTile);
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    auto issue = [&](int k) {
        int64_t s0 = (int64_t)k * kTile;
        int cnt = (int)min((int64_t)kTile, n - s0);
        uint32_t bytes = (uint32_t)cnt * sizeof(float4);
        mbar_arrive_expect_tx(&bar[k & 1], bytes);
        bulk_g2s(buf[k & 1], src + s0, bytes, &bar[k & 1]);
    };
    if (tid == 0 && ntiles > 0) issue(0);
    bool ok = true;
    for (int k = 0; k < ntiles; ++k) {
        if (tid == 0 && k + 1 < ntiles) issue(k + 1);
        if (!mbar_wait(&bar[k & 1], (k >> 1) & 1)) ok = false;
        if (__syncthreads_or(!ok)) {
            if (tid == 0) set_error(err, kErrWaitTimeout);
            // drain the copy still in flight (bounded) before leaving
            if (tid == 0 && k + 1 < ntiles) mbar_wait(&bar[(k + 1) & 1], ((k + 1) >> 1) & 1);
            return;
        }
        const int cnt = (int)min((int64_t)kTile, n - (int64_t)k * kTile);
        const float4 *b = buf[k & 1];
        float part[kTPT];
#pragma unroll
        for (int q = 0; q < kTPT; ++q) part[q] = 0.f;
#pragma unroll 8
        for (int s = 0; s < cnt; ++s) {
            const float4 q = b[s];
#pragma unroll
            for (int k2 = 0; k2 < kTPT; ++k2) {
                const float dx = xt[k2] - q.x;
                const float dy = yt[k2] - q.y;
                const float d2 = fmaf(dx, dx, fmaf(dy, dy, c2));
                part[k2] = fmaf(rsqrtf(d2), q.z, part[k2]);
            }
        }
#pragma unroll
        for (int q = 0; q < kTPT; ++q) acc[q] += (double)part[q];
        __syncthreads();   // every thread is done with buf[k&1] before it is refilled
    }
#pragma unroll
    for (int k = 0; k < kTPT; ++k) {
        int64_t t = t0 + k * kThreads + tid;
        if (t < n) out[t] = (Tout)acc[k];
    }
}

template <class Tin, class Tout>
__global__ void __launch_bounds__(256) dense_f64(const double *__restrict__ pts, const Tin *__restrict__ v,
                                                 int64_t n, double c2, Tout *__restrict__ out) {
    constexpr int kT = 512;
    __shared__ double sx[kT], sy[kT], sv[kT];
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const double xt = t < n ? pts[2 * t] : 0.0;
    const double yt = t < n ? pts[2 * t + 1] : 0.0;
    double acc = 0.0;
    for (int64_t s0 = 0; s0 < n; s0 += kT) {
        const int cnt = (int)min((int64_t)kT, n - s0);
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
            sx[i] = pts[2 * (s0 + i)];
            sy[i] = pts[2 * (s0 + i) + 1];
            sv[i] = (double)v[s0 + i];
        }
        __syncthreads();
        for (int s = 0; s < cnt; ++s) {
            const double dx = xt - sx[s];
            const double dy = yt - sy[s];
            acc += sv[s] / sqrt(fma(dx, dx, fma(dy, dy, c2)));
        }
        __syncthreads();
    }
    if (t < n) out[t] = (Tout)acc;
}

// Block-diagonal FP64 dense product of a batched plan: points of problem b
// occupy [off[b], off[b+1]) (Morton order); target i sums over the sources of
// its own problem only, with that problem's shape.  One thread per target, the
// problem found by binary search; sources are read through L1 (the threads of
// a warp share one problem almost always, so their loads coincide).
__global__ void __launch_bounds__(256) dense_f64_seg(const double2 *__restrict__ pos, const int64_t *__restrict__ off,
                                                     int nprob, const double *__restrict__ prob_c,
                                                     const double *__restrict__ v, int64_t n,
                                                     double *__restrict__ out) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n) return;
    int lo = 0, hi = nprob;   // off[lo] <= t < off[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= t) lo = mid;
        else hi = mid;
    }
    const double c = prob_c[lo], c2 = c * c;
    const double2 xt = pos[t];
    double acc = 0.0;
    for (int64_t j = off[lo]; j < off[lo + 1]; ++j) {
        const double2 xs = pos[j];
        const double dx = xt.x - xs.x, dy = xt.y - xs.y;
        acc += v[j] / sqrt(fma(dx, dx, fma(dy, dy, c2)));
    }
    out[t] = acc;
}

}  // namespace

void dense_f64_async(const double *d_points, int64_t N, double c, const double *d_v, double *d_out, cudaStream_t s) {
    dense_f64<double, double><<<(unsigned)((N + 255) / 256), 256, 0, s>>>(d_points, d_v, N, c * c, d_out);
    IMQ_LAUNCH_CHECK();
}

void dense_f64_seg_async(const double *d_points, const int64_t *d_off, int nprob, const double *d_prob_c,
                         const double *d_v, double *d_out, int64_t N, cudaStream_t s) {
    dense_f64_seg<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(reinterpret_cast<const double2 *>(d_points), d_off,
                                                               nprob, d_prob_c, d_v, N, d_out);
    IMQ_LAUNCH_CHECK();
}

void dense_matvec_dev(const double *d_points, int64_t N, double c, const void *d_v, void *d_out,
                      int nrhs, imq_dtype dt, cudaStream_t s) {
    AsyncMem err(sizeof(int), s);
    IMQ_CUDA(cudaMemsetAsync(err.ptr, 0, sizeof(int), s));
    if (dt == IMQ_F32) {
        AsyncMem src(sizeof(float4) * (size_t)N, s);
        for (int r = 0; r < nrhs; ++r) {
            const float *v = static_cast<const float *>(d_v) + (size_t)r * N;
            float *o = static_cast<float *>(d_out) + (size_t)r * N;
            pack_sources<float><<<(unsigned)((N + 255) / 256), 256, 0, s>>>(d_points, v, N, src.as<float4>());
            IMQ_LAUNCH_CHECK();
            const unsigned grid = (unsigned)((N + kThreads * kTPT - 1) / (kThreads * kTPT));
            dense_f32<float><<<grid, kThreads, 0, s>>>(src.as<float4>(), N, (float)(c * c), o, err.as<int>());
            IMQ_LAUNCH_CHECK();
        }
    } else {
        for (int r = 0; r < nrhs; ++r) {
            const double *v = static_cast<const double *>(d_v) + (size_t)r * N;
            double *o = static_cast<double *>(d_out) + (size_t)r * N;
            dense_f64<double, double><<<(unsigned)((N + 255) / 256), 256, 0, s>>>(d_points, v, N, c * c, o);
            IMQ_LAUNCH_CHECK();
        }
    }
    int h_err = 0;
    IMQ_CUDA(cudaMemcpyAsync(&h_err, err.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
    IMQ_CUDA(cudaStreamSynchronize(s));
    if (h_err & kErrWaitTimeout) fail(IMQ_TIMEOUT, "dense matvec: shared-memory tile wait timed out");
}

// ------------------------------------------------------------------ allocation-free variant
// imq_dense_matvec_noalloc: the FP32 dense product above with its scratch (the
// packed (x, y, v, 0) source records and the wait-timeout word) held in one
// file-scope device array instead of memory obtained from cudaMallocAsync.
// Every GPU that loads the library keeps this array (IMQ_NOALLOC_MAX_N + 1
// float4 records, 4 MiB + 16 B) until the process exits.  The host only ever
// handles the array through the device address cudaGetSymbolAddress returns
// for the current device; the array's name in host code is a host-side stand-in
// and must never be passed to a kernel.
namespace {

static __device__ __align__(256) float4 g_noalloc_scratch[IMQ_NOALLOC_MAX_N + 1];

std::mutex g_noalloc_mu;
float4 *g_noalloc_addr[64] = {nullptr};

// Device address of the scratch array on the current device, resolved once per
// device.  The first resolution on a device also clears the error word (the
// last record), enqueued on `s`; from then on the word collects the timeouts
// of every call until imq_sync_check reads and clears it.
float4 *noalloc_scratch(cudaStream_t s) {
    int dev = 0;
    IMQ_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) fail(IMQ_UNSUPPORTED, "imq_dense_matvec_noalloc: device index out of range");
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) {
            (void)cudaGetLastError();
            fail(IMQ_CUDA_ERROR, std::string("imq_dense_matvec_noalloc: cudaGetSymbolAddress failed: ") +
                                     cudaGetErrorString(e));
        }
        IMQ_CUDA(cudaMemsetAsync(static_cast<float4 *>(p) + IMQ_NOALLOC_MAX_N, 0, sizeof(float4), s));
        g_noalloc_addr[dev] = static_cast<float4 *>(p);
    }
    return g_noalloc_addr[dev];
}

bool is_device_memory(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

int *noalloc_error_word() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        (void)cudaGetLastError();
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    return g_noalloc_addr[dev] ? reinterpret_cast<int *>(g_noalloc_addr[dev] + IMQ_NOALLOC_MAX_N) : nullptr;
}

void dense_matvec_noalloc(const double *points, int64_t N, double c, const float *v, float *out, cudaStream_t s) {
    if (!points || !v || !out) fail(IMQ_INVALID_ARG, "imq_dense_matvec_noalloc: NULL pointer");
    if (N < 1) fail(IMQ_INVALID_ARG, "imq_dense_matvec_noalloc: N must be >= 1");
    if (N > IMQ_NOALLOC_MAX_N)
        fail(IMQ_INVALID_ARG, "imq_dense_matvec_noalloc: N = " + std::to_string(N) +
                                  " exceeds the fixed scratch capacity IMQ_NOALLOC_MAX_N = " +
                                  std::to_string((long long)IMQ_NOALLOC_MAX_N));
    if (!(c > 0) || !(c < INFINITY)) fail(IMQ_INVALID_ARG, "imq_dense_matvec_noalloc: c must be finite and > 0");
    if (!is_device_memory(points) || !is_device_memory(v) || !is_device_memory(out))
        fail(IMQ_INVALID_ARG, "imq_dense_matvec_noalloc: points, v and out must be device memory");
    check_device();
    float4 *src = noalloc_scratch(s);
    // a bounded tile wait that runs out sets a bit here; imq_sync_check reports it
    int *err = reinterpret_cast<int *>(src + IMQ_NOALLOC_MAX_N);
    pack_sources<float><<<(unsigned)((N + 255) / 256), 256, 0, s>>>(points, v, N, src);
    IMQ_LAUNCH_CHECK();
    const unsigned grid = (unsigned)((N + kThreads * kTPT - 1) / (kThreads * kTPT));
    dense_f32<float><<<grid, kThreads, 0, s>>>(src, N, (float)(c * c), out, err);
    IMQ_LAUNCH_CHECK();
}

}  // namespace imq

extern "C" imq_status imq_dense_matvec_noalloc(const double *points, int64_t N, double c, const float *v,
                                               float *out, void *stream) {
    return imq::guarded_call([&] {
        imq::dense_matvec_noalloc(points, N, c, v, out, static_cast<cudaStream_t>(stream));
    });
}
