#include <string>
// Host utilities of the library: error handling, device memory, exclusive scan.
#include <cstdio>
#include <cstring>
#include <mutex>

#include "imq_internal.h"
#include "ptx.cuh"
#include "util.cuh"

namespace imq {

void fail(imq_status s, const std::string &msg) { throw Error{s, msg}; }

void cuda_check(cudaError_t e, const char *what, const char *file, int line) {
    if (e == cudaSuccess) return;
    char buf[512];
    snprintf(buf, sizeof(buf), "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
    if (e == cudaErrorMemoryAllocation) {
        (void)cudaGetLastError();
        fail(IMQ_OOM, buf);
    }
    fail(IMQ_CUDA_ERROR, buf);
}

namespace {
thread_local const Allocator *t_alloc = nullptr;
}

UseAllocator::UseAllocator(const Allocator *a) : prev(t_alloc) { t_alloc = (a && a->alloc) ? a : nullptr; }
UseAllocator::~UseAllocator() { t_alloc = prev; }

void DevMem::alloc(size_t n) {
    release();
    if (n == 0) n = 16;
    if (t_alloc) {
        ptr = t_alloc->alloc(n, t_alloc->ctx);
        if (!ptr) fail(IMQ_OOM, "the caller's allocator returned NULL for " + std::to_string(n) + " bytes");
        by = *t_alloc;
        bytes = n;
        return;
    }
    by = Allocator{};
    cudaError_t e = cudaMalloc(&ptr, n);
    if (e != cudaSuccess) {
        ptr = nullptr;
        (void)cudaGetLastError();
        fail(e == cudaErrorMemoryAllocation ? IMQ_OOM : IMQ_CUDA_ERROR,
             std::string("cudaMalloc of ") + std::to_string(n) + " bytes failed: " + cudaGetErrorString(e));
    }
    bytes = n;
}

void DevMem::release() {
    if (ptr) {
        if (by.free) by.free(ptr, bytes, by.ctx);
        else cudaFree(ptr);
    }
    ptr = nullptr;
    bytes = 0;
    by = Allocator{};
}

AsyncMem::AsyncMem(size_t bytes, cudaStream_t s) : stream(s) {
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMallocAsync(&ptr, bytes, s);
    if (e != cudaSuccess) {
        ptr = nullptr;
        (void)cudaGetLastError();
        fail(e == cudaErrorMemoryAllocation ? IMQ_OOM : IMQ_CUDA_ERROR,
             std::string("cudaMallocAsync failed: ") + cudaGetErrorString(e));
    }
}

AsyncMem::~AsyncMem() {
    if (ptr) cudaFreeAsync(ptr, stream);
}

// ------------------------------------------------------------------ phase timer
void PhaseTimer::start(int phase, cudaStream_t s) {
    Rec r{phase, nullptr, nullptr};
    IMQ_CUDA(cudaEventCreate(&r.a));
    IMQ_CUDA(cudaEventCreate(&r.b));
    IMQ_CUDA(cudaEventRecord(r.a, s));
    recs.push_back(r);
}

void PhaseTimer::stop(cudaStream_t s) { IMQ_CUDA(cudaEventRecord(recs.back().b, s)); }

void PhaseTimer::collect(float *ms, int n) {
    for (int k = 0; k < n; ++k) ms[k] = 0.f;
    if (recs.empty()) return;
    IMQ_CUDA(cudaEventSynchronize(recs.back().b));
    for (auto &r : recs) {
        float t = 0.f;
        IMQ_CUDA(cudaEventElapsedTime(&t, r.a, r.b));
        if (r.phase >= 0 && r.phase < n) ms[r.phase] += t;
    }
}

PhaseTimer::~PhaseTimer() {
    for (auto &r : recs) {
        if (r.a) cudaEventDestroy(r.a);
        if (r.b) cudaEventDestroy(r.b);
    }
}

// ------------------------------------------------------------------ device error word
// One int per device, a file-scope device variable: resolving its address
// (cudaGetSymbolAddress, once per device) allocates nothing, so checking for a
// failed bounded wait never needs device memory of its own.
namespace {
__device__ int g_err_word_dev;
std::mutex g_err_mu;
int *g_err_word[64] = {nullptr};
}  // namespace

int *device_error_word() {
    int dev = 0;
    IMQ_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) fail(IMQ_UNSUPPORTED, "device index out of range");
    std::lock_guard<std::mutex> lk(g_err_mu);
    if (!g_err_word[dev]) {
        void *p = nullptr;
        IMQ_CUDA(cudaGetSymbolAddress(&p, g_err_word_dev));
        g_err_word[dev] = static_cast<int *>(p);
    }
    return g_err_word[dev];
}

cudaStream_t GraphCapture::begin() {
    IMQ_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    IMQ_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    capturing = true;
    return cs;
}

cudaGraphExec_t GraphCapture::instantiate() {
    capturing = false;
    IMQ_CUDA(cudaStreamEndCapture(cs, &graph));
    IMQ_CUDA(cudaGraphInstantiate(&exec, graph, cudaGraphInstantiateFlagUseNodePriority));
    return exec;
}

GraphCapture::~GraphCapture() {
    if (capturing) {
        cudaGraph_t partial = nullptr;
        if (cudaStreamEndCapture(cs, &partial) == cudaSuccess && partial) cudaGraphDestroy(partial);
        (void)cudaGetLastError();
    }
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (cs) cudaStreamDestroy(cs);
}

void AuxStream::ensure() {
    if (s) return;
    int least = 0, greatest = 0;
    IMQ_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    IMQ_CUDA(cudaStreamCreateWithPriority(&hi, cudaStreamNonBlocking, greatest));
    IMQ_CUDA(cudaStreamCreateWithPriority(&s, cudaStreamNonBlocking, least));
    IMQ_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    IMQ_CUDA(cudaEventCreateWithFlags(&xready, cudaEventDisableTiming));
    IMQ_CUDA(cudaEventCreateWithFlags(&mready, cudaEventDisableTiming));
    IMQ_CUDA(cudaEventCreateWithFlags(&join, cudaEventDisableTiming));
    IMQ_CUDA(cudaEventCreateWithFlags(&done, cudaEventDisableTiming));
}

AuxStream::~AuxStream() {
    if (fork) cudaEventDestroy(fork);
    if (xready) cudaEventDestroy(xready);
    if (mready) cudaEventDestroy(mready);
    if (join) cudaEventDestroy(join);
    if (done) cudaEventDestroy(done);
    if (s) cudaStreamDestroy(s);
    if (hi) cudaStreamDestroy(hi);
}

namespace {
// A wait that nothing satisfies: the bounded mbarrier wait gives up after its
// limit and reports through the error word (self-test of the timeout path).
__global__ void k_wait_never(int *err) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (!mbar_wait(&bar, 0) && threadIdx.x == 0) set_error(err, kErrWaitTimeout);
}
}  // namespace

void selftest_wait_timeout(cudaStream_t s) {
    k_wait_never<<<1, 32, 0, s>>>(device_error_word());
    IMQ_LAUNCH_CHECK();
    check_device_errors(s);
}

void check_device_errors(cudaStream_t s) {
    // the shared word, and the allocation-free dense product's own word if that
    // entry point has run on this device
    int *w[2] = {device_error_word(), noalloc_error_word()};
    int h[2] = {0, 0};
    for (int k = 0; k < 2; ++k)
        if (w[k]) IMQ_CUDA(cudaMemcpyAsync(&h[k], w[k], sizeof(int), cudaMemcpyDeviceToHost, s));
    IMQ_CUDA(cudaStreamSynchronize(s));
    const int any = h[0] | h[1];
    if (any) {
        for (int k = 0; k < 2; ++k)
            if (h[k]) IMQ_CUDA(cudaMemsetAsync(w[k], 0, sizeof(int), s));
        IMQ_CUDA(cudaStreamSynchronize(s));
        if (any & kErrWaitTimeout) fail(IMQ_TIMEOUT, "a bounded wait in a kernel ran out; results are invalid");
        fail(IMQ_CUDA_ERROR, "a kernel reported error flags " + std::to_string(any));
    }
}

// ------------------------------------------------------------------ scan
namespace {
constexpr int kScanBlock = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanBlock * kScanItems;

template <class T>
__device__ T block_exclusive_scan(T v, T *sh, T *total) {
    // Hillis-Steele over a 1024-thread block; returns the exclusive prefix of v.
    const int tid = threadIdx.x;
    sh[tid] = v;
    __syncthreads();
    for (int off = 1; off < kScanBlock; off <<= 1) {
        T a = tid >= off ? sh[tid - off] : T(0);
        __syncthreads();
        sh[tid] += a;
        __syncthreads();
    }
    T incl = sh[tid];
    if (total) *total = sh[kScanBlock - 1];
    __syncthreads();
    return incl - v;
}

template <class T>
__global__ void __launch_bounds__(kScanBlock) scan_tiles(const T *in, T *out, T *tile_sums, int64_t n) {
    __shared__ T sh[kScanBlock];
    __shared__ T tot;
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    T loc[kScanItems];
    T s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        loc[k] = base + k < n ? in[base + k] : T(0);
        s += loc[k];
    }
    T pre = block_exclusive_scan<T>(s, sh, &tot);
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n) out[base + k] = pre;
        pre += loc[k];
    }
    if (threadIdx.x == 0 && tile_sums) tile_sums[blockIdx.x] = tot;
}

template <class T>
__global__ void add_tile_offsets(T *out, const T *tile_off, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += tile_off[i / kScanTile];
}

template <class T>
__global__ void write_total(const T *in, const T *out, int64_t n, T *total) {
    *total = n > 0 ? out[n - 1] + in[n - 1] : T(0);
}
}  // namespace

template <class T>
void exclusive_scan(const T *d_in, T *d_out, int64_t n, T *d_total, cudaStream_t s) {
    if (n <= 0) {
        if (d_total) IMQ_CUDA(cudaMemsetAsync(d_total, 0, sizeof(T), s));
        return;
    }
    const int64_t ntiles = (n + kScanTile - 1) / kScanTile;
    if (ntiles == 1) {
        scan_tiles<T><<<1, kScanBlock, 0, s>>>(d_in, d_out, nullptr, n);
        IMQ_LAUNCH_CHECK();
    } else {
        AsyncMem sums(sizeof(T) * ntiles, s), offs(sizeof(T) * ntiles, s);
        scan_tiles<T><<<(unsigned)ntiles, kScanBlock, 0, s>>>(d_in, d_out, sums.as<T>(), n);
        IMQ_LAUNCH_CHECK();
        exclusive_scan<T>(sums.as<T>(), offs.as<T>(), ntiles, nullptr, s);
        add_tile_offsets<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(d_out, offs.as<T>(), n);
        IMQ_LAUNCH_CHECK();
    }
    if (d_total) {
        write_total<T><<<1, 1, 0, s>>>(d_in, d_out, n, d_total);
        IMQ_LAUNCH_CHECK();
    }
}

template void exclusive_scan<int32_t>(const int32_t *, int32_t *, int64_t, int32_t *, cudaStream_t);
template void exclusive_scan<int64_t>(const int64_t *, int64_t *, int64_t, int64_t *, cudaStream_t);
template void exclusive_scan<uint32_t>(const uint32_t *, uint32_t *, int64_t, uint32_t *, cudaStream_t);

}  // namespace imq
