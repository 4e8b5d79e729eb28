// Internal declarations of the GB300 IMQ library (not part of the ABI).
//
// Geometry (paper Section 2.2, Eq. (11)-(13)): sources Y_j = (x_j, -c/2),
// targets X_i = (x_i, +c/2); multipole centres Z_B = (centre_B, -c/2) lie in
// the source plane, local centres C_B = (centre_B, +c/2) in the target plane.
//
// Expansion coefficients are stored in a parity-reduced real layout: because
// every source lies in the plane of its multipole centre and every target in
// the plane of its local centre, only the (n, m) terms with n + m even carry
// information (P_n^m(0) = 0 otherwise).  Slots run m-major: for m = 0..p, for
// n = m, m+2, ..., <= p: one real (m = 0) or a (Re, Im) pair (m > 0).
//
// Coefficients are scaled by the box side h so that FP32 stays in range:
//   multipole  Mh_n^m = M_n^m * sqrt((n+m)!(n-m)!) / h^n
//   local      Lh_n^m = L_n^m * h^n / sqrt((n+m)!(n-m)!)
// with M_n^m = sum_j u_j conj(U_n^m(Y_j - Z)) and Phi(X) = sum L_n^m conj(U_n^m(X - C)),
// U/T the regular/irregular solid harmonics U_n^m = r^n P_n^m e^{im om}/(n+m)!,
// T_n^m = (n-m)! P_n^m e^{im om}/r^{n+1}  (P_n^m without Condon-Shortley phase).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <memory>
#include <string>
#include <vector>

#include "../../include/imq.h"

namespace imq {

struct Error {
    imq_status status;
    std::string msg;
};

[[noreturn]] void fail(imq_status s, const std::string &msg);
void set_last_error(const std::string &msg);
void cuda_check(cudaError_t e, const char *what, const char *file, int line);
#define IMQ_CUDA(call) ::imq::cuda_check((call), #call, __FILE__, __LINE__)
#define IMQ_LAUNCH_CHECK() ::imq::cuda_check(cudaGetLastError(), "kernel launch", __FILE__, __LINE__)

// ---------------------------------------------------------------- device memory
// Caller-supplied allocator of plan-owned buffers (imq_options.alloc / free).
struct Allocator {
    void *(*alloc)(size_t, void *) = nullptr;
    void (*free)(void *, size_t, void *) = nullptr;
    void *ctx = nullptr;
};

// While alive, DevMem::alloc on this thread uses `a` (if it has an alloc function).
struct UseAllocator {
    const Allocator *prev;
    explicit UseAllocator(const Allocator *a);
    ~UseAllocator();
    UseAllocator(const UseAllocator &) = delete;
    UseAllocator &operator=(const UseAllocator &) = delete;
};

struct DevMem {
    void *ptr = nullptr;
    size_t bytes = 0;
    Allocator by;   // who allocated ptr (free == nullptr: cudaMalloc)
    DevMem() = default;
    DevMem(const DevMem &) = delete;
    DevMem &operator=(const DevMem &) = delete;
    DevMem(DevMem &&o) noexcept : ptr(o.ptr), bytes(o.bytes), by(o.by) { o.ptr = nullptr; o.bytes = 0; }
    DevMem &operator=(DevMem &&o) noexcept {
        release();
        ptr = o.ptr; bytes = o.bytes; by = o.by; o.ptr = nullptr; o.bytes = 0;
        return *this;
    }
    ~DevMem() { release(); }
    void alloc(size_t n);
    void release();
    template <class T> T *as() const { return static_cast<T *>(ptr); }
};

// Stream-ordered scratch (cudaMallocAsync) freed on the same stream.
struct AsyncMem {
    void *ptr = nullptr;
    cudaStream_t stream = nullptr;
    AsyncMem(size_t bytes, cudaStream_t s);
    AsyncMem(const AsyncMem &) = delete;
    AsyncMem &operator=(const AsyncMem &) = delete;
    ~AsyncMem();
    template <class T> T *as() const { return static_cast<T *>(ptr); }
};

// ---------------------------------------------------------------- layout
struct Layout {
    int p = 0;
    int parity = 0;                // 0: slots with n+m even, 1: n+m odd
    int K = 0;                     // reals per expansion
    std::vector<int> slot_n, slot_m, slot_part;   // per real slot
    std::vector<int> re_slot;      // [(p+1)*(p+1)] index n*(p+1)+m -> slot of Re part or -1
    std::vector<int> im_slot;      // same for Im part (-1 for m = 0 or odd n+m)
    void build(int p_, int parity_ = 0);
};

// Shape parameter seen by a kernel: one value, or (batched plans) one per problem
// looked up through the box's problem index.
struct ShapeC {
    double c0;
    const int32_t *box_prob;   // nullptr: every box has c0
    const double *prob_c;
#ifdef __CUDACC__
    __host__ __device__ __forceinline__ double of(int box) const { return box_prob ? prob_c[box_prob[box]] : c0; }
#endif
};

constexpr int kOffsetClasses = 40;          // V-list offsets in [-3,3]^2 minus [-1,1]^2
int offset_class(int dx, int dy);           // -1 for |dx|,|dy| <= 1 or out of range
void offset_of_class(int k, int *dx, int *dy);

// ---------------------------------------------------------------- operators (host, FP64)
// Real K x K matrices stored input-major: op[i * K + o] multiplies input slot i into output o.
void build_m2m_ops(const Layout &L, std::vector<double> &out);          // [4][K][K], quadrant q = 2*ybit + xbit
void build_l2l_ops(const Layout &L, std::vector<double> &out);          // [4][K][K]
// [40][K_in][K_out] for side h; Lo the output (local) layout, L the input (multipole) layout
void build_m2l_ops(const Layout &Lo, const Layout &L, double h, double c, std::vector<double> &out);
void p2m_coefficients(const Layout &L, std::vector<double> &coef);      // per slot: Ptilde_n^m(0)
void l2p_dz_coefficients(const Layout &Lo, std::vector<double> &coef);  // odd slots: d/dz of L2P

// ---------------------------------------------------------------- plan
struct ListCSR {
    DevMem off, items;   // int32[nbox+1], int32[total]
    int64_t total = 0;
};

struct TypedOps {        // operator set in one precision
    DevMem m2m, l2l, m2l, p2mc;
    DevMem M, L;         // expansion workspace (nbox x K), owned by the plan
    bool ready = false;
    // derivative in c (odd-parity locals): M2L even->odd, L2L odd, d/dz L2P coefficients
    DevMem m2l_odd, l2l_odd, dzc, Lodd;
    bool dz_ready = false;
    // tensor-core M2L (FP32 only): swizzled fp16 hi/lo operator images and their coefficient
    // scales, packed fp16 hi/lo multipole rows with their box scales
    DevMem m2l_img, Mpk, m2l_tmask;   // m2l_tmask: uint64 per tile, bit o = offset class o present
    DevMem m2l_order, m2l_counter;    // tiles heaviest first; the persistent kernel's work counter
    int m2l_nblk = 0;                 // operator blocks (levels, or problem-levels) in m2l_img
    bool umma = false;
};

// Additive Schwarz preconditioner over leaf neighbourhood patches (cg.cu).
struct Schwarz {
    bool ready = false;
    int nmax = 0;
    double shift = 0;
    int npatch = 0;
    DevMem patch_off;    // int32[npatch+1] offsets into patch_pts
    DevMem patch_pts;    // int32[] sorted point indices of each patch
    DevMem fac_off;      // int64[npatch] offset of each patch's factor
    DevMem factor;       // float[] or double[] column-major n x n Cholesky factors, or packed
                         // lower inverse factors (inverse)
    bool fp64 = false;
    bool inverse = false; // factor holds each patch's packed inverse factor L^{-1} (FP32, n <= 224)
    int maxn = 0;         // points of the largest patch
    DevMem pt_off;       // int32[N+1] reverse map: point -> patch slots
    DevMem pt_slot;      // int32[] patch slot (patch_off[b] + local index)
    DevMem ypatch;       // double[total slots] per-patch solutions
    int64_t total_slots = 0;
};

// A CUDA graph captured on a private stream.  begin() creates the stream and
// starts a thread-local capture; instantiate() ends it and returns the
// executable graph.  If anything throws in between, the destructor ends a
// capture still open and destroys the partial graph, the executable graph and
// the stream, so no capture is left active and nothing leaks.
struct GraphCapture {
    cudaStream_t cs = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool capturing = false;
    cudaStream_t begin();
    cudaGraphExec_t instantiate();
    GraphCapture() = default;
    GraphCapture(const GraphCapture &) = delete;
    GraphCapture &operator=(const GraphCapture &) = delete;
    ~GraphCapture();
};

// Coarse space of the two-level Schwarz preconditioner (coarse.cu): the indicator
// vectors of the largest tree boxes holding at most `cp` points (disjoint Morton
// ranges covering all points), the Galerkin matrix E = Z^T A Z and its inverse.
struct Coarse {
    bool ready = false;
    int cp = 0;          // max points per coarse box
    int nc = 0;          // coarse boxes
    DevMem cbeg;         // int32[nc + 1] Morton-order point ranges
    DevMem einv;         // double[nc * nc] E^{-1} (symmetric)
    DevMem g, cc;        // double[nc] restriction and coarse solution
    double shift = 0;    // diagonal shift that made E factorable (relative to its mean diagonal)
    bool gram_fp64 = false;   // E assembled with FP64 pairs
    int gram_mode = 0;        // imq_cg_options.coarse_gram of the last set-up
};
constexpr int kCoarseMax = 16384;   // largest coarse space (E^{-1} is nc^2 doubles)

// Streams and fork/join events of the concurrent FP32 product (per plan): the
// far-field chain runs on a highest-priority stream, the near field on a
// lowest-priority one, so free SM slots go to the latency-bound chain first.
struct AuxStream {
    cudaStream_t hi = nullptr, s = nullptr;
    cudaEvent_t fork = nullptr, xready = nullptr, mready = nullptr, join = nullptr, done = nullptr;
    void ensure();
    AuxStream() = default;
    AuxStream(const AuxStream &) = delete;
    AuxStream &operator=(const AuxStream &) = delete;
    ~AuxStream();
};

struct Plan {
    Allocator allocator;   // the caller's allocator of this plan's buffers (empty: cudaMalloc)
    int device = 0;
    int64_t N = 0;
    double c = 0, x0 = 0, y0 = 0, side = 1;
    int p = 0, leaf = 0;
    int nbox = 0, nleaf = 0, max_level = 0;
    int m2l_level_lo = 2, m2l_level_hi = 1;   // levels holding V pairs
    Layout layout;       // multipoles and value locals (n+m even)
    Layout layout_odd;   // locals of the c-derivative (n+m odd)
    int64_t n_nodes = 0; // evaluation plans: the first n_nodes points are nodes, the rest targets
    int m2l_kernel = 0;  // imq_m2l_kernel
    int algorithm = 0;   // imq_algorithm
    bool trans64 = false; // FP32 product with M2M / M2L / L2L in FP64 (imq_options.translations)
    bool trans_mixed = false;   // FP32 product with M2M / L2L in FP64, M2L on the tensor cores
    // tile shapes of the FP32 product (imq_options; 0 = default): P2P warps per CTA and
    // target chunk, tensor-core M2L pipeline stages
    int p2p_warps = 0, p2p_chunk = 0, m2l_stages = 0, m2l_split = 0;
    int tc_depth = 0;    // IMQ_ALG_TREECODE: depth of the uniform partition (paper's L + 1)
    int nprob = 1;       // batched plans: independent problems sharing one flattened tree
    DevMem box_prob;     // int32[nbox] problem of each box (batched plans only)
    DevMem prob_c;       // double[nprob] shape of each problem (batched plans only)
    DevMem pt_prob;      // int32[N] problem of each sorted point (batched plans only)
    std::vector<int64_t> prob_off;   // host: sorted point offsets of the problems [nprob+1]
    std::vector<double> h_prob_c;
    DevMem box_opslot;   // int32[nbox] M2L operator slot of each box (batched plans only)
    std::vector<double2> h_slot_hc;  // (h, c) of each M2L operator slot (batched plans)
    ShapeC shape() const {
        return ShapeC{c, nprob > 1 ? box_prob.as<int32_t>() : nullptr, nprob > 1 ? prob_c.as<double>() : nullptr};
    }
    std::vector<int> level_start;              // boxes of level l: [level_start[l], level_start[l+1])
    std::vector<int> parent_start;             // internal boxes of level l: parents[parent_start[l] ..]
    DevMem parents;                            // int32: internal boxes, level by level, in box order
    // tree, device
    DevMem codes;      // uint32[N] sorted
    DevMem perm;       // int64[N] sorted -> input
    DevMem level, prefix, begin, end, parent, child;   // per box (child: int32[4*nbox])
    DevMem centre;     // double2[nbox]
    DevMem leaves;     // int32[nleaf]
    ListCSR U, V, W, X;
    DevMem colleagues; // int32[9*nbox]
    DevMem vtab;       // int32[40*nbox] V source per offset class, -1 if none
    DevMem m2l_tiles;  // int4[n_m2l_tiles]: (level - m2l_level_lo, first index into m2l_tbox, boxes)
    DevMem m2l_tbox;   // int32[]: boxes of the M2L levels grouped by (level, quadrant)
    int n_m2l_tiles = 0;
    DevMem xboxes;     // int32[nxbox] boxes whose X list is not empty
    DevMem xcum;       // int32[n_x]: per box list, exclusive prefix of source counts
    DevMem xtot;       // int32[nbox] total X-list source points of a box
    int nxbox = 0;
    DevMem utot;       // int32[nbox] total U-list source points of a leaf
    DevMem ucum;       // int32[n_u]: per leaf list, exclusive prefix of source counts
    DevMem uoff;       // float2[n_u]: (centre_target - centre_source)
    // points, device, sorted order
    DevMem pos;        // double2[N]
    DevMem loc;        // float2[N]  offset from the leaf centre
    DevMem rec4;       // float4[N]  P2P source records (x, y, u0, u1) of the current product
    DevMem rec4b;      // float4[N]  (u2, u3, 0, 0) for three or four right-hand sides at once
    DevMem p2p_order;  // int32[nleaf] leaves by P2P pair count, most first
    DevMem p2p_counter;// int32 work counter of the persistent P2P kernel
    DevMem leaf_of;    // int32[N]
    // far field (FP32, fixed p): M2P items (leaf, W source, first point, partial offset)
    DevMem m2p_items;  // int4[n_m2p_items]
    DevMem wbase;      // int32[nleaf] offset of each leaf's M2P partial sums
    DevMem wpart;      // float[32 * n_m2p_items] partial sums, W-entry major then 32-point chunk
    int n_m2p_items = -1;   // -1: not built yet
    DevMem near;       // float[nrhs * N] near-field (P2P) sums of the current FP32 product
    AuxStream aux;     // the P2P / M2P stream of the concurrent FP32 product
    // operators
    std::vector<double> h_m2m, h_l2l, h_m2l, h_p2mc;   // FP64 host copies (h_m2l: [lev][40][K][K])
    std::vector<double> h_m2l_odd, h_l2l_odd, h_dzc;   // derivative path ([lev][40][K][Ko], [4][Ko][Ko])
    TypedOps ops32, ops64;
    Schwarz schwarz;
    Coarse coarse;
    // statistics
    int64_t p2p_pairs = 0, m2l_pairs = 0;
    int64_t device_bytes() const;
    // CUDA graph of the FP32 product (gather, expansions, near field, scatter) on the plan's own
    // input / output buffers, replayed by calls that synchronise anyway (host buffers); declared
    // last so that it is released before the streams and buffers it refers to
    struct ProductGraph {
        std::unique_ptr<GraphCapture> cap;
        cudaGraphExec_t exec = nullptr;
        int nrhs = 0;
        DevMem in, out, us, bs;
    } pgraph;
};

// Optional per-phase timing of a product with CUDA events on the launching stream.
enum Phase { kPhGather = 0, kPhP2M, kPhM2M, kPhM2L, kPhP2L, kPhL2L, kPhFar, kPhP2P, kPhScatter, kNumPhases };
struct PhaseTimer {
    struct Rec { int phase; cudaEvent_t a, b; };
    std::vector<Rec> recs;
    int launches = 0;
    void start(int phase, cudaStream_t s);
    void stop(cudaStream_t s);
    void collect(float *ms, int n);   // synchronises on the last event
    ~PhaseTimer();
};

// tree.cu
void build_tree(Plan &P, const double *d_points, cudaStream_t s, bool check_dups);
// expansions.cu
void ensure_ops(Plan &P, bool fp64, cudaStream_t s);
template <class T>
int fmm_apply(Plan &P, const T *u_sorted, T *b_sorted, int nrhs, cudaStream_t s, PhaseTimer *tm = nullptr);
template <class Tin, class T>
void gather_sorted(const Plan &P, const Tin *v, T *us, int nrhs, cudaStream_t s);
template <class T, class Tout>
void scatter_sorted(const Plan &P, const T *bs, Tout *out, int nrhs, cudaStream_t s);
// cg.cu
void cg_solve(Plan &P, const double *f_dev, double *x_dev, int nrhs, const imq_cg_options &o, Plan *RP,
              imq_cg_info *info, cudaStream_t s);
double device_dot(const double *a, const double *b, int64_t n, cudaStream_t s);   // deterministic, synchronises
void schwarz_setup(Plan &P, int nmax, double shift, bool fp64, cudaStream_t s);
int schwarz_nmax_of(const imq_cg_options &o);   // the patch size a solve uses (0: 224 FP32, 160 FP64)
// z = M r; Sv: per-solve state whose done flag skips the work (nullptr: always run)
void schwarz_apply(const Plan &P, const Schwarz &Z, const double *r, double *z, double c, int64_t n, const void *Sv,
                   cudaStream_t s);
// coarse.cu: two-level Schwarz coarse space (single plans)
void coarse_setup(Plan &P, int cp, int gram, cudaStream_t s);   // gram: imq_cg_options.coarse_gram
// g = Z^T (r - b), b = b32 (FP32) or b64 (FP64) or none: one block per coarse box, fixed-order FP64 sums
void coarse_restrict(const Plan &P, const double *r, const float *b32, const double *b64, const int *done,
                     cudaStream_t s);
// cc = E^{-1} g
void coarse_solve(const Plan &P, const int *done, cudaStream_t s);
// z = y + Z cc (y may be null: z = Z cc)
void coarse_prolong(const Plan &P, const double *y, double *z, const int *done, cudaStream_t s);
// cg_batched.cu
// rel_out / iters_out: host [nrhs][nprob] or nullptr
void cg_solve_batched(Plan &P, const double *f_dev, double *x_dev, int nrhs, const imq_cg_options &o,
                      imq_cg_info *info, double *rel_out, int32_t *iters_out, cudaStream_t s);
// m2l.cu
int m2l_tiled_rows(int K);
void m2l_tiled_launch(const Plan &P, const float *M, float *L, const float *ops, cudaStream_t s, int Kout = 0);
// expansions.cu building blocks reused by the derivative path
template <class T>
void upward_launch(Plan &P, const T *u, T *M, const T *coef, const T *m2m, cudaStream_t s, int *launches);
template <class T>
void l2l_launch(Plan &P, T *L, const T *op, int K, cudaStream_t s, int *launches);
template <class T>
void m2l_direct_launch(Plan &P, const T *M, T *L, const T *ops, int Kin, int Kout, cudaStream_t s, int *launches);
template <class T>
void p2l_odd_launch(Plan &P, const T *u, T *Lodd, cudaStream_t s);
template <class T>
void p2p_apply(Plan &P, const T *u, T *bs, cudaStream_t s);
// dz.cu: b = (dA/dc) u in Morton order
template <class T>
int fmm_apply_dz(Plan &P, const T *u_sorted, T *b_sorted, int nrhs, cudaStream_t s);
void build_m2l_tiles(Plan &P, cudaStream_t s);
// p2m.cu: P2M for a compile-time order (FP32)
bool p2m_fixed_p_supported(int p);
// Mpk (may be null): also write the scaled fp16 hi / lo rows [hi | pad to KP | lo | pad] of the tensor-core
// M2L, with the row's inverse scale in its padding
void p2m_fixed_p_launch(const Plan &P, const float *u, float *M, const float *coef, cudaStream_t s,
                        float *Mpk = nullptr, int KP = 0);
void p2l_fixed_p_prepare(cudaStream_t s);
void p2l_fixed_p_launch(const Plan &P, const float *u, float *L, cudaStream_t s);
// far.cu: L2P + M2P for a compile-time order (FP32)
bool far_fixed_p_supported(int p);
void far_fixed_p_prepare(cudaStream_t s);
void ensure_m2p_items(Plan &P, cudaStream_t s);   // host sync: call outside stream capture
void far_m2p_launch(Plan &P, const float *M, cudaStream_t s);   // W-list M2P partial sums
// b = L2P + the leaf's M2P partial sums (+ near[i] if near is not null)
void far_l2p_launch(Plan &P, const float *L, const float *coef, const float *near, float *b, cudaStream_t s);
// p2p.cu: near[i] = the P2P sum of point i (FP32, stored, not added)
// u, near: [nrhs][N]; one kernel value per pair serves up to four right-hand sides
void p2p_near_f32(Plan &P, const float *u, float *near, int nrhs, cudaStream_t s);
// m2l_umma.cu: tensor-core M2L over the same tiles (value path, FP32 in and out)
bool m2l_umma_supported(int K, int Kout);
void m2l_umma_prepare(const Plan &P, const float *ops, int nblk, int Kout, DevMem &img, DevMem &Mpk, DevMem &tmask,
                      DevMem &order, DevMem &counter, cudaStream_t s);
// packed: Mpk already holds the fp16 hi / lo rows of every box (written by P2M and M2M)
void m2l_umma_launch(const Plan &P, const float *M, float *L, const TypedOps &O, int Kout, cudaStream_t s,
                     bool packed = false);
int m2l_umma_kp(int K);   // padded length KP of each half (hi, lo) of a packed row
int m2l_umma_max_stages(int K, int Kout);   // pipeline stages that fit in shared memory
int m2l_umma_min_stages();                  // fewest pipeline stages the kernel runs with
int m2l_default_split(int ntiles);          // CTAs per M2L tile when the plan does not choose
// batch.cu
template <class T>
void generate_m2l_ops(const Layout &Lo, const Layout &Li, const std::vector<double2> &slot_hc, int Kp, DevMem &dst,
                      cudaStream_t s);
void build_batched_plan(Plan &P, const double *d_points, const std::vector<int64_t> &offs,
                        const std::vector<double> &cs, bool dups, cudaStream_t s);
// dense.cu
void dense_matvec_dev(const double *d_points, int64_t N, double c, const void *d_v, void *d_out,
                      int nrhs, imq_dtype dt, cudaStream_t s);
// FP64 dense product, kernel launch only (no host synchronisation; graph-capturable)
void dense_f64_async(const double *d_points, int64_t N, double c, const double *d_v, double *d_out, cudaStream_t s);
// FP64 dense product of a batched plan's block-diagonal matrix, in Morton order:
// problem b owns [d_off[b], d_off[b+1]) with shape d_prob_c[b] (kernel launch only)
void dense_f64_seg_async(const double *d_points, const int64_t *d_off, int nprob, const double *d_prob_c,
                         const double *d_v, double *d_out, int64_t N, cudaStream_t s);
// api.cu helpers
void check_device();
template <class F>
imq_status guarded_call(F &&f) {   // run f, translate exceptions into a status and the thread's last error
    try {
        f();
        set_last_error("");
        return IMQ_OK;
    } catch (const Error &e) {
        set_last_error(e.msg);
        return e.status;
    } catch (...) {
        set_last_error("unexpected internal error");
        return IMQ_CUDA_ERROR;
    }
}

// Measured choice of p and leaf size (autotune.cu); arguments already checked.  v: the caller's
// test vectors (float[nrhs][N], host or device) or nullptr for SplitMix64 values.
void autotune(const double *points, const int64_t *offsets, int nprob, const double *cvals, double target,
              const int32_t *p_cand, int n_p, const int32_t *leaf_cand, int n_leaf, int nrhs, const float *v,
              const imq_options *opt, cudaStream_t s, imq_tune_result *out);

}  // namespace imq
