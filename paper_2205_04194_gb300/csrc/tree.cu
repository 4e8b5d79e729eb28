// GPU quadtree build: Morton codes, stable radix sort, adaptive boxes and the
// U/V/W/X interaction lists.
//
// Paper Section 2.2: a square D containing the points is partitioned into
// 2^{l+1} x 2^{l+1} blocks per level, children by bisecting edges; the
// well-separated sets S_p and the not-well-separated sets NS_p of Algorithm 1
// decide which block pairs use the expansion and which are summed directly.
// This builder generalises the partition to an adaptive tree:
//   * D = (x0, y0, S), default the exact bounding square of the points;
//   * q = floor(((x - x0) / S) * 65536) in FP64 with each operation rounded as
//     written (__dsub_rn / __ddiv_rn / __dmul_rn: no contraction), clamped to
//     [0, 65535]; Morton code = x bits at even, y bits at odd positions;
//   * stable LSD radix sort of (code, input index), 4 passes of 8 bits;
//   * a box (level, prefix) is split into its non-empty quadrants while it
//     holds more than `leaf` points and level < 16; boxes are numbered in
//     (level, prefix) order;
//   * colleagues: same-level adjacent boxes; V: children of the parent's
//     colleagues not adjacent to the box (the paper's S_p, M2L); U: adjacent
//     leaves of any level (NS_p, direct sum); W: descendants of colleagues that
//     are not adjacent but whose parent is (M2P); X: the transpose of W (P2L).
//     Adjacent = closed squares intersect.  Each list is sorted by box number.
#include <algorithm>
#include <cstring>

#include "imq_internal.h"
#include "ptx.cuh"
#include "util.cuh"

namespace imq {
namespace {

constexpr int kStack = 96;

struct Box4 {
    double x, y, z, w;
};

__device__ __forceinline__ uint32_t part1by1(uint32_t x) {
    x &= 0xFFFFu;
    x = (x | (x << 8)) & 0x00FF00FFu;
    x = (x | (x << 4)) & 0x0F0F0F0Fu;
    x = (x | (x << 2)) & 0x33333333u;
    x = (x | (x << 1)) & 0x55555555u;
    return x;
}

__device__ __forceinline__ uint32_t compact1by1(uint32_t x) {
    x &= 0x55555555u;
    x = (x | (x >> 1)) & 0x33333333u;
    x = (x | (x >> 2)) & 0x0F0F0F0Fu;
    x = (x | (x >> 4)) & 0x00FF00FFu;
    x = (x | (x >> 8)) & 0x0000FFFFu;
    return x;
}

// ------------------------------------------------------------------ bbox / codes
__global__ void bbox_partial(const double *__restrict__ pts, int64_t n, Box4 *part, int *err) {
    __shared__ double s[4][256];
    double mnx = INFINITY, mny = INFINITY, mxx = -INFINITY, mxy = -INFINITY;
    bool bad = false;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double x = pts[2 * i], y = pts[2 * i + 1];
        if (!isfinite(x) || !isfinite(y)) bad = true;
        mnx = fmin(mnx, x); mny = fmin(mny, y); mxx = fmax(mxx, x); mxy = fmax(mxy, y);
    }
    if (bad) set_error(err, kErrNonFinite);
    s[0][threadIdx.x] = mnx; s[1][threadIdx.x] = mny; s[2][threadIdx.x] = mxx; s[3][threadIdx.x] = mxy;
    __syncthreads();
    for (int off = 128; off > 0; off >>= 1) {
        if (threadIdx.x < off) {
            s[0][threadIdx.x] = fmin(s[0][threadIdx.x], s[0][threadIdx.x + off]);
            s[1][threadIdx.x] = fmin(s[1][threadIdx.x], s[1][threadIdx.x + off]);
            s[2][threadIdx.x] = fmax(s[2][threadIdx.x], s[2][threadIdx.x + off]);
            s[3][threadIdx.x] = fmax(s[3][threadIdx.x], s[3][threadIdx.x + off]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = Box4{s[0][0], s[1][0], s[2][0], s[3][0]};
}

__global__ void morton_codes(const double *__restrict__ pts, int64_t n, double x0, double y0, double S,
                             uint32_t *__restrict__ codes, int32_t *__restrict__ idx) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double tx = __dmul_rn(__ddiv_rn(__dsub_rn(pts[2 * i], x0), S), 65536.0);
    double ty = __dmul_rn(__ddiv_rn(__dsub_rn(pts[2 * i + 1], y0), S), 65536.0);
    double fx = floor(tx), fy = floor(ty);
    if (!(fx >= 0.0)) fx = 0.0;
    if (!(fy >= 0.0)) fy = 0.0;
    if (fx > 65535.0) fx = 65535.0;
    if (fy > 65535.0) fy = 65535.0;
    codes[i] = part1by1((uint32_t)fx) | (part1by1((uint32_t)fy) << 1);
    idx[i] = (int32_t)i;
}

// ------------------------------------------------------------------ radix sort
constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortIter = 16;
constexpr int kSortTile = kSortThreads * kSortIter;   // 4096

__global__ void __launch_bounds__(kSortThreads) radix_hist(const uint32_t *__restrict__ keys, int64_t n, int shift,
                                                           uint32_t *__restrict__ counts, int ntiles) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int k = threadIdx.x; k < kSortTile; k += kSortThreads) {
        const int64_t e = base + k;
        if (e < n) atomicAdd(&h[(keys[e] >> shift) & 0xFFu], 1u);
    }
    __syncthreads();
    counts[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

__global__ void __launch_bounds__(kSortThreads) radix_scatter(const uint32_t *__restrict__ kin,
                                                              const int32_t *__restrict__ vin,
                                                              uint32_t *__restrict__ kout, int32_t *__restrict__ vout,
                                                              int64_t n, int shift, const uint32_t *__restrict__ offs,
                                                              int ntiles) {
    __shared__ uint32_t wc[kSortWarps][256];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int k = threadIdx.x; k < kSortWarps * 256; k += kSortThreads) (&wc[0][0])[k] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortTile + (int64_t)w * (32 * kSortIter);
    const uint32_t lt = (1u << lane) - 1u;
    for (int it = 0; it < kSortIter; ++it) {
        const int64_t e = base + it * 32 + lane;
        const bool valid = e < n;
        const uint32_t d = valid ? ((kin[e] >> shift) & 0xFFu) : (0x100u + lane);
        const uint32_t peers = __match_any_sync(0xFFFFFFFFu, d);
        if (valid && (peers & lt) == 0) wc[w][d] += __popc(peers);
    }
    __syncthreads();
    {
        const int d = threadIdx.x;   // 256 threads = 256 digits
        uint32_t run = offs[(int64_t)d * ntiles + blockIdx.x];
        for (int ww = 0; ww < kSortWarps; ++ww) {
            const uint32_t t = wc[ww][d];
            wc[ww][d] = run;
            run += t;
        }
    }
    __syncthreads();
    for (int it = 0; it < kSortIter; ++it) {
        const int64_t e = base + it * 32 + lane;
        const bool valid = e < n;
        const uint32_t key = valid ? kin[e] : 0u;
        const uint32_t d = valid ? ((key >> shift) & 0xFFu) : (0x100u + lane);
        const uint32_t peers = __match_any_sync(0xFFFFFFFFu, d);
        uint32_t basepos = 0;
        if (valid) basepos = wc[w][d];
        __syncwarp();
        if (valid) {
            const uint32_t pos = basepos + __popc(peers & lt);
            kout[pos] = key;
            vout[pos] = vin[e];
            if ((peers & lt) == 0) wc[w][d] = basepos + __popc(peers);
        }
        __syncwarp();
    }
}

// ------------------------------------------------------------------ boxes
__device__ int lower_bound_u32(const uint32_t *a, int lo, int hi, uint32_t key) {
    while (lo < hi) {
        const int mid = lo + ((hi - lo) >> 1);
        if (a[mid] < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// depth > 0: uniform partition (the paper's blocks), split every box above that depth
__global__ void split_count(int lb, int nl, int lev, int leaf, int depth, const uint32_t *__restrict__ codes,
                            const int32_t *__restrict__ begin, const int32_t *__restrict__ end,
                            const uint32_t *__restrict__ prefix, int32_t *__restrict__ qb, int32_t *__restrict__ nchild) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nl) return;
    const int b = lb + i;
    const int bg = begin[b], en = end[b];
    int cnt = 0;
    if (depth > 0 ? lev < depth : (en - bg > leaf && lev < IMQ_MAX_LEVEL)) {
        const int shift = 32 - 2 * (lev + 1);
        const uint32_t P = prefix[b];
        qb[5 * i] = bg;
        qb[5 * i + 4] = en;
        for (int q = 1; q < 4; ++q) qb[5 * i + q] = lower_bound_u32(codes, bg, en, (4u * P + q) << shift);
        for (int q = 0; q < 4; ++q) cnt += qb[5 * i + q + 1] > qb[5 * i + q];
    }
    nchild[i] = cnt;
}

__global__ void make_children(int lb, int nl, int lev, int nb0, const int32_t *__restrict__ qb,
                              const int32_t *__restrict__ nchild, const int32_t *__restrict__ cbase,
                              const uint32_t *__restrict__ prefix, int32_t *level, uint32_t *pref, int32_t *begin,
                              int32_t *end, int32_t *parent, int32_t *child) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nl || nchild[i] == 0) return;
    const int b = lb + i;
    int idx = nb0 + cbase[i];
    const uint32_t P = prefix[b];
    for (int q = 0; q < 4; ++q) {
        const int lo = qb[5 * i + q], hi = qb[5 * i + q + 1];
        if (hi > lo) {
            level[idx] = lev + 1;
            pref[idx] = 4u * P + q;
            begin[idx] = lo;
            end[idx] = hi;
            parent[idx] = b;
            child[4 * idx] = child[4 * idx + 1] = child[4 * idx + 2] = child[4 * idx + 3] = -1;
            child[4 * b + q] = idx;
            ++idx;
        }
    }
}

struct BoxView {
    const int32_t *level;
    const int2 *ixy;
    const int32_t *child;
    const int32_t *parent;
    const int32_t *col;    // [nbox][9]
    const int8_t *isleaf;
    __device__ __forceinline__ bool adjacent(int a, int b) const {
        const int la = level[a], lbv = level[b];
        const int L = max(la, lbv);
        const int sa = L - la, sb = L - lbv;
        const int2 A = ixy[a], B = ixy[b];
        const int ax0 = A.x << sa, ax1 = (A.x + 1) << sa, ay0 = A.y << sa, ay1 = (A.y + 1) << sa;
        const int bx0 = B.x << sb, bx1 = (B.x + 1) << sb, by0 = B.y << sb, by1 = (B.y + 1) << sb;
        return ax0 <= bx1 && bx0 <= ax1 && ay0 <= by1 && by0 <= ay1;
    }
};

__global__ void box_geometry(int nbox, const int32_t *__restrict__ level, const uint32_t *__restrict__ prefix,
                             const int32_t *__restrict__ child, double x0, double y0, double S, int2 *ixy,
                             double2 *centre, int8_t *isleaf) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbox) return;
    const uint32_t P = prefix[b];
    const int ix = (int)compact1by1(P), iy = (int)compact1by1(P >> 1);
    ixy[b] = make_int2(ix, iy);
    const double h = S / (double)(1 << level[b]);
    centre[b] = make_double2(__dadd_rn(x0, __dmul_rn((double)ix + 0.5, h)), __dadd_rn(y0, __dmul_rn((double)iy + 0.5, h)));
    isleaf[b] = (child[4 * b] < 0 && child[4 * b + 1] < 0 && child[4 * b + 2] < 0 && child[4 * b + 3] < 0) ? 1 : 0;
}

__global__ void colleagues_level(int lb, int nl, BoxView T, int32_t *col, int32_t *vcount, int *err) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nl) return;
    const int b = lb + i;
    const int pb = T.parent[b];
    int nc = 0, nv = 0;
    for (int k = 0; k < 9; ++k) {
        const int q = col[9 * pb + k];
        if (q < 0) break;
        for (int c4 = 0; c4 < 4; ++c4) {
            const int d = T.child[4 * q + c4];
            if (d < 0) continue;
            if (T.adjacent(d, b)) {
                if (nc < 9) col[9 * b + nc] = d;
                else set_error(err, kErrListOverflow);
                ++nc;
            } else {
                ++nv;
            }
        }
    }
    for (int k = nc; k < 9; ++k) col[9 * b + k] = -1;
    vcount[b] = nv;
}

__global__ void v_fill(int nbox, BoxView T, const int32_t *__restrict__ voff, int32_t *__restrict__ vitems) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbox || b == 0) return;
    const int pb = T.parent[b];
    int w = voff[b];
    for (int k = 0; k < 9; ++k) {
        const int q = T.col[9 * pb + k];
        if (q < 0) break;
        for (int c4 = 0; c4 < 4; ++c4) {
            const int d = T.child[4 * q + c4];
            if (d >= 0 && !T.adjacent(d, b)) vitems[w++] = d;
        }
    }
}

__device__ void insertion_sort(int32_t *a, int n) {
    for (int i = 1; i < n; ++i) {
        const int32_t v = a[i];
        int j = i - 1;
        while (j >= 0 && a[j] > v) { a[j + 1] = a[j]; --j; }
        a[j + 1] = v;
    }
}

// U and W of leaf b.  mode 0: count into ucnt/wcnt; mode 1: write at uoff/woff.
__global__ void uw_lists(int nbox, BoxView T, int mode, int32_t *ucnt, int32_t *wcnt, const int32_t *uoffs,
                         const int32_t *woffs, int32_t *uitems, int32_t *witems, int *err) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbox || !T.isleaf[b]) return;
    int stack[kStack];
    int nu = 0, nw = 0;
    const int ub = mode ? uoffs[b] : 0, wb = mode ? woffs[b] : 0;
    // coarser adjacent leaves: leaf colleagues of the ancestors (root level first)
    {
        int chain[IMQ_MAX_LEVEL + 1];
        int nchain = 0;
        for (int a = T.parent[b]; a >= 0; a = T.parent[a]) chain[nchain++] = a;
        for (int k = nchain - 1; k >= 0; --k) {
            const int a = chain[k];
            for (int j = 0; j < 9; ++j) {
                const int q = T.col[9 * a + j];
                if (q < 0) break;
                if (T.isleaf[q] && T.adjacent(q, b)) {
                    if (mode) uitems[ub + nu] = q;
                    ++nu;
                }
            }
        }
    }
    const int ufine = nu;
    // same-level and finer adjacent leaves: descend from the colleagues
    int sp = 0;
    for (int j = 8; j >= 0; --j) {
        const int q = T.col[9 * b + j];
        if (q >= 0) stack[sp++] = q;
    }
    while (sp > 0) {
        const int q = stack[--sp];
        if (T.isleaf[q]) {
            if (mode) uitems[ub + nu] = q;
            ++nu;
        } else {
            for (int c4 = 3; c4 >= 0; --c4) {
                const int d = T.child[4 * q + c4];
                if (d >= 0 && T.adjacent(d, b)) {
                    if (sp < kStack) stack[sp++] = d;
                    else set_error(err, kErrStackOverflow);
                }
            }
        }
    }
    // W: children of (descendants of) colleagues that are not adjacent, parent adjacent
    sp = 0;
    for (int j = 8; j >= 0; --j) {
        const int q = T.col[9 * b + j];
        if (q >= 0 && q != b && !T.isleaf[q]) stack[sp++] = q;
    }
    while (sp > 0) {
        const int q = stack[--sp];
        for (int c4 = 3; c4 >= 0; --c4) {
            const int d = T.child[4 * q + c4];
            if (d < 0) continue;
            if (T.adjacent(d, b)) {
                if (!T.isleaf[d]) {
                    if (sp < kStack) stack[sp++] = d;
                    else set_error(err, kErrStackOverflow);
                }
            } else {
                if (mode) witems[wb + nw] = d;
                ++nw;
            }
        }
    }
    if (mode) {
        insertion_sort(uitems + ub + ufine, nu - ufine);
        insertion_sort(witems + wb, nw);
    } else {
        ucnt[b] = nu;
        wcnt[b] = nw;
    }
}

__global__ void x_count(int nbox, const int8_t *isleaf, const int32_t *woff, const int32_t *witems, int32_t *xcnt) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbox || !isleaf[b]) return;
    for (int k = woff[b]; k < woff[b + 1]; ++k) atomicAdd(&xcnt[witems[k]], 1);
}

__global__ void x_fill(int nbox, const int8_t *isleaf, const int32_t *woff, const int32_t *witems,
                       const int32_t *xoff, int32_t *cursor, int32_t *xitems) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbox || !isleaf[b]) return;
    for (int k = woff[b]; k < woff[b + 1]; ++k) {
        const int d = witems[k];
        xitems[xoff[d] + atomicAdd(&cursor[d], 1)] = b;
    }
}

__global__ void sort_segments(int nbox, const int32_t *off, int32_t *items) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbox) return;
    insertion_sort(items + off[b], off[b + 1] - off[b]);
}

// ------------------------------------------------------------------ per point / per list auxiliaries
__global__ void gather_points(const double *__restrict__ pts, const int32_t *__restrict__ perm, int64_t n,
                              double2 *__restrict__ pos) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) {
        const int64_t j = perm[i];
        pos[i] = make_double2(pts[2 * j], pts[2 * j + 1]);
    }
}

__global__ void leaf_points(int nbox, const int8_t *isleaf, const int32_t *begin, const int32_t *end,
                            const double2 *centre, const double2 *pos, int32_t *leaf_of, float2 *loc) {
    const int b = blockIdx.x;
    if (b >= nbox || !isleaf[b]) return;
    const double2 cb = centre[b];
    for (int i = begin[b] + threadIdx.x; i < end[b]; i += blockDim.x) {
        leaf_of[i] = b;
        const double2 p = pos[i];
        loc[i] = make_float2((float)(p.x - cb.x), (float)(p.y - cb.y));
    }
}

__global__ void dup_check(int64_t n, const uint32_t *codes, const double2 *pos, int *err) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t ci = codes[i];
    const double2 pi = pos[i];
    for (int64_t j = i + 1; j < n && codes[j] == ci; ++j) {
        const double2 pj = pos[j];
        if (pj.x == pi.x && pj.y == pi.y) set_error(err, kErrDuplicate);
    }
}

__global__ void u_aux(int nbox, const int8_t *isleaf, const int32_t *begin, const int32_t *end,
                      const double2 *centre, const int32_t *uoff, const int32_t *uitems, int32_t *ucum,
                      int32_t *utot, float2 *udelta, unsigned long long *pairs) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbox) return;
    if (!isleaf[b]) { utot[b] = 0; return; }
    const double2 cb = centre[b];
    int run = 0;
    for (int k = uoff[b]; k < uoff[b + 1]; ++k) {
        const int s = uitems[k];
        ucum[k] = run;
        run += end[s] - begin[s];
        const double2 cs = centre[s];
        udelta[k] = make_float2((float)(cb.x - cs.x), (float)(cb.y - cs.y));
    }
    utot[b] = run;
    atomicAdd(pairs, (unsigned long long)run * (unsigned long long)(end[b] - begin[b]));
}

// per X entry: exclusive prefix of source points within the box's list; per box: total
__global__ void x_aux(int nbox, const int32_t *begin, const int32_t *end, const int32_t *xoff,
                      const int32_t *xitems, int32_t *xcum, int32_t *xtot) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbox) return;
    int run = 0;
    for (int k = xoff[b]; k < xoff[b + 1]; ++k) {
        xcum[k] = run;
        run += end[xitems[k]] - begin[xitems[k]];
    }
    xtot[b] = run;
}

__global__ void v_table(int nbox, const int2 *ixy, const int32_t *voff, const int32_t *vitems, int32_t *vtab) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbox) return;
    for (int k = 0; k < kOffsetClasses; ++k) vtab[(int64_t)kOffsetClasses * b + k] = -1;
    const int2 B = ixy[b];
    for (int k = voff[b]; k < voff[b + 1]; ++k) {
        const int s = vitems[k];
        const int dx = ixy[s].x - B.x, dy = ixy[s].y - B.y;
        // class numbering of offset_class(): row-major over [-3,3]^2 skipping [-1,1]^2
        int cls = -1, k2 = 0;
        for (int a = -3; a <= 3 && cls < 0; ++a)
            for (int c = -3; c <= 3; ++c) {
                if (a >= -1 && a <= 1 && c >= -1 && c <= 1) continue;
                if (a == dx && c == dy) { cls = k2; break; }
                ++k2;
            }
        if (cls >= 0) vtab[(int64_t)kOffsetClasses * b + cls] = s;
    }
}

template <class T>
struct DVec {
    DevMem m;
    size_t n = 0, cap = 0;
    T *ptr() const { return m.as<T>(); }
    void reserve(size_t c, cudaStream_t s) {
        if (c <= cap) return;
        size_t nc = std::max(c, cap * 2);
        DevMem nm;
        nm.alloc(nc * sizeof(T));
        if (n) IMQ_CUDA(cudaMemcpyAsync(nm.ptr, m.ptr, n * sizeof(T), cudaMemcpyDeviceToDevice, s));
        IMQ_CUDA(cudaStreamSynchronize(s));
        m = std::move(nm);
        cap = nc;
    }
};

template <class T>
void shrink_into(DevMem &dst, const DVec<T> &v, cudaStream_t s) {
    dst.alloc(std::max<size_t>(v.n, 1) * sizeof(T));
    if (v.n) IMQ_CUDA(cudaMemcpyAsync(dst.ptr, v.ptr(), v.n * sizeof(T), cudaMemcpyDeviceToDevice, s));
}

int read_i32(const int32_t *d, cudaStream_t s) {
    int32_t h = 0;
    IMQ_CUDA(cudaMemcpyAsync(&h, d, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    IMQ_CUDA(cudaStreamSynchronize(s));
    return h;
}

}  // namespace

int offset_class(int dx, int dy) {
    if (dx < -3 || dx > 3 || dy < -3 || dy > 3) return -1;
    if (dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1) return -1;
    int k = 0;
    for (int a = -3; a <= 3; ++a)
        for (int b = -3; b <= 3; ++b) {
            if (a >= -1 && a <= 1 && b >= -1 && b <= 1) continue;
            if (a == dx && b == dy) return k;
            ++k;
        }
    return -1;
}

void offset_of_class(int k, int *dx, int *dy) {
    int c = 0;
    for (int a = -3; a <= 3; ++a)
        for (int b = -3; b <= 3; ++b) {
            if (a >= -1 && a <= 1 && b >= -1 && b <= 1) continue;
            if (c == k) { *dx = a; *dy = b; return; }
            ++c;
        }
    *dx = *dy = 0;
}

// The paper's Algorithm 1 on the uniform partition: the far field of a target
// block at level l comes from the blocks of S_p, the children of its parent's
// neighbours that are not adjacent to it -- the V list of its ancestor at that
// level -- evaluated at the targets themselves (M2P).  The W list of each leaf
// becomes the union of the V lists of the leaf and of its ancestors (coarsest
// level first), and the V lists are emptied so that no M2L / L2L work is done.
void treecode_lists(Plan &P, cudaStream_t s) {
    const int nb = P.nbox;
    std::vector<int32_t> voff(nb + 1), par(nb), lev(nb), wcnt(nb, 0);
    IMQ_CUDA(cudaMemcpyAsync(voff.data(), P.V.off.ptr, 4 * (size_t)(nb + 1), cudaMemcpyDeviceToHost, s));
    IMQ_CUDA(cudaMemcpyAsync(par.data(), P.parent.ptr, 4 * (size_t)nb, cudaMemcpyDeviceToHost, s));
    IMQ_CUDA(cudaMemcpyAsync(lev.data(), P.level.ptr, 4 * (size_t)nb, cudaMemcpyDeviceToHost, s));
    std::vector<int32_t> vitems(std::max<int64_t>(1, P.V.total));
    if (P.V.total > 0)
        IMQ_CUDA(cudaMemcpyAsync(vitems.data(), P.V.items.ptr, 4 * (size_t)P.V.total, cudaMemcpyDeviceToHost, s));
    std::vector<int32_t> leaves(std::max(1, P.nleaf));
    IMQ_CUDA(cudaMemcpyAsync(leaves.data(), P.leaves.ptr, 4 * (size_t)P.nleaf, cudaMemcpyDeviceToHost, s));
    IMQ_CUDA(cudaStreamSynchronize(s));
    std::vector<std::vector<int32_t>> T(nb);
    for (int k = 0; k < P.nleaf; ++k) {
        const int b = leaves[k];
        std::vector<int32_t> chain;
        for (int a = b; a >= 0; a = par[a]) chain.push_back(a);
        for (auto it = chain.rbegin(); it != chain.rend(); ++it)
            for (int e = voff[*it]; e < voff[*it + 1]; ++e) T[b].push_back(vitems[e]);
    }
    std::vector<int32_t> toff(nb + 1, 0), titems;
    for (int b = 0; b < nb; ++b) {
        toff[b + 1] = toff[b] + (int32_t)T[b].size();
        titems.insert(titems.end(), T[b].begin(), T[b].end());
    }
    P.W.off.alloc(4 * (size_t)(nb + 1));
    P.W.items.alloc(4 * std::max<size_t>(1, titems.size()));
    P.W.total = (int64_t)titems.size();
    IMQ_CUDA(cudaMemcpyAsync(P.W.off.ptr, toff.data(), 4 * (size_t)(nb + 1), cudaMemcpyHostToDevice, s));
    if (!titems.empty())
        IMQ_CUDA(cudaMemcpyAsync(P.W.items.ptr, titems.data(), 4 * titems.size(), cudaMemcpyHostToDevice, s));
    IMQ_CUDA(cudaMemsetAsync(P.V.off.ptr, 0, 4 * (size_t)(nb + 1), s));
    P.V.total = 0;
    IMQ_CUDA(cudaMemsetAsync(P.vtab.ptr, 0xFF, sizeof(int32_t) * kOffsetClasses * (size_t)nb, s));
    P.m2l_pairs = 0;
    P.m2l_level_lo = IMQ_MAX_LEVEL + 1;
    P.m2l_level_hi = 0;
    IMQ_CUDA(cudaStreamSynchronize(s));
}

void build_tree(Plan &P, const double *d_points, cudaStream_t s, bool check_dups) {
    const int64_t N = P.N;
    int *err = device_error_word();
    AsyncMem lerr(sizeof(int), s);
    IMQ_CUDA(cudaMemsetAsync(lerr.ptr, 0, sizeof(int), s));
    // ---- domain and finiteness
    {
        const int nb = (int)std::min<int64_t>(1024, std::max<int64_t>(1, (N + 255) / 256));
        AsyncMem part(sizeof(Box4) * nb, s);
        bbox_partial<<<nb, 256, 0, s>>>(d_points, N, part.as<Box4>(), lerr.as<int>());
        IMQ_LAUNCH_CHECK();
        std::vector<Box4> h(nb);
        int herr = 0;
        IMQ_CUDA(cudaMemcpyAsync(h.data(), part.ptr, sizeof(Box4) * nb, cudaMemcpyDeviceToHost, s));
        IMQ_CUDA(cudaMemcpyAsync(&herr, lerr.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
        IMQ_CUDA(cudaStreamSynchronize(s));
        if (herr & kErrNonFinite) fail(IMQ_INVALID_ARG, "imq_plan: a coordinate is NaN or infinite");
        if (P.side <= 0) {   // exact bounding square
            double mnx = INFINITY, mny = INFINITY, mxx = -INFINITY, mxy = -INFINITY;
            for (auto &q : h) {
                mnx = std::min(mnx, q.x); mny = std::min(mny, q.y);
                mxx = std::max(mxx, q.z); mxy = std::max(mxy, q.w);
            }
            P.x0 = mnx;
            P.y0 = mny;
            double sd = std::max(mxx - mnx, mxy - mny);
            P.side = sd > 0 ? sd : 1.0;
        }
    }
    // ---- Morton codes + stable radix sort
    P.codes.alloc(sizeof(uint32_t) * N);
    P.perm.alloc(sizeof(int32_t) * N);
    {
        AsyncMem k2(sizeof(uint32_t) * N, s), v2(sizeof(int32_t) * N, s);
        uint32_t *ka = P.codes.as<uint32_t>(), *kb = k2.as<uint32_t>();
        int32_t *va = P.perm.as<int32_t>(), *vb = v2.as<int32_t>();
        morton_codes<<<blocks_for(N, 256), 256, 0, s>>>(d_points, N, P.x0, P.y0, P.side, ka, va);
        IMQ_LAUNCH_CHECK();
        const int ntiles = (int)((N + kSortTile - 1) / kSortTile);
        AsyncMem cnt(sizeof(uint32_t) * 256 * ntiles, s), off(sizeof(uint32_t) * 256 * ntiles, s);
        for (int pass = 0; pass < 4; ++pass) {
            const int shift = 8 * pass;
            radix_hist<<<ntiles, kSortThreads, 0, s>>>(ka, N, shift, cnt.as<uint32_t>(), ntiles);
            IMQ_LAUNCH_CHECK();
            exclusive_scan<uint32_t>(cnt.as<uint32_t>(), off.as<uint32_t>(), (int64_t)256 * ntiles, nullptr, s);
            radix_scatter<<<ntiles, kSortThreads, 0, s>>>(ka, va, kb, vb, N, shift, off.as<uint32_t>(), ntiles);
            IMQ_LAUNCH_CHECK();
            std::swap(ka, kb);
            std::swap(va, vb);
        }
        // after 4 passes the result is back in (ka, va) == P.codes / P.perm
    }
    P.pos.alloc(sizeof(double2) * N);
    gather_points<<<blocks_for(N, 256), 256, 0, s>>>(d_points, P.perm.as<int32_t>(), N, P.pos.as<double2>());
    IMQ_LAUNCH_CHECK();
    if (check_dups) {
        dup_check<<<blocks_for(N, 256), 256, 0, s>>>(N, P.codes.as<uint32_t>(), P.pos.as<double2>(), lerr.as<int>());
        IMQ_LAUNCH_CHECK();
    }

    // ---- boxes, level by level
    DVec<int32_t> level, begin, end, parent, child;
    DVec<uint32_t> prefix;
    size_t cap0 = (size_t)std::max<int64_t>(1024, 2 * (4 * N / std::max(1, P.leaf) + 16));
    level.reserve(cap0, s); begin.reserve(cap0, s); end.reserve(cap0, s); parent.reserve(cap0, s);
    prefix.reserve(cap0, s); child.reserve(4 * cap0, s);
    {
        int32_t h_root[5] = {0, 0, (int32_t)N, -1, 0};
        int32_t neg[4] = {-1, -1, -1, -1};
        uint32_t zero = 0;
        IMQ_CUDA(cudaMemcpyAsync(level.ptr(), &h_root[0], 4, cudaMemcpyHostToDevice, s));
        IMQ_CUDA(cudaMemcpyAsync(begin.ptr(), &h_root[1], 4, cudaMemcpyHostToDevice, s));
        IMQ_CUDA(cudaMemcpyAsync(end.ptr(), &h_root[2], 4, cudaMemcpyHostToDevice, s));
        IMQ_CUDA(cudaMemcpyAsync(parent.ptr(), &h_root[3], 4, cudaMemcpyHostToDevice, s));
        IMQ_CUDA(cudaMemcpyAsync(prefix.ptr(), &zero, 4, cudaMemcpyHostToDevice, s));
        IMQ_CUDA(cudaMemcpyAsync(child.ptr(), neg, 16, cudaMemcpyHostToDevice, s));
        IMQ_CUDA(cudaStreamSynchronize(s));
        level.n = begin.n = end.n = parent.n = prefix.n = 1;
        child.n = 4;
    }
    P.level_start = {0, 1};
    int nb = 1;
    for (int lev = 0; lev < IMQ_MAX_LEVEL; ++lev) {
        const int lb = P.level_start[lev], nl = P.level_start[lev + 1] - lb;
        if (nl == 0) break;
        AsyncMem qb(sizeof(int32_t) * 5 * nl, s), nch(sizeof(int32_t) * nl, s), cb(sizeof(int32_t) * nl, s),
            tot(sizeof(int32_t), s);
        split_count<<<blocks_for(nl, 256), 256, 0, s>>>(lb, nl, lev, P.leaf, P.tc_depth, P.codes.as<uint32_t>(), begin.ptr(),
                                                         end.ptr(), prefix.ptr(), qb.as<int32_t>(), nch.as<int32_t>());
        IMQ_LAUNCH_CHECK();
        exclusive_scan<int32_t>(nch.as<int32_t>(), cb.as<int32_t>(), nl, tot.as<int32_t>(), s);
        const int nnew = read_i32(tot.as<int32_t>(), s);
        if (nnew == 0) break;
        const size_t need = (size_t)nb + nnew;
        level.reserve(need, s); begin.reserve(need, s); end.reserve(need, s); parent.reserve(need, s);
        prefix.reserve(need, s); child.reserve(4 * need, s);
        make_children<<<blocks_for(nl, 256), 256, 0, s>>>(lb, nl, lev, nb, qb.as<int32_t>(), nch.as<int32_t>(),
                                                           cb.as<int32_t>(), prefix.ptr(), level.ptr(), prefix.ptr(),
                                                           begin.ptr(), end.ptr(), parent.ptr(), child.ptr());
        IMQ_LAUNCH_CHECK();
        nb += nnew;
        level.n = begin.n = end.n = parent.n = prefix.n = nb;
        child.n = 4 * (size_t)nb;
        P.level_start.push_back(nb);
    }
    P.nbox = nb;
    P.max_level = (int)P.level_start.size() - 2;
    shrink_into(P.level, level, s);
    shrink_into(P.begin, begin, s);
    shrink_into(P.end, end, s);
    shrink_into(P.parent, parent, s);
    shrink_into(P.prefix, prefix, s);
    shrink_into(P.child, child, s);
    IMQ_CUDA(cudaStreamSynchronize(s));

    // ---- geometry, colleagues, lists
    DevMem ixy, isleaf;
    ixy.alloc(sizeof(int2) * nb);
    isleaf.alloc(nb);
    P.centre.alloc(sizeof(double2) * nb);
    box_geometry<<<blocks_for(nb, 256), 256, 0, s>>>(nb, P.level.as<int32_t>(), P.prefix.as<uint32_t>(),
                                                      P.child.as<int32_t>(), P.x0, P.y0, P.side, ixy.as<int2>(),
                                                      P.centre.as<double2>(), isleaf.as<int8_t>());
    IMQ_LAUNCH_CHECK();
    P.colleagues.alloc(sizeof(int32_t) * 9 * nb);
    {
        int32_t rootcol[9] = {0, -1, -1, -1, -1, -1, -1, -1, -1};
        IMQ_CUDA(cudaMemcpyAsync(P.colleagues.ptr, rootcol, sizeof(rootcol), cudaMemcpyHostToDevice, s));
    }
    BoxView T{P.level.as<int32_t>(), ixy.as<int2>(), P.child.as<int32_t>(), P.parent.as<int32_t>(),
              P.colleagues.as<int32_t>(), isleaf.as<int8_t>()};
    DevMem vcnt;
    vcnt.alloc(sizeof(int32_t) * nb);
    IMQ_CUDA(cudaMemsetAsync(vcnt.ptr, 0, sizeof(int32_t) * nb, s));
    for (int lev = 1; lev <= P.max_level; ++lev) {
        const int lb = P.level_start[lev], nl = P.level_start[lev + 1] - lb;
        colleagues_level<<<blocks_for(nl, 128), 128, 0, s>>>(lb, nl, T, P.colleagues.as<int32_t>(),
                                                             vcnt.as<int32_t>(), lerr.as<int>());
        IMQ_LAUNCH_CHECK();
    }
    auto make_csr = [&](ListCSR &L, const int32_t *cnt) {
        L.off.alloc(sizeof(int32_t) * (nb + 1));
        exclusive_scan<int32_t>(cnt, L.off.as<int32_t>(), nb, L.off.as<int32_t>() + nb, s);
        L.total = read_i32(L.off.as<int32_t>() + nb, s);
        L.items.alloc(sizeof(int32_t) * std::max<int64_t>(1, L.total));
    };
    make_csr(P.V, vcnt.as<int32_t>());
    v_fill<<<blocks_for(nb, 128), 128, 0, s>>>(nb, T, P.V.off.as<int32_t>(), P.V.items.as<int32_t>());
    IMQ_LAUNCH_CHECK();
    DevMem ucnt, wcnt, xcnt, cursor;
    ucnt.alloc(sizeof(int32_t) * nb);
    wcnt.alloc(sizeof(int32_t) * nb);
    IMQ_CUDA(cudaMemsetAsync(ucnt.ptr, 0, sizeof(int32_t) * nb, s));
    IMQ_CUDA(cudaMemsetAsync(wcnt.ptr, 0, sizeof(int32_t) * nb, s));
    uw_lists<<<blocks_for(nb, 64), 64, 0, s>>>(nb, T, 0, ucnt.as<int32_t>(), wcnt.as<int32_t>(), nullptr, nullptr,
                                               nullptr, nullptr, lerr.as<int>());
    IMQ_LAUNCH_CHECK();
    make_csr(P.U, ucnt.as<int32_t>());
    make_csr(P.W, wcnt.as<int32_t>());
    uw_lists<<<blocks_for(nb, 64), 64, 0, s>>>(nb, T, 1, nullptr, nullptr, P.U.off.as<int32_t>(),
                                               P.W.off.as<int32_t>(), P.U.items.as<int32_t>(),
                                               P.W.items.as<int32_t>(), lerr.as<int>());
    IMQ_LAUNCH_CHECK();
    xcnt.alloc(sizeof(int32_t) * nb);
    cursor.alloc(sizeof(int32_t) * nb);
    IMQ_CUDA(cudaMemsetAsync(xcnt.ptr, 0, sizeof(int32_t) * nb, s));
    IMQ_CUDA(cudaMemsetAsync(cursor.ptr, 0, sizeof(int32_t) * nb, s));
    x_count<<<blocks_for(nb, 128), 128, 0, s>>>(nb, isleaf.as<int8_t>(), P.W.off.as<int32_t>(),
                                                P.W.items.as<int32_t>(), xcnt.as<int32_t>());
    IMQ_LAUNCH_CHECK();
    make_csr(P.X, xcnt.as<int32_t>());
    x_fill<<<blocks_for(nb, 128), 128, 0, s>>>(nb, isleaf.as<int8_t>(), P.W.off.as<int32_t>(),
                                               P.W.items.as<int32_t>(), P.X.off.as<int32_t>(), cursor.as<int32_t>(),
                                               P.X.items.as<int32_t>());
    IMQ_LAUNCH_CHECK();
    sort_segments<<<blocks_for(nb, 128), 128, 0, s>>>(nb, P.X.off.as<int32_t>(), P.X.items.as<int32_t>());
    IMQ_LAUNCH_CHECK();

    // ---- leaves, per-point data, P2P and M2L auxiliaries
    {
        std::vector<int8_t> hl(nb);
        IMQ_CUDA(cudaMemcpyAsync(hl.data(), isleaf.ptr, nb, cudaMemcpyDeviceToHost, s));
        IMQ_CUDA(cudaStreamSynchronize(s));
        std::vector<int32_t> lv;
        for (int b = 0; b < nb; ++b)
            if (hl[b]) lv.push_back(b);
        P.nleaf = (int)lv.size();
        P.leaves.alloc(sizeof(int32_t) * std::max(1, P.nleaf));
        IMQ_CUDA(cudaMemcpyAsync(P.leaves.ptr, lv.data(), sizeof(int32_t) * lv.size(), cudaMemcpyHostToDevice, s));
        IMQ_CUDA(cudaStreamSynchronize(s));
    }
    P.leaf_of.alloc(sizeof(int32_t) * N);
    P.loc.alloc(sizeof(float2) * N);
    leaf_points<<<nb, 128, 0, s>>>(nb, isleaf.as<int8_t>(), P.begin.as<int32_t>(), P.end.as<int32_t>(),
                                   P.centre.as<double2>(), P.pos.as<double2>(), P.leaf_of.as<int32_t>(),
                                   P.loc.as<float2>());
    IMQ_LAUNCH_CHECK();
    P.ucum.alloc(sizeof(int32_t) * std::max<int64_t>(1, P.U.total));
    P.utot.alloc(sizeof(int32_t) * nb);
    P.uoff.alloc(sizeof(float2) * std::max<int64_t>(1, P.U.total));
    {
        AsyncMem pairs(sizeof(unsigned long long), s);
        IMQ_CUDA(cudaMemsetAsync(pairs.ptr, 0, sizeof(unsigned long long), s));
        u_aux<<<blocks_for(nb, 128), 128, 0, s>>>(nb, isleaf.as<int8_t>(), P.begin.as<int32_t>(),
                                                  P.end.as<int32_t>(), P.centre.as<double2>(), P.U.off.as<int32_t>(),
                                                  P.U.items.as<int32_t>(), P.ucum.as<int32_t>(),
                                                  P.utot.as<int32_t>(), P.uoff.as<float2>(),
                                                  pairs.as<unsigned long long>());
        IMQ_LAUNCH_CHECK();
        unsigned long long hp = 0;
        IMQ_CUDA(cudaMemcpyAsync(&hp, pairs.ptr, sizeof(hp), cudaMemcpyDeviceToHost, s));
        IMQ_CUDA(cudaStreamSynchronize(s));
        P.p2p_pairs = (int64_t)hp;
    }
    P.vtab.alloc(sizeof(int32_t) * kOffsetClasses * (size_t)nb);
    v_table<<<blocks_for(nb, 128), 128, 0, s>>>(nb, ixy.as<int2>(), P.V.off.as<int32_t>(), P.V.items.as<int32_t>(),
                                                P.vtab.as<int32_t>());
    IMQ_LAUNCH_CHECK();
    P.m2l_pairs = P.V.total;
    {
        std::vector<int32_t> hx(nb + 1), xb;
        IMQ_CUDA(cudaMemcpyAsync(hx.data(), P.X.off.ptr, sizeof(int32_t) * (nb + 1), cudaMemcpyDeviceToHost, s));
        IMQ_CUDA(cudaStreamSynchronize(s));
        for (int b = 0; b < nb; ++b)
            if (hx[b + 1] > hx[b]) xb.push_back(b);
        P.nxbox = (int)xb.size();
        P.xboxes.alloc(sizeof(int32_t) * std::max<size_t>(1, xb.size()));
        if (!xb.empty())
            IMQ_CUDA(cudaMemcpyAsync(P.xboxes.ptr, xb.data(), sizeof(int32_t) * xb.size(), cudaMemcpyHostToDevice, s));
        IMQ_CUDA(cudaStreamSynchronize(s));
    }
    // levels that hold V pairs
    {
        std::vector<int32_t> hoff(nb + 1);
        IMQ_CUDA(cudaMemcpyAsync(hoff.data(), P.V.off.ptr, sizeof(int32_t) * (nb + 1), cudaMemcpyDeviceToHost, s));
        IMQ_CUDA(cudaStreamSynchronize(s));
        P.m2l_level_lo = IMQ_MAX_LEVEL + 1;
        P.m2l_level_hi = 0;
        for (int lev = 0; lev <= P.max_level; ++lev) {
            if (hoff[P.level_start[lev + 1]] > hoff[P.level_start[lev]]) {
                P.m2l_level_lo = std::min(P.m2l_level_lo, lev);
                P.m2l_level_hi = std::max(P.m2l_level_hi, lev);
            }
        }
    }
    P.xcum.alloc(sizeof(int32_t) * std::max<int64_t>(1, P.X.total));
    P.xtot.alloc(sizeof(int32_t) * nb);
    x_aux<<<blocks_for(nb, 128), 128, 0, s>>>(nb, P.begin.as<int32_t>(), P.end.as<int32_t>(), P.X.off.as<int32_t>(),
                                              P.X.items.as<int32_t>(), P.xcum.as<int32_t>(), P.xtot.as<int32_t>());
    IMQ_LAUNCH_CHECK();
    if (P.tc_depth > 0) treecode_lists(P, s);
    build_m2l_tiles(P, s);
    int herr = 0;
    IMQ_CUDA(cudaMemcpyAsync(&herr, lerr.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
    IMQ_CUDA(cudaStreamSynchronize(s));
    if (herr & kErrDuplicate) fail(IMQ_DUPLICATE_POINTS, "imq_plan: two points are exactly equal");
    if (herr & (kErrListOverflow | kErrStackOverflow))
        fail(IMQ_CUDA_ERROR, "imq_plan: internal list capacity exceeded");
    (void)err;
}

}  // namespace imq
