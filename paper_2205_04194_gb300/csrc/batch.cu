// Batched plans: many independent problems (their own points, their own shape
// c, one expansion order p) merged into one flattened tree, so that every
// phase of the fast product is one launch over all problems.
//
// Boxes of all problems are renumbered in (level, problem, prefix) order, so a
// level is still one contiguous range and the per-level kernels (M2M, L2L)
// cover every problem at once.  Interaction lists never cross problems.  Each
// box carries its problem index; kernels that depend on c read it through
// ShapeC.  The M2L operators depend on c / h, so there is one operator set per
// (problem, level); they are generated on the device (the host would need
// minutes for hundreds of problems): one CTA per (problem-level, offset class)
// evaluates the normalised irregular solid harmonics of the translation
// vector in FP64 and folds them into the real parity-reduced operator with a
// host-built table of the factorial scale factors -- the same construction
// as operators.cpp, evaluated in parallel.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "imq_internal.h"
#include "util.cuh"

namespace imq {
namespace {

constexpr int kMaxJ = 2 * IMQ_MAX_P;   // harmonic degree reached by M2L

struct OpPair {     // one (output complex coefficient, input complex coefficient) pair
    int16_t k, l, n, m;      // output (k, l >= 0), input (n, m >= 0)
    int32_t oRe, oIm, iRe, iIm;
    double s1, s2;           // scale factors of the +m and -m terms (0 if absent)
};

double log_s(int n, int m) {
    m = std::abs(m);
    return 0.5 * (std::lgamma(n + m + 1.0) + std::lgamma(n - m + 1.0));
}

// One CTA per (slot, class): op[slot][class][iSlot][oSlot (padded to Kp)].
template <class T>
__global__ void k_m2l_generate(int nslot, const double2 *__restrict__ slot_hc,   // (h, c) per slot
                               const OpPair *__restrict__ pairs, int npairs, int p, int Kin, int Kp,
                               T *__restrict__ ops) {
    __shared__ double Pt[(kMaxJ + 1) * (kMaxJ + 1)];   // Ptilde_j^i(cos th)
    __shared__ double cs[kMaxJ + 1], sn[kMaxJ + 1], pw[kMaxJ + 1];
    const int slot = blockIdx.x / kOffsetClasses, cls = blockIdx.x % kOffsetClasses;
    if (slot >= nslot) return;
    int dx = 0, dy = 0;
    {   // same enumeration as offset_of_class()
        int c2 = 0;
        for (int a = -3; a <= 3; ++a)
            for (int b = -3; b <= 3; ++b) {
                if (a >= -1 && a <= 1 && b >= -1 && b <= 1) continue;
                if (c2 == cls) { dx = a; dy = b; }
                ++c2;
            }
    }
    const double h = slot_hc[slot].x, c = slot_hc[slot].y;
    const double vx = -dx * h, vy = -dy * h, vz = c;
    const double r = sqrt(vx * vx + vy * vy + vz * vz);
    const double ct = vz / r, st = sqrt(fmax(0.0, 1.0 - ct * ct));
    const double om = atan2(vy, vx);
    const int J = 2 * p, S1 = J + 1;
    if (threadIdx.x == 0) {
        // normalised associated Legendre functions, as in operators.cpp
        Pt[0] = 1.0;
        for (int m = 1; m <= J; ++m) Pt[m * S1 + m] = Pt[(m - 1) * S1 + (m - 1)] * sqrt((2.0 * m - 1.0) / (2.0 * m)) * st;
        for (int m = 0; m < J; ++m) Pt[(m + 1) * S1 + m] = sqrt(2.0 * m + 1.0) * ct * Pt[m * S1 + m];
        for (int m = 0; m <= J; ++m)
            for (int n = m + 2; n <= J; ++n)
                Pt[n * S1 + m] = ((2.0 * n - 1.0) * ct * Pt[(n - 1) * S1 + m] -
                                  sqrt((double)(n - 1) * (n - 1) - (double)m * m) * Pt[(n - 2) * S1 + m]) /
                                 sqrt((double)n * n - (double)m * m);
        double q = 1.0 / r;
        for (int j = 0; j <= J; ++j) {
            pw[j] = q;            // (h/r)^j / r
            q *= h / r;
        }
    }
    for (int i = threadIdx.x; i <= J; i += blockDim.x) {
        cs[i] = cos(i * om);
        sn[i] = sin(i * om);
    }
    __syncthreads();
    T *op = ops + ((size_t)slot * kOffsetClasses + cls) * Kin * Kp;
    // I(j, i): Ptilde e^{i i om} with I(j, -i) = (-1)^i conj(I(j, i))
    auto harm = [&](int j, int i, double &re, double &im) {
        const int a = i < 0 ? -i : i;
        re = Pt[j * S1 + a] * cs[a];
        im = Pt[j * S1 + a] * sn[a];
        if (i < 0) {
            im = -im;
            if (a & 1) { re = -re; im = -im; }
        }
    };
    for (int e = threadIdx.x; e < npairs; e += blockDim.x) {
        const OpPair q = pairs[e];
        const int j = q.n + q.k;
        const double sgk = (q.k & 1) ? -1.0 : 1.0;
        double r1, i1;
        harm(j, q.m + q.l, r1, i1);
        const double f1 = sgk * q.s1 * pw[j];
        r1 *= f1;
        i1 *= f1;
        if (q.m == 0) {
            op[(size_t)q.iRe * Kp + q.oRe] = (T)r1;
            if (q.oIm >= 0) op[(size_t)q.iRe * Kp + q.oIm] = (T)i1;
        } else {
            double r2, i2;
            harm(j, q.l - q.m, r2, i2);
            const double f2 = sgk * q.s2 * pw[j];
            r2 *= f2;
            i2 *= f2;
            const double sg = (q.m & 1) ? -1.0 : 1.0;
            const double ar = r1 + sg * r2, ai = i1 + sg * i2;   // A = T1 + sgn T2
            const double br = r1 - sg * r2, bi = i1 - sg * i2;   // B = T1 - sgn T2
            op[(size_t)q.iRe * Kp + q.oRe] = (T)ar;
            op[(size_t)q.iIm * Kp + q.oRe] = (T)(-bi);
            if (q.oIm >= 0) {
                op[(size_t)q.iRe * Kp + q.oIm] = (T)ai;
                op[(size_t)q.iIm * Kp + q.oIm] = (T)br;
            }
        }
    }
}

std::vector<OpPair> op_pairs(const Layout &Lo, const Layout &Li) {
    std::vector<OpPair> v;
    const int p = Lo.p;
    for (int k = 0; k <= p; ++k)
        for (int l = 0; l <= k; ++l) {
            const int oRe = Lo.re_slot[k * (p + 1) + l];
            if (oRe < 0) continue;
            const int oIm = Lo.im_slot[k * (p + 1) + l];
            for (int n = 0; n <= p; ++n)
                for (int m = 0; m <= n; ++m) {
                    const int iRe = Li.re_slot[n * (p + 1) + m];
                    if (iRe < 0) continue;
                    OpPair q;
                    q.k = (int16_t)k; q.l = (int16_t)l; q.n = (int16_t)n; q.m = (int16_t)m;
                    q.oRe = oRe; q.oIm = oIm; q.iRe = iRe; q.iIm = Li.im_slot[n * (p + 1) + m];
                    const int j = n + k;
                    q.s1 = std::exp(log_s(j, m + l) - log_s(k, l) - log_s(n, m));
                    q.s2 = m > 0 ? std::exp(log_s(j, l - m) - log_s(k, l) - log_s(n, m)) : 0.0;
                    v.push_back(q);
                }
        }
    return v;
}

}  // namespace

// Generate the M2L operators of every (h, c) slot into `dst` ([nslot][40][Kin][Kp], zero padded).
template <class T>
void generate_m2l_ops(const Layout &Lo, const Layout &Li, const std::vector<double2> &slot_hc, int Kp, DevMem &dst,
                      cudaStream_t s) {
    const auto pairs = op_pairs(Lo, Li);
    const int nslot = (int)slot_hc.size();
    const size_t n = (size_t)std::max(1, nslot) * kOffsetClasses * Li.K * Kp;
    dst.alloc(sizeof(T) * n);
    IMQ_CUDA(cudaMemsetAsync(dst.ptr, 0, sizeof(T) * n, s));
    if (nslot == 0) return;
    AsyncMem dpairs(sizeof(OpPair) * pairs.size(), s), dhc(sizeof(double2) * nslot, s);
    IMQ_CUDA(cudaMemcpyAsync(dpairs.ptr, pairs.data(), sizeof(OpPair) * pairs.size(), cudaMemcpyHostToDevice, s));
    IMQ_CUDA(cudaMemcpyAsync(dhc.ptr, slot_hc.data(), sizeof(double2) * nslot, cudaMemcpyHostToDevice, s));
    k_m2l_generate<T><<<nslot * kOffsetClasses, 256, 0, s>>>(nslot, dhc.as<double2>(), dpairs.as<OpPair>(),
                                                              (int)pairs.size(), Li.p, Li.K, Kp, dst.as<T>());
    IMQ_LAUNCH_CHECK();
    IMQ_CUDA(cudaStreamSynchronize(s));
}

template void generate_m2l_ops<float>(const Layout &, const Layout &, const std::vector<double2> &, int, DevMem &,
                                      cudaStream_t);
template void generate_m2l_ops<double>(const Layout &, const Layout &, const std::vector<double2> &, int, DevMem &,
                                       cudaStream_t);

}  // namespace imq

namespace imq {
namespace {

template <class T>
std::vector<T> d2h(const DevMem &d, size_t n, cudaStream_t s) {
    std::vector<T> h(n);
    if (n) IMQ_CUDA(cudaMemcpyAsync(h.data(), d.ptr, sizeof(T) * n, cudaMemcpyDeviceToHost, s));
    return h;
}

template <class T>
void h2d(DevMem &d, const std::vector<T> &h, cudaStream_t s) {
    d.alloc(sizeof(T) * std::max<size_t>(1, h.size()));
    if (!h.empty()) IMQ_CUDA(cudaMemcpyAsync(d.ptr, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice, s));
}

struct HostTree {
    int nbox = 0, nleaf = 0, max_level = 0, lo = 0, hi = -1;
    int64_t N = 0, p2p_pairs = 0;
    std::vector<int> level_start;
    std::vector<int32_t> level, begin, end, parent, child, leaves, perm, leaf_of, vtab, utot, xtot;
    std::vector<uint32_t> prefix, codes;
    std::vector<double2> centre, pos;
    std::vector<float2> loc, uoff;
    std::vector<int32_t> Uoff, Uit, Voff, Vit, Woff, Wit, Xoff, Xit, ucum, xcum;
};

HostTree download(Plan &Q, cudaStream_t s) {
    HostTree t;
    t.nbox = Q.nbox;
    t.nleaf = Q.nleaf;
    t.max_level = Q.max_level;
    t.lo = Q.m2l_level_lo;
    t.hi = Q.m2l_level_hi;
    t.N = Q.N;
    t.p2p_pairs = Q.p2p_pairs;
    t.level_start = Q.level_start;
    const size_t nb = Q.nbox, N = Q.N;
    t.level = d2h<int32_t>(Q.level, nb, s);
    t.begin = d2h<int32_t>(Q.begin, nb, s);
    t.end = d2h<int32_t>(Q.end, nb, s);
    t.parent = d2h<int32_t>(Q.parent, nb, s);
    t.child = d2h<int32_t>(Q.child, 4 * nb, s);
    t.leaves = d2h<int32_t>(Q.leaves, Q.nleaf, s);
    t.perm = d2h<int32_t>(Q.perm, N, s);
    t.leaf_of = d2h<int32_t>(Q.leaf_of, N, s);
    t.vtab = d2h<int32_t>(Q.vtab, (size_t)kOffsetClasses * nb, s);
    t.utot = d2h<int32_t>(Q.utot, nb, s);
    t.xtot = d2h<int32_t>(Q.xtot, nb, s);
    t.prefix = d2h<uint32_t>(Q.prefix, nb, s);
    t.codes = d2h<uint32_t>(Q.codes, N, s);
    t.centre = d2h<double2>(Q.centre, nb, s);
    t.pos = d2h<double2>(Q.pos, N, s);
    t.loc = d2h<float2>(Q.loc, N, s);
    t.uoff = d2h<float2>(Q.uoff, Q.U.total, s);
    t.Uoff = d2h<int32_t>(Q.U.off, nb + 1, s);
    t.Uit = d2h<int32_t>(Q.U.items, Q.U.total, s);
    t.Voff = d2h<int32_t>(Q.V.off, nb + 1, s);
    t.Vit = d2h<int32_t>(Q.V.items, Q.V.total, s);
    t.Woff = d2h<int32_t>(Q.W.off, nb + 1, s);
    t.Wit = d2h<int32_t>(Q.W.items, Q.W.total, s);
    t.Xoff = d2h<int32_t>(Q.X.off, nb + 1, s);
    t.Xit = d2h<int32_t>(Q.X.items, Q.X.total, s);
    t.ucum = d2h<int32_t>(Q.ucum, Q.U.total, s);
    t.xcum = d2h<int32_t>(Q.xcum, Q.X.total, s);
    IMQ_CUDA(cudaStreamSynchronize(s));
    return t;
}

}  // namespace

void build_batched_plan(Plan &P, const double *d_points, const std::vector<int64_t> &offs,
                        const std::vector<double> &cs, bool dups, cudaStream_t s) {
    const int B = (int)cs.size();
    P.nprob = B;
    P.h_prob_c = cs;
    std::vector<HostTree> H(B);
    for (int b = 0; b < B; ++b) {
        Plan Q;
        Q.device = P.device;
        Q.N = offs[b + 1] - offs[b];
        Q.c = cs[b];
        Q.p = P.p;
        Q.leaf = P.leaf;
        Q.x0 = P.x0;
        Q.y0 = P.y0;
        Q.side = P.side;
        Q.layout = P.layout;
        build_tree(Q, d_points + 2 * offs[b], s, dups);
        H[b] = download(Q, s);
    }
    // ---- new box numbering: (level, problem, prefix)
    int maxL = 0;
    for (auto &t : H) maxL = std::max(maxL, t.max_level);
    std::vector<std::vector<int32_t>> nid(B);
    for (int b = 0; b < B; ++b) nid[b].assign(H[b].nbox, -1);
    P.level_start.assign(1, 0);
    int nb = 0;
    for (int lev = 0; lev <= maxL; ++lev) {
        for (int b = 0; b < B; ++b) {
            const HostTree &t = H[b];
            if (lev > t.max_level) continue;
            for (int o = t.level_start[lev]; o < t.level_start[lev + 1]; ++o) nid[b][o] = nb++;
        }
        P.level_start.push_back(nb);
    }
    P.nbox = nb;
    P.max_level = maxL;
    P.N = offs[B];
    auto map = [&](int b, int o) { return o < 0 ? -1 : nid[b][o]; };
    // ---- per-box arrays
    std::vector<int32_t> level(nb), begin(nb), end(nb), parent(nb), child(4 * (size_t)nb), vtab((size_t)kOffsetClasses * nb),
        utot(nb), xtot(nb), box_prob(nb);
    std::vector<uint32_t> prefix(nb);
    std::vector<double2> centre(nb);
    for (int b = 0; b < B; ++b) {
        const HostTree &t = H[b];
        for (int o = 0; o < t.nbox; ++o) {
            const int n = nid[b][o];
            level[n] = t.level[o];
            prefix[n] = t.prefix[o];
            begin[n] = (int32_t)(t.begin[o] + offs[b]);
            end[n] = (int32_t)(t.end[o] + offs[b]);
            parent[n] = map(b, t.parent[o]);
            for (int q = 0; q < 4; ++q) child[4 * (size_t)n + q] = map(b, t.child[4 * (size_t)o + q]);
            for (int k = 0; k < kOffsetClasses; ++k)
                vtab[(size_t)kOffsetClasses * n + k] = map(b, t.vtab[(size_t)kOffsetClasses * o + k]);
            utot[n] = t.utot[o];
            xtot[n] = t.xtot[o];
            centre[n] = t.centre[o];
            box_prob[n] = b;
        }
    }
    // ---- lists (CSR in new box order; items stay sorted: the renumbering is monotone within a problem)
    std::vector<int> owner(nb), oldid(nb);
    for (int b = 0; b < B; ++b)
        for (int o = 0; o < H[b].nbox; ++o) {
            owner[nid[b][o]] = b;
            oldid[nid[b][o]] = o;
        }
    auto merge_list = [&](ListCSR &L, auto get_off, auto get_items, std::vector<int32_t> *cum_out,
                          auto get_cum, std::vector<float2> *delta_out, auto get_delta) {
        std::vector<int32_t> off(nb + 1, 0), items;
        for (int n = 0; n < nb; ++n) {
            const int b = owner[n], o = oldid[n];
            const auto &offv = get_off(H[b]);
            const auto &it = get_items(H[b]);
            for (int k = offv[o]; k < offv[o + 1]; ++k) {
                items.push_back(map(b, it[k]));
                if (cum_out) cum_out->push_back(get_cum(H[b])[k]);
                if (delta_out) delta_out->push_back(get_delta(H[b])[k]);
            }
            off[n + 1] = (int32_t)items.size();
        }
        L.total = (int64_t)items.size();
        h2d(L.off, off, s);
        h2d(L.items, items, s);
        return off;
    };
    std::vector<int32_t> ucum, xcum;
    std::vector<float2> uoff;
    auto noneI = [](const HostTree &) -> const std::vector<int32_t> & { static std::vector<int32_t> e; return e; };
    auto noneF = [](const HostTree &) -> const std::vector<float2> & { static std::vector<float2> e; return e; };
    merge_list(P.U, [](const HostTree &t) -> const std::vector<int32_t> & { return t.Uoff; },
               [](const HostTree &t) -> const std::vector<int32_t> & { return t.Uit; }, &ucum,
               [](const HostTree &t) -> const std::vector<int32_t> & { return t.ucum; }, &uoff,
               [](const HostTree &t) -> const std::vector<float2> & { return t.uoff; });
    merge_list(P.V, [](const HostTree &t) -> const std::vector<int32_t> & { return t.Voff; },
               [](const HostTree &t) -> const std::vector<int32_t> & { return t.Vit; }, nullptr, noneI, nullptr, noneF);
    merge_list(P.W, [](const HostTree &t) -> const std::vector<int32_t> & { return t.Woff; },
               [](const HostTree &t) -> const std::vector<int32_t> & { return t.Wit; }, nullptr, noneI, nullptr, noneF);
    const auto xoffv =
        merge_list(P.X, [](const HostTree &t) -> const std::vector<int32_t> & { return t.Xoff; },
                   [](const HostTree &t) -> const std::vector<int32_t> & { return t.Xit; }, &xcum,
                   [](const HostTree &t) -> const std::vector<int32_t> & { return t.xcum; }, nullptr, noneF);
    // ---- points, leaves
    const int64_t N = P.N;
    std::vector<int32_t> perm(N), leaf_of(N), pt_prob(N), leaves, xboxes;
    std::vector<uint32_t> codes(N);
    std::vector<double2> pos(N);
    std::vector<float2> loc(N);
    int64_t pairs = 0;
    for (int b = 0; b < B; ++b) {
        const HostTree &t = H[b];
        for (int64_t i = 0; i < t.N; ++i) {
            const int64_t g = offs[b] + i;
            perm[g] = (int32_t)(offs[b] + t.perm[i]);
            leaf_of[g] = map(b, t.leaf_of[i]);
            pt_prob[g] = b;
            codes[g] = t.codes[i];
            pos[g] = t.pos[i];
            loc[g] = t.loc[i];
        }
        pairs += t.p2p_pairs;
    }
    for (int n = 0; n < nb; ++n) {
        if (child[4 * (size_t)n] < 0 && child[4 * (size_t)n + 1] < 0 && child[4 * (size_t)n + 2] < 0 &&
            child[4 * (size_t)n + 3] < 0)
            leaves.push_back(n);
        if (xoffv[n + 1] > xoffv[n]) xboxes.push_back(n);
    }
    P.nleaf = (int)leaves.size();
    P.nxbox = (int)xboxes.size();
    P.p2p_pairs = pairs;
    P.m2l_pairs = P.V.total;
    h2d(P.level, level, s); h2d(P.begin, begin, s); h2d(P.end, end, s); h2d(P.parent, parent, s);
    h2d(P.child, child, s); h2d(P.vtab, vtab, s); h2d(P.utot, utot, s); h2d(P.xtot, xtot, s);
    h2d(P.prefix, prefix, s); h2d(P.centre, centre, s); h2d(P.box_prob, box_prob, s);
    h2d(P.ucum, ucum, s); h2d(P.uoff, uoff, s); h2d(P.xcum, xcum, s);
    h2d(P.perm, perm, s); h2d(P.leaf_of, leaf_of, s); h2d(P.pt_prob, pt_prob, s); h2d(P.codes, codes, s);
    h2d(P.pos, pos, s); h2d(P.loc, loc, s); h2d(P.leaves, leaves, s); h2d(P.xboxes, xboxes, s);
    h2d(P.prob_c, cs, s);
    P.prob_off = offs;
    // ---- M2L operator slots (problem, level) and quadrant-grouped tiles
    std::vector<double2> slot_hc;
    std::vector<int32_t> box_opslot(nb, -1);
    std::vector<int4> tiles;
    std::vector<int32_t> order;
    std::vector<std::vector<int>> slot_of(B);
    P.m2l_level_lo = IMQ_MAX_LEVEL + 1;
    P.m2l_level_hi = 0;
    for (int b = 0; b < B; ++b) {
        slot_of[b].assign(maxL + 1, -1);
        for (int lev = H[b].lo; lev <= H[b].hi; ++lev) {
            slot_of[b][lev] = (int)slot_hc.size();
            slot_hc.push_back(make_double2(P.side / (double)(1 << lev), cs[b]));
            P.m2l_level_lo = std::min(P.m2l_level_lo, lev);
            P.m2l_level_hi = std::max(P.m2l_level_hi, lev);
        }
    }
    constexpr int kTB = 128;
    for (int lev = 0; lev <= maxL; ++lev)
        for (int b = 0; b < B; ++b) {
            if (lev > H[b].max_level || slot_of[b][lev] < 0) continue;
            const int sl = slot_of[b][lev];
            for (int q = 0; q < 4; ++q) {
                const int start = (int)order.size();
                const HostTree &t = H[b];
                for (int o = t.level_start[lev]; o < t.level_start[lev + 1]; ++o)
                    if ((int)(t.prefix[o] & 3u) == q) order.push_back(nid[b][o]);
                const int cnt = (int)order.size() - start;
                for (int k = 0; k < cnt; k += kTB) tiles.push_back(make_int4(sl, start + k, std::min(kTB, cnt - k), 0));
            }
            for (int o = H[b].level_start[lev]; o < H[b].level_start[lev + 1]; ++o) box_opslot[nid[b][o]] = sl;
        }
    P.n_m2l_tiles = (int)tiles.size();
    h2d(P.m2l_tiles, tiles, s);
    h2d(P.m2l_tbox, order, s);
    h2d(P.box_opslot, box_opslot, s);
    P.h_slot_hc = slot_hc;
    IMQ_CUDA(cudaStreamSynchronize(s));
}

}  // namespace imq
