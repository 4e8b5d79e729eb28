// The product with dA/dc, dA_ij/dc = -c / (|x_i - x_j|^2 + c^2)^{3/2}.
//
// Under the lift of the paper's Eq. (11) the vertical offset between a target
// X_i = (x_i, +c/2) and a source Y_j = (x_j, -c/2) is c, so d/dc of
// G(X;Y) = 1/|X - Y| is the derivative of G in the target's vertical
// coordinate.  The same multipoles therefore serve, and the derivative is
// taken where the field is evaluated:
//   * local expansion: d/dz conj(U_k^l(X - C)) = conj(U_{k-1}^l(X - C)); at an
//     in-plane target only k+l odd survives, so the derivative uses the
//     odd-parity locals (M2L, P2L and L2L into the odd layout);
//   * multipole (W list): d/dz T_n^m(X - Z) = -T_{n+1}^m(X - Z);
//   * near field: the kernel -c (r^2 + c^2)^{-3/2} directly.
// Both identities are checked against finite differences in the oracle tests.
#include <type_traits>

#include "fmm_common.cuh"
#include "imq_internal.h"
#include "ptx.cuh"
#include "util.cuh"

namespace imq {
namespace {

template <class T>
__global__ void k_far_dz(int nleaf, const int32_t *__restrict__ leaves, const int32_t *__restrict__ begin,
                         const int32_t *__restrict__ end, const int32_t *__restrict__ level,
                         const double2 *__restrict__ centre, const float2 *__restrict__ loc,
                         const double2 *__restrict__ pos, const int32_t *__restrict__ woff,
                         const int32_t *__restrict__ witems, const T *__restrict__ M, const T *__restrict__ Lodd,
                         const T *__restrict__ dzc, int Ke, int Ko, int p, double S, ShapeC shape,
                         T *__restrict__ bs) {
    __shared__ T tab2[(IMQ_MAX_P + 2) * (IMQ_MAX_P + 2)], tabi[(IMQ_MAX_P + 2) * (IMQ_MAX_P + 2)];
    fill_recurrence_tables<T>(tab2, tabi, p + 1);
    __syncthreads();
    const int P1 = p + 2;   // table stride
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= nleaf) return;
    const int b = leaves[warp];
    const double2 cb = centre[b];
    const T hb = box_side<T>(S, level[b]);
    const T inv_h = (T)1 / hb;
    const T c = (T)shape.of(b);
    const T *Lb = Lodd + (int64_t)b * Ko;
    for (int i = begin[b] + lane; i < end[b]; i += 32) {
        T wx, wy;
        point_offset<T>(i, loc, pos, cb, cb, wx, wy);
        T phi_l = 0;
        {   // d/dz L2P: sum eps_m dzc Re(Lh_k^l conj(w)^l |w|^{k-1-l}) / h over odd slots
            const T ux = wx * inv_h, uy = wy * inv_h;
            const T r2 = ux * ux + uy * uy;
            T zr = 1, zi = 0;
            int slot = 0;
            for (int m = 0; m < p; ++m) {
                T qr = zr, qi = zi;
                const T eps = m ? (T)2 : (T)1;
                for (int k = m + 1; k <= p; k += 2) {
                    const T lr = Lb[slot];
                    const T li = m ? Lb[slot + 1] : (T)0;
                    phi_l += eps * dzc[slot] * (lr * qr - li * qi);
                    qr *= r2;
                    qi *= r2;
                    slot += m ? 2 : 1;
                }
                const T nr = zr * ux + zi * uy;
                zi = zi * ux - zr * uy;
                zr = nr;
            }
        }
        T phi = phi_l * inv_h;
        // d/dz M2P over the W list: -sum eps_m sqrt((n+1+m)(n+1-m)) Re(Mh_n^m G_{n+1}^m) / h_s
        for (int e = woff[b]; e < woff[b + 1]; ++e) {
            const int s = witems[e];
            const double2 cs = centre[s];
            T vx, vy;
            point_offset<T>(i, loc, pos, cs, cb, vx, vy);
            const T hs = box_side<T>(S, level[s]);
            const T inv = rsq<T>(vx * vx + vy * vy + c * c);
            const T a = hs * inv, t = c * inv;
            const T zr0 = vx * inv * a, zi0 = vy * inv * a;
            const T ta = t * a, a2 = a * a;
            const T *Ms = M + (int64_t)s * Ke;
            T gr = inv, gi = 0;   // G_0^0
            T acc = 0;
            int slot = 0;
            for (int m = 0; m <= p; ++m) {
                if (m > 0) {
                    const T f = sqrt((T)(2 * m - 1) / (T)(2 * m));
                    const T nr = (gr * zr0 - gi * zi0) * f;
                    gi = (gr * zi0 + gi * zr0) * f;
                    gr = nr;
                }
                const T eps = m ? (T)2 : (T)1;
                T g2r = 0, g2i = 0, g1r = gr, g1i = gi;
                for (int n = m + 1; n <= p + 1; ++n) {
                    const T c1 = (T)(2 * n - 1) * ta;
                    const T c2 = tab2[n * P1 + m] * a2;
                    const T iv = tabi[n * P1 + m];
                    const T nr = (c1 * g1r - c2 * g2r) * iv;
                    const T ni = (c1 * g1i - c2 * g2i) * iv;
                    g2r = g1r; g2i = g1i; g1r = nr; g1i = ni;
                    if (((n - m) & 1) == 1) {   // pairs with Mh_{n-1}^m
                        const T mr = Ms[slot];
                        const T mi = m ? Ms[slot + 1] : (T)0;
                        acc -= eps * sqrt((T)((n + m) * (n - m))) * (mr * nr - mi * ni);
                        slot += m ? 2 : 1;
                    }
                }
            }
            phi += acc / hs;
        }
        bs[i] = phi;
    }
}

// Near field of the derivative: b_i += sum_U u_j * (-c) * (r^2 + c^2)^{-3/2}.
constexpr int kDzWarps = 4;

__device__ __forceinline__ int dz_source_index(int q, int &r, int u1, const int32_t *__restrict__ ucum,
                                               const int32_t *__restrict__ uitems, const int32_t *__restrict__ begin) {
    while (r + 1 < u1 && ucum[r + 1] <= q) ++r;
    return begin[uitems[r]] + (q - ucum[r]);
}

template <class T>
__device__ __forceinline__ T dz_reduce32(T (&acc)[32], int lane) {
#pragma unroll
    for (int k = 16; k >= 1; k >>= 1) {
        const bool upper = (lane & k) != 0;
#pragma unroll
        for (int i = 0; i < k; ++i) {
            const T send = upper ? acc[i] : acc[i + k];
            const T keep = upper ? acc[i + k] : acc[i];
            acc[i] = keep + __shfl_xor_sync(0xFFFFFFFFu, send, k);
        }
    }
    return acc[0];
}

template <class T>
__global__ void __launch_bounds__(32 * kDzWarps) k_p2p_dz(
    int nleaf, const int32_t *__restrict__ leaves, const int32_t *__restrict__ begin, const int32_t *__restrict__ end,
    const int32_t *__restrict__ uoffs, const int32_t *__restrict__ uitems, const int32_t *__restrict__ ucum,
    const int32_t *__restrict__ utot, const float2 *__restrict__ udelta, const float2 *__restrict__ loc,
    const double2 *__restrict__ pos, const T *__restrict__ u, ShapeC shape, T *__restrict__ bs) {
    __shared__ T tgx[kDzWarps][32], tgy[kDzWarps][32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int widx = blockIdx.x * kDzWarps + w;
    if (widx >= nleaf) return;
    const int b = leaves[widx];
    const int tb = begin[b], nt = end[b] - tb;
    const int u0 = uoffs[b], u1 = uoffs[b + 1];
    const int St = utot[b];
    const T c = (T)shape.of(b);
    const T c2 = c * c;
    for (int tc = 0; tc < nt; tc += 32) {
        const int ntc = min(32, nt - tc);
        if (lane < ntc) {
            if constexpr (std::is_same<T, float>::value) {
                tgx[w][lane] = loc[tb + tc + lane].x;
                tgy[w][lane] = loc[tb + tc + lane].y;
            } else {
                tgx[w][lane] = pos[tb + tc + lane].x;
                tgy[w][lane] = pos[tb + tc + lane].y;
            }
        }
        __syncwarp();
        T acc[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) acc[i] = 0;
        int r = u0;
        for (int q0 = 0; q0 < St; q0 += 32) {
            const int q = q0 + lane;
            T xs = 0, ys = 0, us = 0;
            if (q < St) {
                const int j = dz_source_index(q, r, u1, ucum, uitems, begin);
                if constexpr (std::is_same<T, float>::value) {
                    const float2 l = loc[j];
                    const float2 d = udelta[r];
                    xs = l.x - d.x;
                    ys = l.y - d.y;
                } else {
                    xs = pos[j].x;
                    ys = pos[j].y;
                }
                us = -c * u[j];
            }
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                if (i < ntc) {
                    const T dx = tgx[w][i] - xs, dy = tgy[w][i] - ys;
                    const T rs = rsq<T>(dx * dx + (dy * dy + c2));
                    acc[i] += us * rs * rs * rs;
                }
            }
        }
        const T tot = dz_reduce32<T>(acc, lane);
        if (lane < ntc) bs[tb + tc + lane] += tot;
        __syncwarp();
    }
}

template <class T>
void upload_pad(DevMem &dst, const std::vector<double> &src, size_t blocks, int rows, int cols, int colp,
                cudaStream_t s) {
    std::vector<T> tmp(blocks * (size_t)rows * colp, (T)0);
    for (size_t bk = 0; bk < blocks; ++bk)
        for (int i = 0; i < rows; ++i)
            for (int r = 0; r < cols; ++r)
                tmp[(bk * rows + i) * colp + r] = (T)src[(bk * rows + i) * cols + r];
    dst.alloc(sizeof(T) * std::max<size_t>(1, tmp.size()));
    IMQ_CUDA(cudaMemcpyAsync(dst.ptr, tmp.data(), sizeof(T) * tmp.size(), cudaMemcpyHostToDevice, s));
    IMQ_CUDA(cudaStreamSynchronize(s));
}

void ensure_ops_dz(Plan &P, bool fp64, cudaStream_t s) {
    if (P.nprob > 1) fail(IMQ_UNSUPPORTED, "the c-derivative product is not available on batched plans");
    ensure_ops(P, fp64, s);
    TypedOps &O = fp64 ? P.ops64 : P.ops32;
    if (O.dz_ready) return;
    const int Ke = P.layout.K;
    if (P.layout_odd.K == 0) P.layout_odd.build(P.p, 1);
    const int Ko = P.layout_odd.K;
    const int nlev = std::max(0, P.m2l_level_hi - P.m2l_level_lo + 1);
    if (P.h_l2l_odd.empty()) {
        build_l2l_ops(P.layout_odd, P.h_l2l_odd);
        l2p_dz_coefficients(P.layout_odd, P.h_dzc);
        P.h_m2l_odd.assign((size_t)std::max(1, nlev) * kOffsetClasses * Ke * Ko, 0.0);
        std::vector<double> tmp;
        for (int li = 0; li < nlev; ++li) {
            const double h = P.side / (double)(1 << (P.m2l_level_lo + li));
            build_m2l_ops(P.layout_odd, P.layout, h, P.c, tmp);
            std::copy(tmp.begin(), tmp.end(), P.h_m2l_odd.begin() + (size_t)li * kOffsetClasses * Ke * Ko);
        }
    }
    const size_t blocks = (size_t)std::max(1, nlev) * kOffsetClasses;
    const size_t es = fp64 ? sizeof(double) : sizeof(float);
    if (fp64) {
        upload_pad<double>(O.m2l_odd, P.h_m2l_odd, blocks, Ke, Ko, Ko, s);
        upload_pad<double>(O.l2l_odd, P.h_l2l_odd, 4, Ko, Ko, Ko, s);
        upload_pad<double>(O.dzc, P.h_dzc, 1, 1, Ko, Ko, s);
    } else {
        const int RR = m2l_tiled_rows(Ko);
        if (RR < 0) fail(IMQ_UNSUPPORTED, "expansion order too large for the M2L kernel");
        upload_pad<float>(O.m2l_odd, P.h_m2l_odd, blocks, Ke, Ko, 16 * RR, s);
        upload_pad<float>(O.l2l_odd, P.h_l2l_odd, 4, Ko, Ko, Ko, s);
        upload_pad<float>(O.dzc, P.h_dzc, 1, 1, Ko, Ko, s);
    }
    O.Lodd.alloc(es * (size_t)P.nbox * std::max(1, Ko));
    O.dz_ready = true;
}

}  // namespace

template <class T>
int fmm_apply_dz(Plan &P, const T *us, T *bs, int nrhs, cudaStream_t s) {
    const bool f64 = std::is_same<T, double>::value;
    ensure_ops_dz(P, f64, s);
    TypedOps &O = f64 ? P.ops64 : P.ops32;
    const int Ke = P.layout.K, Ko = P.layout_odd.K, nb = P.nbox;
    T *M = O.M.as<T>(), *Lo = O.Lodd.as<T>();
    int launches = 0;
    for (int r = 0; r < nrhs; ++r) {
        const T *u = us + (size_t)r * P.N;
        T *b = bs + (size_t)r * P.N;
        IMQ_CUDA(cudaMemsetAsync(M, 0, sizeof(T) * (size_t)nb * Ke, s));
        IMQ_CUDA(cudaMemsetAsync(Lo, 0, sizeof(T) * (size_t)nb * std::max(1, Ko), s));
        upward_launch<T>(P, u, M, O.p2mc.as<T>(), O.m2m.as<T>(), s, &launches);
        if constexpr (std::is_same<T, float>::value) {
            if (P.n_m2l_tiles > 0) {
                m2l_tiled_launch(P, M, Lo, O.m2l_odd.as<float>(), s, Ko);
                ++launches;
            }
        } else {
            m2l_direct_launch<T>(P, M, Lo, O.m2l_odd.as<T>(), Ke, Ko, s, &launches);
        }
        p2l_odd_launch<T>(P, u, Lo, s);
        l2l_launch<T>(P, Lo, O.l2l_odd.as<T>(), Ko, s, &launches);
        k_far_dz<T><<<blocks_for((int64_t)P.nleaf * 32, 128), 128, 0, s>>>(
            P.nleaf, P.leaves.as<int32_t>(), P.begin.as<int32_t>(), P.end.as<int32_t>(), P.level.as<int32_t>(),
            P.centre.as<double2>(), P.loc.as<float2>(), P.pos.as<double2>(), P.W.off.as<int32_t>(),
            P.W.items.as<int32_t>(), M, Lo, O.dzc.as<T>(), Ke, Ko, P.p, P.side, P.shape(), b);
        IMQ_LAUNCH_CHECK();
        k_p2p_dz<T><<<(unsigned)((P.nleaf + kDzWarps - 1) / kDzWarps), 32 * kDzWarps, 0, s>>>(
            P.nleaf, P.leaves.as<int32_t>(), P.begin.as<int32_t>(), P.end.as<int32_t>(), P.U.off.as<int32_t>(),
            P.U.items.as<int32_t>(), P.ucum.as<int32_t>(), P.utot.as<int32_t>(), P.uoff.as<float2>(),
            P.loc.as<float2>(), P.pos.as<double2>(), u, P.shape(), b);
        IMQ_LAUNCH_CHECK();
        launches += 2;
    }
    return launches;
}

template int fmm_apply_dz<float>(Plan &, const float *, float *, int, cudaStream_t);
template int fmm_apply_dz<double>(Plan &, const double *, double *, int, cudaStream_t);

}  // namespace imq
