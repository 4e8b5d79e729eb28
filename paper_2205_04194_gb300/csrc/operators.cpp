// Host FP64 construction of the translation operators, in the parity-reduced
// real layout described in imq_internal.h.
//
// The expansions follow the paper's Section 2.1-2.2: 1/|X - Y| is expanded in
// spherical harmonics (Eq. (7)); in the separated form Eq. (13) the source
// factor j_{n,m} and the target factor h_{n,m} are the regular and irregular
// solid harmonics.  The translations between centres are those of the fast
// multipole method (Greengard-Rokhlin).  With
//     U_n^m(v) = r^n P_n^m(cos th) e^{i m om} / (n+m)!
//     T_n^m(v) = (n-m)! P_n^m(cos th) e^{i m om} / r^{n+1}
// (m >= 0, no Condon-Shortley phase; X^{-m} = (-1)^m conj(X^m)) they read
//     M2M  M_n^m(P) = sum_{k,l} M_k^l(Q) conj(U_{n-k}^{m-l}(Z_Q - Z_P))
//     L2L  L_j^i(Q) = sum_{k,l} L_k^l(P) conj(U_{k-j}^{l-i}(C_Q - C_P))
//     M2L  L_k^l(B) = (-1)^k sum_{n,m} M_n^m(S) T_{n+k}^{m+l}(C_B - Z_S)
// Every operator is formed in complex arithmetic over all m in [-p, p] and
// then folded into real matrices acting on (Re, Im) of the m >= 0 slots,
// using M^{-m} = (-1)^m conj(M^m).
#include <cmath>
#include <complex>
#include <vector>

#include "imq_internal.h"

namespace imq {

using cd = std::complex<double>;

void Layout::build(int p_, int parity_) {
    p = p_;
    parity = parity_;
    slot_n.clear(); slot_m.clear(); slot_part.clear();
    re_slot.assign((p + 1) * (p + 1), -1);
    im_slot.assign((p + 1) * (p + 1), -1);
    for (int m = 0; m <= p; ++m) {
        for (int n = m + parity; n <= p; n += 2) {
            re_slot[n * (p + 1) + m] = (int)slot_n.size();
            slot_n.push_back(n); slot_m.push_back(m); slot_part.push_back(0);
            if (m > 0) {
                im_slot[n * (p + 1) + m] = (int)slot_n.size();
                slot_n.push_back(n); slot_m.push_back(m); slot_part.push_back(1);
            }
        }
    }
    K = (int)slot_n.size();
}

namespace {

// Ptilde_n^m(x) = sqrt((n-m)!/(n+m)!) P_n^m(x), 0 <= m <= n <= nmax, no phase.
std::vector<double> legendre_normalised(int nmax, double x) {
    std::vector<double> P((nmax + 1) * (nmax + 1), 0.0);
    auto at = [&](int n, int m) -> double & { return P[n * (nmax + 1) + m]; };
    const double s = std::sqrt(std::max(0.0, 1.0 - x * x));
    at(0, 0) = 1.0;
    for (int m = 1; m <= nmax; ++m) at(m, m) = at(m - 1, m - 1) * std::sqrt((2.0 * m - 1.0) / (2.0 * m)) * s;
    for (int m = 0; m < nmax; ++m) at(m + 1, m) = std::sqrt(2.0 * m + 1.0) * x * at(m, m);
    for (int m = 0; m <= nmax; ++m)
        for (int n = m + 2; n <= nmax; ++n)
            at(n, m) = ((2.0 * n - 1.0) * x * at(n - 1, m) -
                        std::sqrt((double)(n - 1) * (n - 1) - (double)m * m) * at(n - 2, m)) /
                       std::sqrt((double)n * n - (double)m * m);
    return P;
}

double log_s(int n, int m) {  // log sqrt((n+m)!(n-m)!)
    m = std::abs(m);
    return 0.5 * (std::lgamma(n + m + 1.0) + std::lgamma(n - m + 1.0));
}

// Harmonic tables for one vector, indexed [n][m + nmax], m in [-n, n].
struct Harm {
    int nmax;
    std::vector<cd> v;
    cd at(int n, int m) const {
        if (n < 0 || std::abs(m) > n) return cd(0, 0);
        return v[n * (2 * nmax + 1) + m + nmax];
    }
};

// Regular U_n^m (scaled by exp(log_scale)) and irregular T_n^m of vector (x, y, z).
// Returned quantities carry the normalisation without the s_nm factor:
//   reg:  r^n Ptilde e^{i m om}           (= U_n^m * s_nm)
//   irr:  Ptilde e^{i m om} / r^{n+1}     (= T_n^m / s_nm)
Harm harmonics(int nmax, double x, double y, double z, bool irregular) {
    Harm H;
    H.nmax = nmax;
    H.v.assign((nmax + 1) * (2 * nmax + 1), cd(0, 0));
    const double r = std::sqrt(x * x + y * y + z * z);
    const double ct = r > 0 ? z / r : 1.0;
    const double om = std::atan2(y, x);
    const auto P = legendre_normalised(nmax, ct);
    for (int n = 0; n <= nmax; ++n) {
        const double radial = irregular ? 1.0 / std::pow(r, n + 1) : std::pow(r, n);
        for (int m = 0; m <= n; ++m) {
            const cd val = radial * P[n * (nmax + 1) + m] * std::polar(1.0, m * om);
            H.v[n * (2 * nmax + 1) + m + nmax] = val;
            if (m > 0) H.v[n * (2 * nmax + 1) - m + nmax] = ((m & 1) ? -1.0 : 1.0) * std::conj(val);
        }
    }
    return H;
}

// Fold a complex coefficient function C(out_n, out_m, in_n, in_m) (signed m) into
// the real input-major K x K matrix op[in * K + out] on the parity-even layout.
template <class F>
void fold(const Layout &Lo, const Layout &Li, F coef, double *op) {
    const int K = Lo.K, p = Lo.p;
    for (int i = 0; i < Li.K * K; ++i) op[i] = 0.0;
    for (int k = 0; k <= p; ++k) {
        for (int l = 0; l <= k; ++l) {
            const int oRe = Lo.re_slot[k * (p + 1) + l];
            if (oRe < 0) continue;
            const int oIm = Lo.im_slot[k * (p + 1) + l];
            for (int n = 0; n <= p; ++n) {
                for (int m = 0; m <= n; ++m) {
                    const int iRe = Li.re_slot[n * (p + 1) + m];
                    if (iRe < 0) continue;
                    const int iIm = Li.im_slot[n * (p + 1) + m];
                    const cd T1 = coef(k, l, n, m);
                    if (m == 0) {
                        op[iRe * K + oRe] += T1.real();
                        if (oIm >= 0) op[iRe * K + oIm] += T1.imag();
                    } else {
                        const double sgn = (m & 1) ? -1.0 : 1.0;
                        const cd T2 = coef(k, l, n, -m);
                        const cd A = T1 + sgn * T2, B = T1 - sgn * T2;
                        op[iRe * K + oRe] += A.real();
                        op[iIm * K + oRe] += -B.imag();
                        if (oIm >= 0) {
                            op[iRe * K + oIm] += A.imag();
                            op[iIm * K + oIm] += B.real();
                        }
                    }
                }
            }
        }
    }
}

// quadrant q = 2*ybit + xbit; child centre - parent centre in units of the parent side
void quadrant_shift(int q, double *dx, double *dy) {
    *dx = (q & 1) ? 0.25 : -0.25;
    *dy = (q & 2) ? 0.25 : -0.25;
}

}  // namespace

void p2m_coefficients(const Layout &L, std::vector<double> &coef) {
    const auto P0 = legendre_normalised(L.p, 0.0);
    coef.resize(L.K);
    for (int s = 0; s < L.K; ++s) coef[s] = P0[L.slot_n[s] * (L.p + 1) + L.slot_m[s]];
}

void l2p_dz_coefficients(const Layout &Lo, std::vector<double> &coef) {
    // d/dz of conj(U_k^l(X - C)) is conj(U_{k-1}^l): in scaled form each odd slot (k, l)
    // contributes Lh_k^l sqrt((k+l)(k-l)) Ptilde_{k-1}^l(0) conj(w)^l |w|^{k-1-l} / h
    const auto P0 = legendre_normalised(Lo.p, 0.0);
    coef.resize(Lo.K);
    for (int s = 0; s < Lo.K; ++s) {
        const int k = Lo.slot_n[s], l = Lo.slot_m[s];
        coef[s] = std::sqrt((double)(k + l) * (double)(k - l)) * P0[(k - 1) * (Lo.p + 1) + l];
    }
}

void build_m2m_ops(const Layout &L, std::vector<double> &out) {
    // Parent side 1, child side 1/2.  Mh(P)_n^m = sum (s_nm / s_kl) 2^{-k} conj(U_{n-k}^{m-l}(t)) Mh(Q)_k^l
    const int K = L.K, p = L.p;
    out.assign(4 * (size_t)K * K, 0.0);
    for (int q = 0; q < 4; ++q) {
        double tx, ty;
        quadrant_shift(q, &tx, &ty);
        const Harm R = harmonics(p, tx, ty, 0.0, false);   // U * s
        auto coef = [&](int n, int m, int k, int l) -> cd {
            const int j = n - k, i = m - l;
            if (j < 0 || std::abs(i) > j) return cd(0, 0);
            const double sc = std::exp(log_s(n, m) - log_s(k, l) - log_s(j, i)) * std::pow(0.5, k);
            return sc * std::conj(R.at(j, i));
        };
        fold(L, L, coef, out.data() + (size_t)q * K * K);
    }
}

void build_l2l_ops(const Layout &L, std::vector<double> &out) {
    // Lh(Q)_j^i = sum (s_kl / s_ji) 2^{-j} conj(U_{k-j}^{l-i}(t)) Lh(P)_k^l, parent side 1
    const int K = L.K, p = L.p;
    out.assign(4 * (size_t)K * K, 0.0);
    for (int q = 0; q < 4; ++q) {
        double tx, ty;
        quadrant_shift(q, &tx, &ty);
        const Harm R = harmonics(p, tx, ty, 0.0, false);
        auto coef = [&](int j, int i, int k, int l) -> cd {
            const int dn = k - j, dm = l - i;
            if (dn < 0 || std::abs(dm) > dn) return cd(0, 0);
            const double sc = std::exp(log_s(k, l) - log_s(j, i) - log_s(dn, dm)) * std::pow(0.5, j);
            return sc * std::conj(R.at(dn, dm));
        };
        fold(L, L, coef, out.data() + (size_t)q * K * K);
    }
}

void build_m2l_ops(const Layout &Lo, const Layout &L, double h, double c, std::vector<double> &out) {
    // Lh_k^l = (-1)^k h^{k+n} s_{n+k,m+l} / (s_kl s_nm) [T_{n+k}^{m+l}(d) / s_{n+k,m+l}] Mh_n^m
    // d = C_B - Z_S = (-dx h, -dy h, c) for a source at box offset (dx, dy).
    const int K = L.K, Ko = Lo.K, p = L.p;
    out.assign((size_t)kOffsetClasses * K * Ko, 0.0);
    for (int k = 0; k < kOffsetClasses; ++k) {
        int dx, dy;
        offset_of_class(k, &dx, &dy);
        const double vx = -dx * h, vy = -dy * h, vz = c;
        const double r = std::sqrt(vx * vx + vy * vy + vz * vz);
        const Harm I = harmonics(2 * p, vx / r, vy / r, vz / r, true);   // unit vector: Ptilde e^{im om}
        auto coef = [&](int kk, int l, int n, int m) -> cd {
            const int j = n + kk, i = m + l;
            const double sc = std::exp(log_s(j, i) - log_s(kk, l) - log_s(n, m)) * std::pow(h / r, j) / r;
            return ((kk & 1) ? -1.0 : 1.0) * sc * I.at(j, i);
        };
        fold(Lo, L, coef, out.data() + (size_t)k * K * Ko);
    }
}

}  // namespace imq
