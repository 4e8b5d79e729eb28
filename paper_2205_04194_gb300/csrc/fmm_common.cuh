// Device helpers shared by the expansion kernels (expansions.cu, dz.cu).
#pragma once

#include <type_traits>

#include "imq_internal.h"

namespace imq {

constexpr int kMaxCol = 10;   // (IMQ_MAX_P / 2) + 1 coefficients per m-column

__device__ __forceinline__ int col_count(int m, int p, int par) {
    // coefficients (n, m), n = m + par, m + par + 2, ... <= p, of column m
    return p - m - par >= 0 ? (p - m - par) / 2 + 1 : 0;
}

__device__ __forceinline__ int col_base(int m, int p, int par = 0) {
    // first slot of column m in the m-major layout of the given parity
    int s = 0;
    for (int mm = 0; mm < m; ++mm) s += col_count(mm, p, par) * (mm ? 2 : 1);
    return s;
}

template <class T>
__device__ __forceinline__ T box_side(double S, int lev) {
    return (T)(S / (double)(1 << lev));
}

// offset of sorted point i from the centre of the box with centre cb,
// where leafc is the centre of the leaf that holds i.
template <class T>
__device__ __forceinline__ void point_offset(int i, const float2 *loc, const double2 *pos, double2 cb, double2 leafc,
                                             T &x, T &y) {
    if constexpr (std::is_same<T, float>::value) {
        const float2 l = loc[i];
        x = l.x + (float)(leafc.x - cb.x);
        y = l.y + (float)(leafc.y - cb.y);
    } else {
        const double2 q = pos[i];
        x = q.x - cb.x;
        y = q.y - cb.y;
    }
}

template <class T>
__device__ __forceinline__ T rsq(T v) {
    if constexpr (std::is_same<T, float>::value) return rsqrtf(v);
    else return 1.0 / sqrt(v);
}

// ------------------------------------------------------------------ recurrence tables
// tab2[n*(p+1)+m] = sqrt((n-1)^2 - m^2), tabi[n*(p+1)+m] = 1/sqrt(n^2 - m^2) (0 where undefined)
template <class T>
__device__ __forceinline__ void fill_recurrence_tables(T *tab2, T *tabi, int p) {
    for (int idx = threadIdx.x; idx < (p + 1) * (p + 1); idx += blockDim.x) {
        const int n = idx / (p + 1), m = idx - n * (p + 1);
        const int a = (n - 1) * (n - 1) - m * m, b = n * n - m * m;
        tab2[idx] = (n >= 1 && a > 0) ? sqrt((T)a) : (T)0;
        tabi[idx] = b > 0 ? (T)1 / sqrt((T)b) : (T)0;
    }
}

}  // namespace imq
