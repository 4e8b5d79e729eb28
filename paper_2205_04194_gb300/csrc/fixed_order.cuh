// Compile-time layout of the parity-reduced expansions (n + m even, m-major
// columns) for kernels specialised on the truncation order P: column m holds
// the terms n = m, m + 2, ... <= P; column 0 is real, the others (re, im).
#pragma once

namespace imq {

__host__ __device__ constexpr int cnt_col(int P, int m) { return (P - m) / 2 + 1; }     // complex terms of column m
__host__ __device__ constexpr int cbase(int P, int m) {                                  // first complex index of column m
    int s = 0;
    for (int mm = 0; mm < m; ++mm) s += cnt_col(P, mm);
    return s;
}
__host__ __device__ constexpr int rbase(int P, int m) {                                  // first real slot of column m
    int s = 0;
    for (int mm = 0; mm < m; ++mm) s += cnt_col(P, mm) * (mm ? 2 : 1);
    return s;
}
__host__ __device__ constexpr int ncplx(int P) { return cbase(P, P + 1); }

// complex index k -> (first complex index of its column, real slot of its term, m)
template <int P>
__device__ __forceinline__ void decode_term(int k, int &m, int &slot) {
    m = 0;
    int kb = 0, rb = 0;
#pragma unroll
    for (int mm = 1; mm <= P; ++mm)
        if (k >= cbase(P, mm)) {
            m = mm;
            kb = cbase(P, mm);
            rb = rbase(P, mm);
        }
    slot = rb + (k - kb) * (m ? 2 : 1);
}

}  // namespace imq
