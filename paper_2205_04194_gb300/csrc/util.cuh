// Small device/host helpers shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace imq {

// Exclusive prefix sum of n values on `s`; if d_total is non-null the grand
// total is written there (device memory).
template <class T>
void exclusive_scan(const T *d_in, T *d_out, int64_t n, T *d_total, cudaStream_t s);

// Per-device error word that kernels OR their DeviceError codes into.
int *device_error_word();

// Error word of imq_dense_matvec_noalloc on the current device (inside its fixed
// scratch array), or nullptr if that entry point has not run on this device.
int *noalloc_error_word();

// Synchronise `s`, read and clear the device error words (the shared one and
// the allocation-free dense product's); throws IMQ_TIMEOUT if a bounded wait
// ran out since the last check (the affected results are invalid).
void check_device_errors(cudaStream_t s);

// Launch one kernel whose bounded wait can never complete, then check the error
// word: throws IMQ_TIMEOUT when the timeout path works.
void selftest_wait_timeout(cudaStream_t s);

inline unsigned blocks_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

}  // namespace imq
