// Device helpers shared by the kernels of libxs (CUDA path only).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace xs {

// Bits of the device error word (one int per context).
enum : int {
    kDevErrTimeout = 1,    // a bounded wait expired
    kDevErrNonFinite = 2,  // a non-finite form factor, or a position non-finite or more than 2^18 cells out
    kDevErrBounds = 4,     // a bounds check of the checked build failed (the access was skipped)
};

// 3x3 inverse cell matrix (row-major), passed by value to kernels.
struct Mat3 {
    double a[9];
};

// Per-atom record produced by the phase kernel: the fractional coordinate of
// each axis as a 32-bit turn count U = round(frac(s) * 2^32) mod 2^32, and the
// form factor's bits.  With integer Miller indices n, n*U mod 2^32 is the
// phase n*s in turns reduced modulo one turn exactly (Sec. 3.1: for q on the
// reciprocal lattice the periodic image of an atom does not matter).
struct AtomRec {
    uint32_t ux, uy, uz;
    float f;
};

__device__ __forceinline__ void set_dev_error(int* err, int bit) {
    if (err) atomicOr(err, bit);
}

// Bounds checks of the checked build (compiled with -DXS_BOUNDS_CHECK): a
// failed check sets kDevErrBounds in the device error word and the caller
// skips the access; no assert, no trap.  In the normal build the condition
// is not evaluated.
#ifdef XS_BOUNDS_CHECK
__device__ __forceinline__ bool xs_in_bounds(int* err, bool ok) {
    if (!ok) set_dev_error(err, kDevErrBounds);
    return ok;
}
#define XS_IN_BOUNDS(err, cond) ::xs::xs_in_bounds((err), (cond))
#else
#define XS_IN_BOUNDS(err, cond) true
#endif

// Phase factor exp(+i 2 pi P / 2^32) for a 32-bit turn count P.
__device__ __forceinline__ void phase_to_cs(uint32_t P, float& c, float& s) {
    float x = (float)(int32_t)P * 0x1p-31f;  // P/2^31 in [-1, 1): angle = pi * x
    sincospif(x, &s, &c);
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

}  // namespace xs
