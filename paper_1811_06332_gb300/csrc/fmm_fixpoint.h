// Leaf coordinates without FP64 arithmetic.  A coordinate x in [0, 1) is
// taken as the fixed-point integer X = floor(x * 2^62), read off the bits of
// the double with integer operations (exact when x >= 2^-10 or when x has no
// bits below 2^-62: an absolute error under 2^-62 otherwise).  Then the leaf
// index at depth d is X >> (62 - d) (exactly floor(x * 2^d)), and the offset
// from the leaf centre, X - (2 i + 1) 2^(61 - d), is an exact integer that
// fix62_to_float rounds to the nearest float (ties to even).  An FP64
// instruction holds a GB300 SM's FP64 pipe for 16 cycles, so the integer
// pipe does this part of the uniform tree build instead.
//
// Compiles as CUDA (host and device) and as plain C++ (the host test).
#pragma once
#include <stdint.h>
#include <string.h>

#ifdef __CUDACC__
#define FMM_HD __host__ __device__ __forceinline__
#else
#define FMM_HD inline
#endif

namespace fmm {

FMM_HD int fix_clz64(uint64_t a) {
#ifdef __CUDA_ARCH__
    return __clzll((long long)a);
#else
    return __builtin_clzll(a);
#endif
}

// X = floor(x * 2^62) for 0 <= x < 1 (+0 and subnormals give 0); false for
// x outside [0, 1), -0, NaN and infinities
FMM_HD bool fix62(double x, int64_t& X) {
    uint64_t u;
#ifdef __CUDA_ARCH__
    u = (uint64_t)__double_as_longlong(x);
#else
    memcpy(&u, &x, 8);
#endif
    const int e = (int)(u >> 52);          // sign bit and biased exponent
    if (e > 1022) return false;            // sign set, or x >= 1, inf, NaN
    if (e == 0) { X = 0; return true; }    // +0 and subnormals (below 2^-1022)
    const uint64_t m = (u & ((1ull << 52) - 1)) | (1ull << 52);   // x = m 2^(e - 1075)
    const int sh = e - 1013;               // X = m 2^(e - 1075 + 62)
    X = sh >= 0 ? (int64_t)(m << sh) : (sh > -64 ? (int64_t)(m >> -sh) : 0);
    return true;
}

// the float nearest to v 2^-62, ties to even (|v| < 2^63; the result is a
// normal float: the smallest nonzero |v| 2^-62 is 2^-62)
FMM_HD float fix62_to_float(int64_t v) {
    if (v == 0) return 0.f;
    const uint32_t sgn = v < 0 ? 0x80000000u : 0u;
    uint64_t a = v < 0 ? 0ull - (uint64_t)v : (uint64_t)v;
    const int lz = fix_clz64(a);
    a <<= lz;                                        // leading one at bit 63
    uint32_t mant = (uint32_t)(a >> 40);             // 24 bits with the leading one
    const uint64_t rem = a & ((1ull << 40) - 1), half = 1ull << 39;
    if (rem > half || (rem == half && (mant & 1u))) ++mant;   // a carry to 2^24 raises the exponent
    // |v| in [2^(63 - lz), 2^(64 - lz)): unbiased exponent of |v| 2^-62 is 1 - lz
    const uint32_t bits = sgn | (((uint32_t)(127 - lz) << 23) + mant);
    float f;
#ifdef __CUDA_ARCH__
    f = __uint_as_float(bits);
#else
    memcpy(&f, &bits, 4);
#endif
    return f;
}

// leaf index along one axis at depth d (0 <= d <= 61) and the FP32 offset
// of x from that leaf's centre, in units of the unit cube
FMM_HD int fix62_leaf(int64_t X, int d) { return (int)(X >> (62 - d)); }
FMM_HD float fix62_offset(int64_t X, int i, int d) {
    return fix62_to_float(X - ((int64_t)(2 * i + 1) << (61 - d)));
}

}  // namespace fmm
