// Layout helpers of the M2L part on the CUDA cores that goes with the
// first-K-part tensor-core kernel (fmm_m2l_rest.cu): the multipole columns
// >= 48 and the matrix entries that reach them.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace fmm {

constexpr int RS_K0 = 48;                     // first multipole column left to this kernel
constexpr int RS_TX = 8, RS_TY = 16;         // target tile: 8 x 16 cells of one class
constexpr int RS_RX = RS_TX + 2, RS_RY = RS_TY + 2;   // source region

__host__ __device__ constexpr int rs_rank(int r) {
    int a = 0;
    while ((a + 1) * (a + 1) <= r) ++a;
    return a;
}
// rows with columns >= 48: ranks 0..p-6
__host__ __device__ constexpr int rs_rows(int p) { return p < 6 ? 0 : (p - 5) * (p - 5); }
// columns of row r above 47
__host__ __device__ constexpr int rs_cols(int p, int r) { return (p - rs_rank(r) + 1) * (p - rs_rank(r) + 1) - RS_K0; }
// a row's entries padded to a multiple of 4 (16-byte shared loads)
__host__ __device__ constexpr int rs_cpad(int p, int r) { return (rs_cols(p, r) + 3) / 4 * 4; }
__host__ __device__ constexpr int rs_roff(int p, int r) {
    int o = 0;
    for (int k = 0; k < r; ++k) o += rs_cpad(p, k);
    return o;
}
__host__ __device__ constexpr int rs_kstride(int p) { return rs_roff(p, rs_rows(p)); }
__host__ __device__ constexpr int rs_cstride(int p) { return ((p + 1) * (p + 1) - RS_K0 + 3) / 4 * 4; }

__device__ __forceinline__ void rs_cp16(void* dst, const void* src, bool ok) {
    // 16-byte asynchronous copy; zero fill (nothing read) when !ok
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(ok ? 16 : 0)
                 : "memory");
}

// d += a * b on two FP32 lanes at once (fma.rn.f32x2: each lane rounded as
// fmaf); the operands are 64-bit registers holding two floats, the lower
// address in the low half, as a 16-byte shared load delivers them
__device__ __forceinline__ void rs_ffma2(uint64_t& d, uint64_t a, uint64_t b) {
    asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(d) : "l"(a), "l"(b));
}

// acc[R0 + j] += sum_c kk[OFF + j pa + c] m[c] for the 2A + 1 rows of rank A
// (columns 48..48 + na - 1, stored padded with zeros to pa), over column
// pairs: the even and odd columns of a row sum in the two halves of acc; then
// the next rank.  m2 holds the column pairs of the source cell.  Every bound
// and index is a compile-time constant.
// Two source cells a and b (two targets) per call, sharing each entry load.
template <int P, int A, int R0, int OFF, int CS2, int NR>
__device__ __forceinline__ void rs_rank_rows2(const float* kk, const uint64_t (&ma)[CS2], const uint64_t (&mb)[CS2],
                                              uint64_t (&aa)[NR], uint64_t (&ab)[NR]) {
    if constexpr (A <= P - 6) {
        constexpr int na = (P - A + 1) * (P - A + 1) - RS_K0, pa = (na + 3) / 4 * 4;
#pragma unroll
        for (int j = 0; j < 2 * A + 1; ++j) {
#pragma unroll
            for (int c = 0; c < pa; c += 4) {
                const ulonglong2 kv = *(const ulonglong2*)(kk + OFF + j * pa + c);
                rs_ffma2(aa[R0 + j], kv.x, ma[c / 2]);
                rs_ffma2(ab[R0 + j], kv.x, mb[c / 2]);
                if (c + 2 < na) {
                    rs_ffma2(aa[R0 + j], kv.y, ma[c / 2 + 1]);
                    rs_ffma2(ab[R0 + j], kv.y, mb[c / 2 + 1]);
                }
            }
        }
        rs_rank_rows2<P, A + 1, R0 + 2 * A + 1, OFF + (2 * A + 1) * pa>(kk, ma, mb, aa, ab);
    }
}

}  // namespace fmm
