// Building blocks of the tensor-core M2L kernels (tcgen05, TMA, mbarrier),
// shared by the per-offset-matrix kernel (fmm_m2l_tc.cu) and the kernel that
// builds the offset matrices on chip (fmm_m2l_tcgen.cu).
#pragma once
#include <cuda.h>
#include <stdint.h>

namespace fmm {

constexpr int TC_K = 96;                       // padded multipole components (K)
constexpr int TC_N = 96;                       // padded local components (N)
constexpr int TC_CH = 12;                      // 16-byte chunks of one A row per K-part
constexpr int TC_PSTEPS = 6;                   // K-steps (32 bytes of a row) per K-part
constexpr int TC_NCH = TC_N / 16;              // N-chunks of at least 16 local components
constexpr long TC_SPIN = 1L << 24;             // bounded waits

struct TcMaps {
    CUtensorMap hi[8];
    CUtensorMap lo[8];
};

// Source slabs (levels with at least 16 cells per class and axis).  A CTA
// owns a column of 8 x 16 x 1 target cells of one class.  For one source
// class and one z shift dz in {-1, 0, 1}, the sources of the (up to 9)
// offsets with x, y shifts dx, dy in {-1, 0, 1} all lie in one slab of
// 10 x 18 x 1 cells, stored [j][chunk][i][16 bytes]: the A operand of offset
// (dx, dy) starts at row i = dx + 1 of group j = dy + 1.  Core matrices stay
// 8 consecutive 16-byte rows; LBO (next chunk along K) is 160 bytes and SBO
// (next group of 8 rows) 1920 bytes.
constexpr int SL_I = 10, SL_J = 18;
constexpr int SL_BYTES = SL_I * TC_CH * SL_J * 16;   // 34560: one slab operand (hi or lo) of one K-part

struct alignas(64) TcLevelMaps {
    TcMaps slab;    // box 10 x 18 x 1 cells, one K-part
    TcMaps tall;    // BF16 only: box 10 x (TY + 2) x 1 cells, half a K-part (fmm_m2l_tct.cu)
};

static __device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Bounded parity wait on an mbarrier; after `spin` polls it records `code`
// in the error word and returns false.
static __device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* err, int code,
                                                 long spin = TC_SPIN) {
    for (long it = 0; it < spin; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    atomicExch(err, code);
    return false;
}

// Shared-memory matrix descriptor, K-major, no swizzle: core matrices of
// 8 rows x 16 bytes stored as 128 contiguous bytes; LBO = distance between
// core matrices along K, SBO = distance between 8-row groups.
static __device__ __forceinline__ uint64_t make_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version
    return d;                // layout type 0: no swizzle
}

// Instruction descriptor, both operands K-major, F32 accumulator:
// kind::f16 with BF16 x BF16 (format 1), or kind::tf32 with TF32 x TF32
// (format 2).
__host__ __device__ constexpr uint32_t make_idesc(int tf, int M, int N) {
    return (1u << 4)                                  // D format F32
           | ((tf ? 2u : 1u) << 7)                    // A format
           | ((tf ? 2u : 1u) << 10)                   // B format
           | ((uint32_t)(N >> 3) << 17)               // N
           | ((uint32_t)(M >> 4) << 24);              // M
}

template <int TF>
static __device__ __forceinline__ void tc_mma(uint32_t dcol, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
    if constexpr (TF)
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dcol),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
            : "memory");
    else
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dcol),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
            : "memory");
}

// 32 consecutive FP32 columns of this thread's TMEM lane (32x32b shape)
static __device__ __forceinline__ void tmem_ld32(uint32_t ta, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
          "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(ta));
}

// 16 consecutive FP32 columns of this thread's TMEM lane (32x32b shape)
static __device__ __forceinline__ void tmem_ld16(uint32_t ta, uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(ta));
}

}  // namespace fmm
