// Offset-grouped M2L on the 5th-generation tensor cores (Eq. M2L regrouped),
// with each offset's matrix precomputed in global memory and streamed by
// bulk copies (the streamed-matrix kernel; fmm_m2l_tcgen.cu holds the
// kernel that builds the matrices on chip, a second autotuner candidate of
// the BF16 form).  This file also holds the operand split of the
// multipoles and the TMA tensor maps, which both kernels use.
//
// On a uniform level, every target cell of one parity class sees the same
// 189 integer offsets o, and all pairs with one offset share one matrix
//     Kt_o(n, m) = D_{n+m}(-o)/m!      (cell units, |n| + |m| <= p)
// so M2L is a sum of dense products  Lt[T, :] += Mt[T + o, :] . Kt_o^T.
// Per CTA: a column of 128 target cells (8 x 16 x 1 in one class)
// accumulates over all 189 offsets in TMEM:
//     D[128 cells x 96] += A_o[128 cells x 96] . B_o[96 x 96]^T
// with A_o the source multipoles (reduced traceless representative, padded
// 81 -> 96) read from a source slab that a 5-D TMA tensor load brings in
// once for up to 9 offsets (out-of-range cells zero-filled at the grid
// boundary), and B_o the precomputed matrix fetched by a bulk copy.
// Split precision: x = hi + lo, three MMAs per K-step (hi.hi + hi.lo +
// lo.hi), FP32 accumulation in TMEM, FP64 write-out.  Two operand types
// share the kernel: BF16 (kind::f16, 16 columns per K-step) and TF32
// (kind::tf32, 8 columns per K-step).  A K-step is 32 bytes of a row in
// both, so the shared-memory layouts agree byte for byte; TF32 rows are
// twice as long and are streamed in two K-parts.
//
// Roles: warp 0 lane 0 issues copies, lane 0 of 2 or 4 warps issues
// tcgen05.mma (each into its own TMEM accumulator), warps 2..5 drain and
// add the accumulators (each reads its lane quadrant).  Every wait is
// bounded and reports a timeout through an error word instead of hanging.
#include <cstdlib>
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include "fmm_internal.h"
#include "fmm_tc_common.cuh"

namespace fmm {

constexpr int TC_PMAX = TC_N * TC_PSTEPS * 32; // 18432: bound on one part block (hi or lo) of a matrix
constexpr int TC_TMEM_COLS = 128;             // one accumulator (96 columns used)

// The matrix of one offset is block-triangular in rank (|n| + |m| <= p), so
// local components are processed in N-chunks: chunk j (rows cw j .. cw j +
// cw - 1, lowest rank a_j) only multiplies multipole components of rank
// <= p - a_j, i.e. the first kch[j] K-steps.  Part t of a matrix holds the
// K-steps 6t .. 6t + 5: chunk j contributes nk[t][j] of them, as cw rows x
// 32 nk[t][j] bytes in the K-major core-matrix layout (SBO = 256 nk[t][j]).
// One offset's matrix is stored as {part 0 hi, part 0 lo, part 1 hi, ...}.
struct TcChunks {
    int tf;                  // 0: BF16 operands, 1: TF32 operands
    int np;                  // K-parts per offset (1 for BF16; 1 or 2 for TF32, by p)
    int cw;                  // chunk width (local components per chunk, N of one MMA)
    int nch;                 // chunks holding real rows
    int kch[TC_NCH];         // K-steps of chunk j
    int nk[2][TC_NCH];       // K-steps of chunk j inside part t
    int boff[2][TC_NCH];     // byte offset of chunk j inside the block of part t
    int pbytes[2];           // bytes of part t's block (hi or lo), a multiple of 1024
    int poff[2];             // byte offset of part t's hi block inside one offset's matrix
    int mbytes;              // bytes of one offset's matrix (every part, hi and lo)
    int bstage;              // bytes of one matrix stage: 2 x largest part block
    int nbst;                // matrix stages (2 or 4)
    int niss;                // MMA-issuing warps (2 or 4; divides nbst)
};

// Two rings: 2 slab buffers ({hi, lo} of one K-part) and nbst matrix
// stages.  The producer (warp 0) walks (source class, dz, part) slabs and,
// after each slab, the matrices of its offsets.  The MMAs of one offset are
// small (N <= 96), and their cost is set by their issue more than by their
// tensor work, so NISS warps (1 and 6, 7, ...) issue round-robin over the
// offsets, each into its own TMEM accumulator of 128 columns; the epilogue
// (warps 2..5) adds them.  A slab is freed when every issuer has committed
// its MMAs.  NISS divides nbst, so every matrix stage has one issuer, which
// waits on its phases in order (a parity wait cannot tell phases two apart).
template <int NISS>
constexpr int sl_threads() { return 32 * (5 + NISS); }
template <int TF, int NISS>
__global__ void __launch_bounds__(sl_threads<NISS>(), 1)
k_m2l_tc_slab(const __grid_constant__ TcMaps maps, const TcChunks ch, int l, int nrows,
              const unsigned char* __restrict__ Kmat, double* __restrict__ Lt, int64_t ncell, int* __restrict__ err,
              float* __restrict__ Lt32) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* bring = smem + 4 * SL_BYTES;
    uint64_t* bars = (uint64_t*)(bring + ch.nbst * ch.bstage);
    uint64_t* sfull = bars;        // [2]
    uint64_t* sempty = bars + 2;   // [2]
    uint64_t* bfull = bars + 4;    // [4]
    uint64_t* bempty = bars + 8;   // [4]
    uint64_t* done = bars + 12;
    uint32_t* tslot = (uint32_t*)(bars + 13);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int hs = 1 << (l - 1);
    const int nti = hs / 8, ntj = hs / 16;
    const int tpc = nti * ntj * hs;
    const int cls = blockIdx.x / tpc, t = blockIdx.x % tpc;
    const int ti = t % nti, tj = (t / nti) % ntj, tk = t / (nti * ntj);
    const int cx = cls & 1, cy = (cls >> 1) & 1, cz = cls >> 2;
    if (ch.niss != NISS || ch.nbst % NISS != 0 || ch.nbst > 4) {   // launch/config mismatch: no barrier is used
        if (threadIdx.x == 0) atomicExch(err, 17);
        return;
    }

    if (threadIdx.x == 0) {
        for (int b = 0; b < 2; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&sfull[b])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&sempty[b])), "r"(NISS));
        }
        for (int b = 0; b < ch.nbst; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bfull[b])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bempty[b])));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(done)), "r"(NISS));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(NISS * TC_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;

    if (warp == 0 && lane == 0) {
        // ---------------- producer ----------------
        int sl = 0, bt = 0;
        bool ok = true;
        for (int sc = 0; sc < 8 && ok; ++sc) {
            const int sx = sc & 1, sy = (sc >> 1) & 1, sz = sc >> 2;
            for (int dz = -1; dz <= 1 && ok; ++dz) {
                if (tk + dz < 0 || tk + dz >= hs) continue;   // plane outside the grid: no sources
                const int oz = 2 * dz + sz - cz;
                for (int pt = 0; pt < ch.np && ok; ++pt) {
                    const int buf = sl & 1;
                    if (!(ok = mbar_wait(smem_u32(&sempty[buf]), ((uint32_t)(sl >> 1) & 1u) ^ 1u, err, 11))) break;
                    const uint32_t fb = smem_u32(&sfull[buf]);
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb),
                                 "r"(2 * SL_BYTES)
                                 : "memory");
                    unsigned char* st = smem + buf * 2 * SL_BYTES;
                    const int c1 = 8 * ti - 1, c3 = 16 * tj - 1, c4 = tk + dz;
                    asm volatile(
                        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                        " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(smem_u32(st)),
                        "l"((uint64_t)&maps.hi[sc]), "r"(0), "r"(c1), "r"(TC_CH * pt), "r"(c3), "r"(c4), "r"(fb)
                        : "memory");
                    asm volatile(
                        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                        " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(smem_u32(st + SL_BYTES)),
                        "l"((uint64_t)&maps.lo[sc]), "r"(0), "r"(c1), "r"(TC_CH * pt), "r"(c3), "r"(c4), "r"(fb)
                        : "memory");
                    ++sl;
                    for (int dy = -1; dy <= 1 && ok; ++dy) {
                        const int oy = 2 * dy + sy - cy;
                        for (int dx = -1; dx <= 1; ++dx) {
                            const int ox = 2 * dx + sx - cx;
                            if (ox >= -1 && ox <= 1 && oy >= -1 && oy <= 1 && oz >= -1 && oz <= 1) continue;
                            const int bs = bt % ch.nbst;
                            if (!(ok = mbar_wait(smem_u32(&bempty[bs]), ((uint32_t)(bt / ch.nbst) & 1u) ^ 1u, err,
                                                 12)))
                                break;
                            const uint32_t bb = smem_u32(&bfull[bs]);
                            const int nb = 2 * ch.pbytes[pt];
                            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bb), "r"(nb)
                                         : "memory");
                            const int ridx = (3 - oz) * 49 + (3 - oy) * 7 + (3 - ox);   // r = -o
                            const unsigned char* kb = Kmat + (int64_t)ridx * ch.mbytes + ch.poff[pt];
                            asm volatile(
                                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
                                "[%3];" ::"r"(smem_u32(bring + bs * ch.bstage)),
                                "l"((uint64_t)kb), "r"(nb), "r"(bb)
                                : "memory");
                            ++bt;
                        }
                    }
                }
            }
        }
        // drain: every issued copy has landed before the CTA may exit
        for (int k = sl > 2 ? sl - 2 : 0; k < sl; ++k)
            mbar_wait(smem_u32(&sfull[k & 1]), (uint32_t)(k >> 1) & 1u, err, 13);
        for (int k = bt > ch.nbst ? bt - ch.nbst : 0; k < bt; ++k)
            mbar_wait(smem_u32(&bfull[k % ch.nbst]), (uint32_t)(k / ch.nbst) & 1u, err, 13);
    } else if ((warp == 1 || warp >= 6) && lane == 0) {
        // ---------------- MMA issuers ----------------
        const int w = warp == 1 ? 0 : warp - 5;
        const uint32_t dbase = tmem + (uint32_t)(w * TC_TMEM_COLS);
        const uint32_t idesc = make_idesc(TF, 128, ch.cw);
        int sl = 0, bt = 0;
        bool ok = true, first = true;
        for (int sc = 0; sc < 8 && ok; ++sc) {
            const int sx = sc & 1, sy = (sc >> 1) & 1, sz = sc >> 2;
            for (int dz = -1; dz <= 1 && ok; ++dz) {
                if (tk + dz < 0 || tk + dz >= hs) continue;
                const int oz = 2 * dz + sz - cz;
                for (int pt = 0; pt < ch.np && ok; ++pt) {
                    const int buf = sl & 1;
                    if (!(ok = mbar_wait(smem_u32(&sfull[buf]), (uint32_t)(sl >> 1) & 1u, err, 14))) break;
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t sbase = smem_u32(smem + buf * 2 * SL_BYTES);
                    for (int dy = -1; dy <= 1 && ok; ++dy) {
                        const int oy = 2 * dy + sy - cy;
                        for (int dx = -1; dx <= 1; ++dx) {
                            const int ox = 2 * dx + sx - cx;
                            if (ox >= -1 && ox <= 1 && oy >= -1 && oy <= 1 && oz >= -1 && oz <= 1) continue;
                            const int mine = bt % NISS == w;
                            const int bs = bt % ch.nbst;
                            ++bt;
                            if (!mine) continue;
                            if (!(ok = mbar_wait(smem_u32(&bfull[bs]), (uint32_t)((bt - 1) / ch.nbst) & 1u, err, 15)))
                                break;
                            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                            const uint32_t bbase = smem_u32(bring + bs * ch.bstage);
                            const uint32_t aoff = (uint32_t)(((dy + 1) * TC_CH * SL_I + (dx + 1)) * 16);
                            // descriptors of K-step 0; a K-step adds 320 bytes (A) or 256 bytes (B),
                            // i.e. 20 or 16 in the address field (no carry: shared addresses < 2^18)
                            const uint64_t ah = make_desc(sbase + aoff, SL_I * 16, TC_CH * SL_I * 16);
                            const uint64_t al = make_desc(sbase + SL_BYTES + aoff, SL_I * 16, TC_CH * SL_I * 16);
                            for (int j = 0; j < ch.nch; ++j) {
                                const int nk = ch.nk[pt][j];
                                const uint32_t dcol = dbase + (uint32_t)(ch.cw * j);
                                const uint64_t bh = make_desc(bbase + ch.boff[pt][j], 128, 256u * nk);
                                const uint64_t bl = make_desc(bbase + ch.pbytes[pt] + ch.boff[pt][j], 128, 256u * nk);
                                // the first offset of each issuer (part 0) holds a K-step of every chunk
                                tc_mma<TF>(dcol, ah, bh, idesc, first ? 0u : 1u);
                                for (int ks = 1; ks < nk; ++ks) tc_mma<TF>(dcol, ah + 20 * ks, bh + 16 * ks, idesc, 1u);
                                for (int ks = 0; ks < nk; ++ks) tc_mma<TF>(dcol, ah + 20 * ks, bl + 16 * ks, idesc, 1u);
                                for (int ks = 0; ks < nk; ++ks) tc_mma<TF>(dcol, al + 20 * ks, bh + 16 * ks, idesc, 1u);
                            }
                            first = false;
                            asm volatile(
                                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                    smem_u32(&bempty[bs]))
                                : "memory");
                        }
                    }
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                     smem_u32(&sempty[buf]))
                                 : "memory");
                    ++sl;
                }
            }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(done))
                     : "memory");
    } else if (warp >= 2 && warp <= 5) {
        // ---------------- epilogue: TMEM (NISS accumulators) -> FP64 L ----------------
        bool ok = true;
        if (lane == 0) ok = mbar_wait(smem_u32(done), 0u, err, 16);
        ok = __shfl_sync(0xffffffffu, ok, 0);
        __syncwarp();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int q = warp & 3;
        const int row = q * 32 + lane;
        const int i = row & 7, j = row >> 3;
        const int64_t h3 = (int64_t)hs * hs * hs;
        const int64_t tg = (int64_t)cls * h3 + ((int64_t)tk * hs + (16 * tj + j)) * hs + (8 * ti + i);
#pragma unroll 1
        for (int cb = 0; cb < TC_N / 32; ++cb) {
            const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(cb * 32);
            double acc[32];
            uint32_t v[32];
            tmem_ld32(ta, v);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int e = 0; e < 32; ++e) acc[e] = (double)__uint_as_float(v[e]);
#pragma unroll 1
            for (int w = 1; w < NISS; ++w) {
                tmem_ld32(ta + (uint32_t)(w * TC_TMEM_COLS), v);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int e = 0; e < 32; ++e) acc[e] += (double)__uint_as_float(v[e]);
            }
            if (ok) {
#pragma unroll
                for (int e = 0; e < 32; ++e) {
                    const int n = cb * 32 + e;
                    if (n < nrows) {
                        if (Lt32) Lt32[(int64_t)n * ncell + tg] = (float)acc[e];
                        else Lt[(int64_t)n * ncell + tg] = acc[e];
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(NISS * TC_TMEM_COLS));
    }
}

// ---------------------------------------------------------------------------
// Operand preparation
// ---------------------------------------------------------------------------
// Split of an FP64 value into hi + lo of the operand type.  BF16 rounds to
// nearest even (the CUDA conversion, from the value rounded to FP32); TF32 (a 32-bit container whose low 13
// mantissa bits are zero) rounds the FP32 value to nearest, ties away from
// zero, on the magnitude bits.  Both parts are exact in the operand type, so
// the tensor core reads them without further rounding.
__device__ __forceinline__ uint32_t tf32_round(float v) {
    return (__float_as_uint(v) + 0x1000u) & 0xFFFFE000u;
}
template <int TF>
struct TcSplit;
template <>
struct TcSplit<0> {
    using T = __nv_bfloat16;
    // through FP32: one conversion from FP64 (this part's FP64 rate is 1/64
    // of FP32), then hi = x rounded to BF16 and lo = the rest, whose FP32
    // difference is exact; hi + lo keeps 16 bits of x, far above the 24 of
    // the FP32 rounding
    static __device__ __forceinline__ void split(double x, T& h, T& l) { split32((float)x, h, l); }
    static __device__ __forceinline__ void split32(float xf, T& h, T& l) {
        h = __float2bfloat16_rn(xf);
        l = __float2bfloat16_rn(xf - __bfloat162float(h));
    }
};
template <>
struct TcSplit<1> {
    using T = uint32_t;
    // as for BF16: one conversion, the rest in FP32
    static __device__ __forceinline__ void split(double x, T& h, T& l) { split32((float)x, h, l); }
    static __device__ __forceinline__ void split32(float xf, T& h, T& l) {
        h = tf32_round(xf);
        l = tf32_round(xf - __uint_as_float(h));
    }
};

// Multipoles of one level (FP64, [ncoef][ncell], parity-class numbering) ->
// hi/lo operands in the TMA layout [class][k][j][chunk][i][16 bytes]
// (components padded to 96; 8 BF16 or 4 TF32 per 16-byte chunk); with
// `scale` each component m is multiplied by 1/m! first (the operand of the
// kernel whose offset matrices hold D_{n+m} without the 1/m! weight).  One
// thread per (cell, chunk): blockIdx.y is the chunk, the cell index splits
// into class and (i, j, k) by shifts (the class grid side is a power of 2).
// M32 (when given, and without scale): the plan's FP32 copy of the same
// multipoles, read instead of M (the split starts from the FP32 value either
// way, so the operands are the same).
template <int TF>
__global__ void k_tc_split_m(int l, int nc, int scale, const double* __restrict__ M, void* __restrict__ hi_,
                             void* __restrict__ lo_, const float* __restrict__ M32) {
    using T = typename TcSplit<TF>::T;
    constexpr int EPC = 16 / (int)sizeof(T);        // elements per 16-byte chunk
    constexpr int NCH = TC_K / EPC;                 // chunks per row
    const int lh = l - 1, hs = 1 << lh, mask = hs - 1;
    const int ncell = 8 << (3 * lh);
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= ncell) return;
    const int c = blockIdx.y;
    const int i = idx & mask, j = (idx >> lh) & mask, k = (idx >> (2 * lh)) & mask, cls = idx >> (3 * lh);
    __align__(16) T vh[EPC], vl[EPC];
#pragma unroll
    for (int e = 0; e < EPC; ++e) {
        const int m = EPC * c + e;
        if (M32) {
            TcSplit<TF>::split32(m < nc ? M32[(int64_t)m * ncell + idx] : 0.f, vh[e], vl[e]);
            continue;
        }
        double x = m < nc ? M[(int64_t)m * ncell + idx] : 0.0;
        if (scale && m < nc) x *= c_invfact[c_tl_idx[m][0]] * c_invfact[c_tl_idx[m][1]] * c_invfact[c_tl_idx[m][2]];
        TcSplit<TF>::split(x, vh[e], vl[e]);
    }
    const int64_t o = ((((int64_t)cls * hs + k) * hs + j) * NCH + c) * hs + i;
    *(uint4*)((unsigned char*)hi_ + o * 16) = *(const uint4*)vh;
    *(uint4*)((unsigned char*)lo_ + o * 16) = *(const uint4*)vl;
}

// Kt_r(n, m) = D_{n+m}(r)/m! (traceless basis, reduced multipole columns),
// zero outside |n| + |m| <= p and in the padding, split into hi/lo and
// stored per offset as parts of N-chunks: 16-byte column group c lies in
// K-step c/2 of part t = (c/2)/6; chunk j's rows rr at byte
// (rr/8) 256 nk[t][j] + (c - 12 t) 128 + (rr%8) 16 inside its block.  One
// thread per (offset, row, 16-byte column group).
template <int TF>
__global__ void k_tc_build_b(int p, int nc, const TcChunks ch, const double* __restrict__ Dtab,
                             unsigned char* __restrict__ B) {
    using T = typename TcSplit<TF>::T;
    constexpr int EPC = 16 / (int)sizeof(T);
    constexpr int NCH = TC_K / EPC;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)343 * TC_N * NCH) return;
    const int r = (int)(t / (TC_N * NCH));
    const int n = (int)((t / NCH) % TC_N), c = (int)(t % NCH);
    const int j = n / ch.cw, rr = n % ch.cw;
    const int step = c / 2, pt = step / TC_PSTEPS;
    if (j >= ch.nch || step >= ch.kch[j]) return;
    const int ns = ns_of(p);
    __align__(16) T vh[EPC], vl[EPC];
#pragma unroll
    for (int e = 0; e < EPC; ++e) {
        const int m = EPC * c + e;
        double v = 0.0;
        if (n < nc && m < nc) {
            const int nx = c_tl_idx[n][0], ny = c_tl_idx[n][1], nz = c_tl_idx[n][2];
            const int mx = c_tl_idx[m][0], my = c_tl_idx[m][1], mz = c_tl_idx[m][2];
            if (nx + ny + nz + mx + my + mz <= p)
                v = Dtab[(int64_t)r * ns + pos_sym(nx + mx, ny + my, nz + mz)] * c_invfact[mx] * c_invfact[my] *
                    c_invfact[mz];
        }
        TcSplit<TF>::split(v, vh[e], vl[e]);
    }
    const int64_t boff = ch.poff[pt] + ch.boff[pt][j] + (rr / 8) * 256 * ch.nk[pt][j] +
                         (c - 2 * TC_PSTEPS * pt) * 128 + (rr % 8) * 16;   // bytes
    unsigned char* bh = B + (int64_t)r * ch.mbytes;
    *(uint4*)(bh + boff) = *(const uint4*)vh;
    *(uint4*)(bh + ch.pbytes[pt] + boff) = *(const uint4*)vl;
}

// Self-test of the bounded wait: one mbarrier expecting one arrival; with
// `arrive` thread 0 arrives before waiting, otherwise nothing ever arrives
// and the wait gives up after `spin` polls, records code 99 and returns.
__global__ void k_wait_selftest(long spin, int arrive, int* err) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (arrive) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&bar)) : "memory");
        mbar_wait(smem_u32(&bar), 0u, err, 99, spin);
    }
}

int wait_selftest(long spin, int arrive, int* err, cudaStream_t s) {
    k_wait_selftest<<<1, 32, 0, s>>>(spin, arrive, err);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

int tc_supported(int p, int basis) { return basis == 1 && p >= 1 && ncoef_of(p, basis) <= TC_K; }
// bytes of the per-offset matrices (any chunk width) of the streamed-matrix kernel
size_t tc_mat_bytes(int tf) { return (size_t)343 * 2 * TC_PMAX * (tf ? 2 : 1); }
int tc_elem_bytes(int tf) { return tf ? 4 : 2; }

// Chunk width: the N of one MMA.  Wider chunks issue fewer, larger MMAs;
// narrower ones skip more of the zero triangle and leave room for four
// matrix stages (four issuers).  Measured best at p = 8: 48 for BF16, 32
// for TF32; the autotuner times the candidates.  For the layout
// diagnostics, FMM_TC_CHUNK (16, 32, 48 or 96) overrides the default.
int tc_default_cw(int tf) { return tf ? 32 : 48; }
static int tc_chunk_width_env(int tf) {
    if (const char* e = getenv("FMM_TC_CHUNK")) {
        const int v = atoi(e);
        if (v == 16 || v == 32 || v == 48 || v == 96) return v;
    }
    return tc_default_cw(tf);
}

static TcChunks tc_chunks(int p, int tf, int cw) {
    TcChunks c{};
    const int nc = ncoef_of(p, 1);
    const int cps = tf ? 8 : 16;   // columns per K-step
    c.tf = tf;
    c.cw = cw;
    c.nch = (nc + c.cw - 1) / c.cw;
    for (int j = 0; j < c.nch; ++j) {
        const int r0 = c.cw * j;
        const int a = fmm_tl_idx[r0][0] + fmm_tl_idx[r0][1] + fmm_tl_idx[r0][2];   // lowest rank in chunk
        const int cols = (p - a + 1) * (p - a + 1);
        c.kch[j] = (cols + cps - 1) / cps;
    }
    // chunk 0 (rank 0) needs the most K-steps; parts beyond it would be empty
    c.np = (c.kch[0] + TC_PSTEPS - 1) / TC_PSTEPS;
    int pbmax = 0, off_all = 0;
    for (int pt = 0; pt < c.np; ++pt) {
        int off = 0;
        for (int j = 0; j < TC_NCH; ++j) {
            const int nk = j < c.nch ? c.kch[j] - TC_PSTEPS * pt : 0;
            c.nk[pt][j] = nk < 0 ? 0 : nk > TC_PSTEPS ? TC_PSTEPS : nk;
            c.boff[pt][j] = off;
            off += 32 * c.cw * c.nk[pt][j];
        }
        c.pbytes[pt] = (off + 1023) / 1024 * 1024;
        c.poff[pt] = off_all;
        off_all += 2 * c.pbytes[pt];
        pbmax = c.pbytes[pt] > pbmax ? c.pbytes[pt] : pbmax;
    }
    c.mbytes = off_all;
    c.bstage = 2 * pbmax;
    const int nb = (227 * 1024 - 1280 - 4 * SL_BYTES) / c.bstage;   // at least 2: bstage <= 2 TC_PMAX
    c.nbst = nb >= 4 ? 4 : 2;
    c.niss = c.nbst;
    return c;
}

// Host-side layout of the kernel for (p, operand type), for diagnostics:
// cw, nch, np, nbst, niss, bstage, mbytes, shared bytes, kch[6], nk[2][6],
// boff[2][6], pbytes[2], poff[2] (42 ints).  Returns the count written.
int tc_layout(int p, int tf, int* out, int nout) {
    const TcChunks c = tc_chunks(p, tf, tc_chunk_width_env(tf));
    int v[42], n = 0;
    v[n++] = c.cw; v[n++] = c.nch; v[n++] = c.np; v[n++] = c.nbst; v[n++] = c.niss; v[n++] = c.bstage;
    v[n++] = c.mbytes; v[n++] = 4 * SL_BYTES + c.nbst * c.bstage + 1024 + 256;
    for (int j = 0; j < TC_NCH; ++j) v[n++] = c.kch[j];
    for (int t = 0; t < 2; ++t)
        for (int j = 0; j < TC_NCH; ++j) v[n++] = c.nk[t][j];
    for (int t = 0; t < 2; ++t)
        for (int j = 0; j < TC_NCH; ++j) v[n++] = c.boff[t][j];
    v[n++] = c.pbytes[0]; v[n++] = c.pbytes[1]; v[n++] = c.poff[0]; v[n++] = c.poff[1];
    const int m = nout < n ? nout : n;
    for (int i = 0; i < m; ++i) out[i] = v[i];
    return m;
}

int tc_first_level() { return 5; }   // class grid of 16 cells per axis: one slab column fits
size_t tc_m_elems(int l) { return l < 1 ? 0 : ((size_t)8 << (3 * (l - 1))) * TC_K; }

// Per-offset matrices of the streamed-matrix kernel in the layout of chunk
// width cw (a plan rebuilds them when its chunk width changes).
int tc_build_mat(int p, int tf, int cw, const double* Dtab, void* B, cudaStream_t s) {
    const int64_t tot = (int64_t)343 * TC_N * (TC_K * tc_elem_bytes(tf) / 16);
    if (cudaMemsetAsync(B, 0, tc_mat_bytes(tf), s) != cudaSuccess) return -2;
    const unsigned g = (unsigned)((tot + 255) / 256);
    if (tf)
        k_tc_build_b<1><<<g, 256, 0, s>>>(p, ncoef_of(p, 1), tc_chunks(p, 1, cw), Dtab, (unsigned char*)B);
    else
        k_tc_build_b<0><<<g, 256, 0, s>>>(p, ncoef_of(p, 1), tc_chunks(p, 0, cw), Dtab, (unsigned char*)B);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

// MMA-issuing warps of the streamed-matrix kernel at chunk width cw (as many
// as matrix stages fit, 2 or 4)
int tc_mat_niss(int p, int tf, int cw) { return tc_chunks(p, tf, cw).niss; }

// Encodes the tensor maps (8 classes x hi/lo) of one level.  Tensor dims
// (innermost first): e (16 bytes), i (hs), chunk (12 or 24), j (hs), k (hs);
// the box takes one K-part (12 chunks) of a 10 x 18 x 1 slab.
static int encode_set(TcMaps* m, int tf, void* hi, void* lo, cuuint64_t hs, const cuuint32_t box[5]) {
    const int es = tc_elem_bytes(tf), epc = 16 / es;
    const cuuint64_t nch = (cuuint64_t)(TC_K / epc);
    const cuuint64_t dims[5] = {(cuuint64_t)epc, hs, nch, hs, hs};
    const cuuint64_t strides[4] = {16, hs * 16, nch * hs * 16, hs * nch * hs * 16};
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    const size_t cls_bytes = (size_t)hs * hs * hs * TC_K * es;
    const CUtensorMapDataType dt = tf ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    for (int c = 0; c < 8; ++c) {
        for (int h = 0; h < 2; ++h) {
            void* base = (char*)(h ? lo : hi) + c * cls_bytes;
            CUresult r = g_encode(h ? &m->lo[c] : &m->hi[c], dt, 5, base, dims, strides, box, estr,
                                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                  CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) return -1;
        }
    }
    return 0;
}

int tc_encode_maps(int l, int tf, void* hi, void* lo, void* out_maps) {
    if (!g_encode) {
        cudaDriverEntryPointQueryResult q;
        void* fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return -2;
        g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    }
    TcLevelMaps* maps = (TcLevelMaps*)out_maps;
    const int epc = 16 / tc_elem_bytes(tf);
    const cuuint64_t hs = (cuuint64_t)1 << (l - 1);
    if (hs < 16) return -1;
    const cuuint32_t slab[5] = {(cuuint32_t)epc, SL_I, (cuuint32_t)TC_CH, SL_J, 1};
    if (encode_set(&maps->slab, tf, hi, lo, hs, slab) != 0) return -1;
    if (tf) return 0;
    unsigned tb[5];
    tct_box(l, tb);
    const cuuint32_t tall[5] = {tb[0], tb[1], tb[2], tb[3], tb[4]};
    return encode_set(&maps->tall, tf, hi, lo, hs, tall) == 0 ? 0 : -1;
}
size_t tc_maps_bytes() { return sizeof(TcLevelMaps); }

template <int TF, int NISS>
static int tc_launch(const TcChunks& ch, int l, int nc, const void* maps, const void* B, double* Lt, float* Lt32,
                     int64_t ncell,
                     int* err, cudaStream_t s) {
    const int hs = 1 << (l - 1);
    const TcLevelMaps* m = (const TcLevelMaps*)maps;
    const int smem = 4 * SL_BYTES + ch.nbst * ch.bstage + 1024 + 256;
    if (cudaFuncSetAttribute(k_m2l_tc_slab<TF, NISS>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
        cudaSuccess)
        return -2;
    const int tpc = (hs / 8) * (hs / 16) * hs;
    k_m2l_tc_slab<TF, NISS><<<(unsigned)(8 * tpc), sl_threads<NISS>(), smem, s>>>(
        m->slab, ch, l, nc, (const unsigned char*)B, Lt, ncell, err, Lt32);
    count_launch();
    return 0;
}

int tc_m2l_level(int p, int tf, int kern, int cw, int niss, int l, const double* M, void* hi, void* lo,
                 const void* maps, const void* B, double* Lt, int* err, cudaStream_t s,
                 const float* M32, float* Lt32) {
    const int hs = 1 << (l - 1);
    if (hs < 16) return -1;
    const int64_t ncell = (int64_t)8 * hs * hs * hs;
    const int nc = ncoef_of(p, 1);
    if (ncell > ((int64_t)1 << 30)) return -1;   // 32-bit cell indices in k_tc_split_m
    // kernel 3 reads the first K-part (16-byte chunks 0..5) only
    const dim3 g((unsigned)((ncell + 255) / 256), (unsigned)(kern == 3 ? 6 : TC_K * tc_elem_bytes(tf) / 16));
    if ((kern >= 1) && tf) return -1;   // the on-chip and swapped kernels take BF16 operands
    // the on-chip kernel's matrices hold D_{n+m} alone: its operand carries 1/m!
    if (tf)
        k_tc_split_m<1><<<g, 256, 0, s>>>(l, nc, 0, M, hi, lo, M32);
    else
        k_tc_split_m<0><<<g, 256, 0, s>>>(l, nc, kern == 1, M, hi, lo, kern == 1 ? nullptr : M32);
    count_launch();
    if (kern == 1) {
        const int rc = tg_m2l_level(p, cw, niss, l, maps, B, Lt, err, s, Lt32);
        if (rc != 0) return rc;
        return cudaGetLastError() == cudaSuccess ? 0 : -2;
    }
    if (kern == 2 || kern == 3) return tct_m2l_level(p, l, kern == 3, maps, B, Lt, err, s, Lt32);
    const TcChunks ch = tc_chunks(p, tf, cw);
    if (ch.niss != 2 && ch.niss != 4) return -1;
    const int rc = tf ? (ch.niss == 4 ? tc_launch<1, 4>(ch, l, nc, maps, B, Lt, Lt32, ncell, err, s)
                                      : tc_launch<1, 2>(ch, l, nc, maps, B, Lt, Lt32, ncell, err, s))
                      : (ch.niss == 4 ? tc_launch<0, 4>(ch, l, nc, maps, B, Lt, Lt32, ncell, err, s)
                                      : tc_launch<0, 2>(ch, l, nc, maps, B, Lt, Lt32, ncell, err, s));
    if (rc != 0) return rc;
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

}  // namespace fmm
