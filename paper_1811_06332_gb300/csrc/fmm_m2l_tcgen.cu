// Offset-grouped M2L on the tensor cores with the offset matrices built on
// chip (Eq. M2L regrouped; BF16 hi/lo operands, FP32 accumulation in TMEM).
//
// On a uniform level every target cell of one parity class sees the same 189
// integer offsets o.  With the multipoles scaled by 1/m! (A[cell, m] =
// Mt_m / m!, reduced traceless representative), the matrix of an offset is
//     B_o(n, m) = D_{n+m}(-o)            (cell units, |n| + |m| <= p, else 0)
// so it is fixed by the D-tensor of the offset alone: ns(p) <= 165 numbers.
// Instead of streaming a 21 KB hi/lo matrix per offset from L2, a CTA copies
// the offset's FP32 D vector (704 bytes) and eight generator warps write the
// matrix into a shared-memory stage: each thread owns one 16-byte group
// (8 multipole columns of one local row) of the rank triangle, looks up its
// 8 D values, splits them into BF16 hi + lo and stores both.  Groups outside
// the triangle are zero in every offset and are cleared once.
//
// Fewer MMAs per K-step: the hi and lo rows of chunk j are stacked along N,
// so  A_hi . [B_hi; B_lo]^T  (N = 2 cw) yields hi.hi in the chunk's main
// columns and hi.lo in its correction columns, and  A_lo . B_hi^T  (N = cw)
// adds lo.hi to the main columns: 2 MMAs per K-step instead of 3.  The
// epilogue adds main + correction columns in FP64.
//
// Roles: warp 0 lane 0 issues the TMA slab loads and the D-vector copies;
// lane 0 of warp 1 (and of warp 10 with two issuers) issues tcgen05.mma;
// warps 2..9 generate the matrices; warps 2..5 then drain TMEM into FP64 L
// (each reads its lane quadrant).  Every wait is bounded and reports a
// timeout through the error word.
#include <cuda.h>
#include <cuda_bf16.h>

#include <cstdlib>
#include <vector>

#include "fmm_internal.h"
#include "fmm_tc_common.cuh"

namespace fmm {

constexpr int TG_GEN_WARPS = 8;                 // generator warps (2..9)
constexpr int TG_GEN_THREADS = 32 * TG_GEN_WARPS;
constexpr int TG_DPAD = 176;                    // floats per D vector: ns(8) = 165, padded to 16 bytes
constexpr int TG_DBYTES = TG_DPAD * 4;          // 704
constexpr int TG_ND = 8;                        // D-vector ring stages
constexpr int TG_TMEM_COLS = 256;               // one issuer's accumulators (2 cw nch <= 192 columns)
constexpr int TG_SMEM_MAX = 227 * 1024;

// Layout of one on-chip matrix stage for order p and chunk width cw.
struct TgLayout {
    int cw;              // local rows per chunk (N of the lo.hi MMA; the hi/lo MMA has N = 2 cw)
    int nch;             // chunks
    int kch[TC_NCH];     // K-steps (16 multipole columns) of chunk j
    int coff[TC_NCH];    // byte offset of chunk j in a stage: 2 cw rows x kch[j] K-steps
    int bstage;          // bytes of one stage (multiple of 1024)
    int nb;              // stages (a multiple of the issuer count)
    int niss;            // MMA-issuing warps (1 or 2)
    int ngroups;         // nonzero 16-byte groups of one matrix (<= TG_GEN_THREADS)
    int smem;            // dynamic shared bytes of the kernel
};

template <int NISS>
constexpr int tg_threads() { return 32 * (2 + TG_GEN_WARPS + (NISS - 1)); }

template <int NISS>
__global__ void __launch_bounds__(tg_threads<NISS>(), 1)
k_m2l_tc_gen(const __grid_constant__ TcMaps maps, const TgLayout lay, int l, int nrows,
             const float* __restrict__ D32, const uint4* __restrict__ groups, double* __restrict__ Lt,
             int64_t ncell, int* __restrict__ err, float* __restrict__ Lt32) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* bring = smem + 4 * SL_BYTES;
    float* dring = (float*)(bring + lay.nb * lay.bstage);
    uint64_t* bars = (uint64_t*)(dring + TG_ND * TG_DPAD);
    uint64_t* sfull = bars;                 // [2]
    uint64_t* sempty = bars + 2;            // [2]
    uint64_t* dfull = bars + 4;             // [TG_ND]
    uint64_t* dempty = dfull + TG_ND;       // [TG_ND]
    uint64_t* bfull = dempty + TG_ND;       // [4]
    uint64_t* bempty = bfull + 4;           // [4]
    uint64_t* done = bempty + 4;
    uint32_t* tslot = (uint32_t*)(done + 1);
    volatile int* sfail = (volatile int*)(tslot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int hs = 1 << (l - 1);
    const int nti = hs / 8, ntj = hs / 16;
    // class fastest: the 8 CTAs of one spatial column read the same source
    // slabs close together in time, so they are served from L2
    const int cls = blockIdx.x & 7, t = blockIdx.x >> 3;
    const int ti = t % nti, tj = (t / nti) % ntj, tk = t / (nti * ntj);
    const int cx = cls & 1, cy = (cls >> 1) & 1, cz = cls >> 2;
    if (lay.niss != NISS || lay.nb % NISS != 0 || lay.nb > 4 || lay.ngroups > TG_GEN_THREADS) {
        if (threadIdx.x == 0) atomicExch(err, 27);   // launch/layout mismatch: no barrier is used
        return;
    }

    if (threadIdx.x == 0) {
        for (int b = 0; b < 2; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&sfull[b])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&sempty[b])), "r"(NISS));
        }
        for (int b = 0; b < TG_ND; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&dfull[b])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&dempty[b])), "r"(TG_GEN_WARPS));
        }
        for (int b = 0; b < lay.nb; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bfull[b])), "r"(TG_GEN_WARPS));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bempty[b])));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(done)), "r"(NISS));
        *sfail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(NISS * TG_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- producer: slabs and D vectors ----------------
            int sl = 0, k = 0;
            bool ok = true;
            for (int sc = 0; sc < 8 && ok; ++sc) {
                const int sx = sc & 1, sy = (sc >> 1) & 1, sz = sc >> 2;
                for (int dz = -1; dz <= 1 && ok; ++dz) {
                    if (tk + dz < 0 || tk + dz >= hs) continue;   // plane outside the grid: no sources
                    const int oz = 2 * dz + sz - cz;
                    const int buf = sl & 1;
                    if (!(ok = mbar_wait(smem_u32(&sempty[buf]), ((uint32_t)(sl >> 1) & 1u) ^ 1u, err, 21))) break;
                    const uint32_t fb = smem_u32(&sfull[buf]);
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(2 * SL_BYTES)
                                 : "memory");
                    unsigned char* st = smem + buf * 2 * SL_BYTES;
                    const int c1 = 8 * ti - 1, c3 = 16 * tj - 1, c4 = tk + dz;
                    asm volatile(
                        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                        " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(smem_u32(st)),
                        "l"((uint64_t)&maps.hi[sc]), "r"(0), "r"(c1), "r"(0), "r"(c3), "r"(c4), "r"(fb)
                        : "memory");
                    asm volatile(
                        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                        " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(smem_u32(st + SL_BYTES)),
                        "l"((uint64_t)&maps.lo[sc]), "r"(0), "r"(c1), "r"(0), "r"(c3), "r"(c4), "r"(fb)
                        : "memory");
                    ++sl;
                    for (int dy = -1; dy <= 1 && ok; ++dy) {
                        const int oy = 2 * dy + sy - cy;
                        for (int dx = -1; dx <= 1; ++dx) {
                            const int ox = 2 * dx + sx - cx;
                            if (ox >= -1 && ox <= 1 && oy >= -1 && oy <= 1 && oz >= -1 && oz <= 1) continue;
                            const int ds = k % TG_ND;
                            if (!(ok = mbar_wait(smem_u32(&dempty[ds]), ((uint32_t)(k / TG_ND) & 1u) ^ 1u, err, 22)))
                                break;
                            const uint32_t db = smem_u32(&dfull[ds]);
                            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(db),
                                         "r"(TG_DBYTES)
                                         : "memory");
                            const int ridx = (3 - oz) * 49 + (3 - oy) * 7 + (3 - ox);   // r = -o
                            asm volatile(
                                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
                                "[%3];" ::"r"(smem_u32(dring + ds * TG_DPAD)),
                                "l"((uint64_t)(D32 + (int64_t)ridx * TG_DPAD)), "r"(TG_DBYTES), "r"(db)
                                : "memory");
                            ++k;
                        }
                    }
                }
            }
            if (!ok) *sfail = 1;
            // drain: every issued copy has landed before the CTA may exit
            for (int q = sl > 2 ? sl - 2 : 0; q < sl; ++q)
                mbar_wait(smem_u32(&sfull[q & 1]), (uint32_t)(q >> 1) & 1u, err, 23);
            for (int q = k > TG_ND ? k - TG_ND : 0; q < k; ++q)
                mbar_wait(smem_u32(&dfull[q % TG_ND]), (uint32_t)(q / TG_ND) & 1u, err, 23);
        }
    } else if (warp == 1 || warp == 2 + TG_GEN_WARPS) {
        if (lane == 0) {
            // ---------------- MMA issuers ----------------
            const int w = warp == 1 ? 0 : 1;
            const uint32_t dbase = tmem + (uint32_t)(w * TG_TMEM_COLS);
            const uint32_t id_hl = make_idesc(0, 128, 2 * lay.cw);   // A_hi . [B_hi; B_lo]
            const uint32_t id_lh = make_idesc(0, 128, lay.cw);       // A_lo . B_hi
            int sl = 0, k = 0;
            bool ok = true, first = true;
            for (int sc = 0; sc < 8 && ok; ++sc) {
                const int sx = sc & 1, sy = (sc >> 1) & 1, sz = sc >> 2;
                for (int dz = -1; dz <= 1 && ok; ++dz) {
                    if (tk + dz < 0 || tk + dz >= hs) continue;
                    const int oz = 2 * dz + sz - cz;
                    const int buf = sl & 1;
                    if (!(ok = mbar_wait(smem_u32(&sfull[buf]), (uint32_t)(sl >> 1) & 1u, err, 24))) break;
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t sbase = smem_u32(smem + buf * 2 * SL_BYTES);
                    for (int dy = -1; dy <= 1 && ok; ++dy) {
                        const int oy = 2 * dy + sy - cy;
                        for (int dx = -1; dx <= 1; ++dx) {
                            const int ox = 2 * dx + sx - cx;
                            if (ox >= -1 && ox <= 1 && oy >= -1 && oy <= 1 && oz >= -1 && oz <= 1) continue;
                            const int mine = k % NISS == w;
                            const int bs = k % lay.nb;
                            const uint32_t ph = (uint32_t)(k / lay.nb) & 1u;
                            ++k;
                            if (!mine) continue;
                            if (!(ok = mbar_wait(smem_u32(&bfull[bs]), ph, err, 25))) break;
                            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                            const uint32_t bbase = smem_u32(bring + bs * lay.bstage);
                            const uint32_t aoff = (uint32_t)(((dy + 1) * TC_CH * SL_I + (dx + 1)) * 16);
                            // K-step 0 descriptors; a K-step adds 320 bytes (A) or 256 bytes (B),
                            // i.e. 20 or 16 in the address field (no carry: shared addresses < 2^18)
                            const uint64_t ah = make_desc(sbase + aoff, SL_I * 16, TC_CH * SL_I * 16);
                            const uint64_t al = make_desc(sbase + SL_BYTES + aoff, SL_I * 16, TC_CH * SL_I * 16);
                            for (int j = 0; j < lay.nch; ++j) {
                                const int nk = lay.kch[j];
                                const uint32_t dcol = dbase + (uint32_t)(2 * lay.cw * j);
                                const uint64_t bd = make_desc(bbase + lay.coff[j], 128, 256u * nk);
                                for (int ks = 0; ks < nk; ++ks) {
                                    tc_mma<0>(dcol, ah + 20 * ks, bd + 16 * ks, id_hl, (first && ks == 0) ? 0u : 1u);
                                    tc_mma<0>(dcol, al + 20 * ks, bd + 16 * ks, id_lh, 1u);
                                }
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
            if (!ok) *sfail = 1;
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(done))
                         : "memory");
        }
    } else {
        // ---------------- generators (warps 2..9) ----------------
        const int gt = (warp - 2) * 32 + lane;
        const bool has = gt < lay.ngroups;
        uint4 gd = make_uint4(0u, 0u, 0u, 0u);
        if (has) gd = groups[gt];
        // clear every stage once: the groups outside the rank triangle stay zero
        {
            uint4* z = (uint4*)bring;
            const int n16 = lay.nb * lay.bstage / 16;
            for (int i = gt; i < n16; i += TG_GEN_THREADS) z[i] = make_uint4(0u, 0u, 0u, 0u);
            asm volatile("bar.sync 1, %0;" ::"r"(TG_GEN_THREADS) : "memory");
        }
        int k = 0;
        bool ok = true;
        for (int sc = 0; sc < 8 && ok; ++sc) {
            const int sx = sc & 1, sy = (sc >> 1) & 1, sz = sc >> 2;
            for (int dz = -1; dz <= 1 && ok; ++dz) {
                if (tk + dz < 0 || tk + dz >= hs) continue;
                const int oz = 2 * dz + sz - cz;
                for (int dy = -1; dy <= 1 && ok; ++dy) {
                    const int oy = 2 * dy + sy - cy;
                    for (int dx = -1; dx <= 1 && ok; ++dx) {
                        const int ox = 2 * dx + sx - cx;
                        if (ox >= -1 && ox <= 1 && oy >= -1 && oy <= 1 && oz >= -1 && oz <= 1) continue;
                        const int ds = k % TG_ND, bs = k % lay.nb;
                        // this offset's D vector
                        bool w_ok = true;
                        if (lane == 0) w_ok = mbar_wait(smem_u32(&dfull[ds]), (uint32_t)(k / TG_ND) & 1u, err, 26);
                        ok = __shfl_sync(0xffffffffu, w_ok, 0);
                        if (!ok) break;
                        float v[8];
                        const float* dv = dring + ds * TG_DPAD;
#pragma unroll
                        for (int e = 0; e < 8; ++e) {
                            const uint32_t word = e < 4 ? gd.x : gd.y;
                            const uint32_t ix = (word >> (8 * (e & 3))) & 0xFFu;
                            v[e] = ix < 255u ? dv[ix] : 0.f;
                        }
                        __syncwarp();
                        if (lane == 0)
                            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&dempty[ds]))
                                         : "memory");
                        // the stage is free once the MMAs of its previous offset completed
                        if (lane == 0)
                            w_ok = mbar_wait(smem_u32(&bempty[bs]), ((uint32_t)(k / lay.nb) & 1u) ^ 1u, err, 28);
                        ok = __shfl_sync(0xffffffffu, w_ok, 0);
                        if (!ok) break;
                        if (has) {
                            uint32_t hw[4], lw[4];
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * e], v[2 * e + 1]);
                                const __nv_bfloat162 lo = __floats2bfloat162_rn(v[2 * e] - __low2float(h),
                                                                                v[2 * e + 1] - __high2float(h));
                                hw[e] = *(const uint32_t*)&h;
                                lw[e] = *(const uint32_t*)&lo;
                            }
                            unsigned char* sb = bring + bs * lay.bstage;
                            *(uint4*)(sb + gd.z) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                            *(uint4*)(sb + gd.w) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
                        }
                        // generic-proxy writes become visible to the tensor core (async proxy)
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                        __syncwarp();
                        if (lane == 0)
                            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&bfull[bs]))
                                         : "memory");
                        ++k;
                    }
                }
            }
        }
        if (!ok && lane == 0) *sfail = 1;
        if (warp >= 2 && warp <= 5) {
            // ---------------- epilogue: TMEM -> FP64 L ----------------
            bool e_ok = true;
            if (lane == 0) e_ok = mbar_wait(smem_u32(done), 0u, err, 29);
            e_ok = __shfl_sync(0xffffffffu, e_ok, 0);
            __syncwarp();
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const bool write = e_ok && *sfail == 0;
            const int q = warp & 3;
            const int row = q * 32 + lane;
            const int i = row & 7, jj = row >> 3;
            const int64_t h3 = (int64_t)hs * hs * hs;
            const int64_t tg = (int64_t)cls * h3 + ((int64_t)tk * hs + (16 * tj + jj)) * hs + (8 * ti + i);
            const uint32_t lbase = tmem + ((uint32_t)(q * 32) << 16);
#pragma unroll 1
            for (int j = 0; j < lay.nch; ++j) {
#pragma unroll 1
                for (int r0 = 0; r0 < lay.cw; r0 += 16) {
                    const int n0 = j * lay.cw + r0;
                    if (n0 >= nrows) break;
                    double acc[16];
#pragma unroll
                    for (int e = 0; e < 16; ++e) acc[e] = 0.0;
#pragma unroll 1
                    for (int w = 0; w < NISS; ++w) {
                        const uint32_t c0 = (uint32_t)(w * TG_TMEM_COLS + 2 * lay.cw * j + r0);
                        uint32_t vm[16], vc[16];
                        tmem_ld16(lbase + c0, vm);
                        tmem_ld16(lbase + c0 + (uint32_t)lay.cw, vc);
                        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                        for (int e = 0; e < 16; ++e)
                            acc[e] += (double)__uint_as_float(vm[e]) + (double)__uint_as_float(vc[e]);
                    }
                    if (write) {
#pragma unroll
                        for (int e = 0; e < 16; ++e)
                            if (n0 + e < nrows) {
                                if (Lt32) Lt32[(int64_t)(n0 + e) * ncell + tg] = (float)acc[e];
                                else Lt[(int64_t)(n0 + e) * ncell + tg] = acc[e];
                            }
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NISS * TG_TMEM_COLS));
    }
}

// D vectors of the 343 integer offsets in FP32, zero-padded to TG_DPAD:
// D32[r][k] = D_k(r) (symmetric storage order, |k| <= p).
__global__ void k_tg_d32(int ns, const double* __restrict__ Dtab, float* __restrict__ D32) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 343 * TG_DPAD) return;
    const int r = t / TG_DPAD, k = t % TG_DPAD;
    D32[t] = k < ns ? (float)Dtab[(int64_t)r * ns + k] : 0.f;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static int tg_rank_tl(int r) {   // rank of the traceless independent component r
    int a = 0;
    while ((a + 1) * (a + 1) <= r) ++a;
    return a;
}

static TgLayout tg_layout(int p, int cw, int niss) {
    TgLayout L{};
    const int nc = ncoef_of(p, 1);
    L.cw = cw;
    L.niss = niss;
    L.nch = (nc + cw - 1) / cw;
    int off = 0;
    for (int j = 0; j < L.nch; ++j) {
        const int a = tg_rank_tl(cw * j);                // lowest rank in the chunk
        const int cols = (p - a + 1) * (p - a + 1);
        L.kch[j] = (cols + 15) / 16;
        L.coff[j] = off;
        off += (2 * cw / 8) * L.kch[j] * 256;
    }
    L.bstage = (off + 1023) / 1024 * 1024;
    int groups = 0;
    for (int r = 0; r < nc; ++r) {
        const int a = tg_rank_tl(r);
        groups += ((p - a + 1) * (p - a + 1) + 7) / 8;
    }
    L.ngroups = groups;
    const int fixed = 4 * SL_BYTES + TG_ND * TG_DBYTES + 512 + 1024;   // slabs, D ring, barriers, alignment
    int nb = (TG_SMEM_MAX - fixed) / L.bstage;
    if (nb > 4) nb = 4;
    nb -= nb % niss;
    L.nb = nb;
    L.smem = fixed + nb * L.bstage;
    return L;
}

// Group descriptors: per nonzero 16-byte group g (row r, columns 8c..8c+7)
// the symmetric positions of n_r + m_e (255 outside the triangle or the
// padding) in x (e = 0..3) and y (e = 4..7), and the byte offsets of its hi
// and lo 16 bytes inside a stage in z and w.
static void tg_groups(int p, const TgLayout& L, std::vector<uint32_t>& out) {
    const int nc = ncoef_of(p, 1);
    out.clear();
    for (int r = 0; r < nc; ++r) {
        const int a = tg_rank_tl(r);
        const int ncol = (p - a + 1) * (p - a + 1);
        const int j = r / L.cw, rr = r % L.cw;
        const unsigned char* n = fmm_tl_idx[r];
        for (int c = 0; c * 8 < ncol; ++c) {
            uint32_t w[2] = {0u, 0u};
            for (int e = 0; e < 8; ++e) {
                const int m = 8 * c + e;
                uint32_t ix = 255u;
                if (m < ncol && m < nc) {
                    const unsigned char* mm = fmm_tl_idx[m];
                    ix = (uint32_t)pos_sym(n[0] + mm[0], n[1] + mm[1], n[2] + mm[2]);
                }
                w[e / 4] |= ix << (8 * (e % 4));
            }
            const int sbo = 256 * L.kch[j];
            const uint32_t hi = (uint32_t)(L.coff[j] + (rr / 8) * sbo + c * 128 + (rr % 8) * 16);
            const uint32_t lo = (uint32_t)(L.coff[j] + ((rr + L.cw) / 8) * sbo + c * 128 + ((rr + L.cw) % 8) * 16);
            out.push_back(w[0]);
            out.push_back(w[1]);
            out.push_back(hi);
            out.push_back(lo);
        }
    }
}

static int tg_cw_default() { return 96; }
static int tg_niss_default() { return 1; }

int tg_supported(int p) { return p >= 1 && p <= 8; }

// Host-side layout for diagnostics: cw, nch, bstage, nb, niss, ngroups, smem,
// kch[6], coff[6] (19 ints), then the group table (4 words per group) when
// groups != NULL.  Returns the number of ints written to out.
int tg_layout_host(int p, int cw, int niss, int* out, int nout, uint32_t* groups, int gcap) {
    if (!tg_supported(p) || (cw != 16 && cw != 32 && cw != 48 && cw != 96) || (niss != 1 && niss != 2)) return -1;
    const TgLayout L = tg_layout(p, cw, niss);
    int v[19], n = 0;
    v[n++] = L.cw; v[n++] = L.nch; v[n++] = L.bstage; v[n++] = L.nb; v[n++] = L.niss; v[n++] = L.ngroups;
    v[n++] = L.smem;
    for (int j = 0; j < TC_NCH; ++j) v[n++] = L.kch[j];
    for (int j = 0; j < TC_NCH; ++j) v[n++] = L.coff[j];
    const int m = nout < n ? nout : n;
    for (int i = 0; i < m; ++i) out[i] = v[i];
    if (groups) {
        std::vector<uint32_t> g;
        tg_groups(p, L, g);
        for (int i = 0; i < (int)g.size() && i < gcap; ++i) groups[i] = g[i];
    }
    return m;
}

size_t tg_b_bytes() { return (size_t)TG_GEN_THREADS * 16 + (size_t)343 * TG_DBYTES; }

// Plan set-up: group table (for the default layout's chunk width; the table
// depends on cw) and the FP32 D vectors, into B = [groups | D32].
int tg_build(int p, int cw, int niss, const double* Dtab, void* B, cudaStream_t s) {
    if (!tg_supported(p)) return -1;
    const TgLayout L = tg_layout(p, cw, niss);
    if (L.ngroups > TG_GEN_THREADS || L.nb < 2 || L.nb < niss) return -1;
    std::vector<uint32_t> g;
    tg_groups(p, L, g);
    g.resize((size_t)TG_GEN_THREADS * 4, 0u);
    if (cudaMemcpyAsync(B, g.data(), g.size() * 4, cudaMemcpyHostToDevice, s) != cudaSuccess) return -2;
    if (cudaStreamSynchronize(s) != cudaSuccess) return -2;   // g goes out of scope
    float* D32 = (float*)((unsigned char*)B + (size_t)TG_GEN_THREADS * 16);
    k_tg_d32<<<(343 * TG_DPAD + 255) / 256, 256, 0, s>>>(ns_of(p), Dtab, D32);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

template <int NISS>
static int tg_launch(const TgLayout& L, int l, int nc, const void* maps, const void* B, double* Lt, float* Lt32,
                     int64_t ncell,
                     int* err, cudaStream_t s) {
    const int hs = 1 << (l - 1);
    const TcLevelMaps* m = (const TcLevelMaps*)maps;
    if (cudaFuncSetAttribute(k_m2l_tc_gen<NISS>, cudaFuncAttributeMaxDynamicSharedMemorySize, L.smem) != cudaSuccess)
        return -2;
    const int tpc = (hs / 8) * (hs / 16) * hs;
    const uint4* groups = (const uint4*)B;
    const float* D32 = (const float*)((const unsigned char*)B + (size_t)TG_GEN_THREADS * 16);
    k_m2l_tc_gen<NISS><<<(unsigned)(8 * tpc), tg_threads<NISS>(), L.smem, s>>>(m->slab, L, l, nc, D32, groups, Lt,
                                                                               ncell, err, Lt32);
    count_launch();
    return 0;
}

// M2L of uniform level l (class grid >= 16 per axis) on the tensor cores with
// on-chip matrices; hi/lo BF16 operands of the level already split (scaled
// by 1/m!) into the slab layout.
int tg_m2l_level(int p, int cw, int niss, int l, const void* maps, const void* B, double* Lt, int* err,
                 cudaStream_t s, float* Lt32) {
    const int hs = 1 << (l - 1);
    if (hs < 16 || !tg_supported(p)) return -1;
    const int64_t ncell = (int64_t)8 * hs * hs * hs;
    const TgLayout L = tg_layout(p, cw, niss);
    if (L.nb < 2) return -1;
    const int nc = ncoef_of(p, 1);
    return niss == 2 ? tg_launch<2>(L, l, nc, maps, B, Lt, Lt32, ncell, err, s)
                     : tg_launch<1>(L, l, nc, maps, B, Lt, Lt32, ncell, err, s);
}

int tg_default_cw() { return tg_cw_default(); }
int tg_default_niss() { return tg_niss_default(); }

}  // namespace fmm
