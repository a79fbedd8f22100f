// Offset-grouped M2L on the tensor cores with the roles of the two operands
// swapped (Eq. M2L regrouped, the third kernel shape of the BF16 form).
//
// On a uniform level every target cell of one parity class sees the same
// 189 offsets o, and all pairs with one offset share the matrix
//     Kt_o(n, m) = D_{n+m}(-o)/m!       (cell units, |n| + |m| <= p).
// Here the matrix is the A operand (M = 128 rows: the local components n,
// 81 of them at p = 8) and the source multipoles are the B operand (N = the
// target cells of a tile, 8 x TY x 1 of one class: 256 at TY = 32, 128 at
// TY = 16), so one MMA covers the whole tile:
//     D[128 x N] += A_o[128 x 16] . B_o[N x 16]^T      per K-step
// with D (local components x cells) in TMEM.  The per-instruction cost of an
// MMA does not grow with N up to 256, so covering 256 cells per MMA issues
// 9 MMAs per offset and 128 cells where the other orientation (cells as M,
// local components as N <= 96) issues 21.
//
// K (the 81 reduced multipole components, padded to 96) runs in two K-parts
// of 48.  For each source class, z shift and K-part, one 5-D TMA load brings
// a slab of (8 + 2) x (TY + 2) x 1 cells (zero fill outside the grid); the B
// operand of offset (dx, dy) is the slab with its start moved by dx cells
// along x and dy rows along y (no-swizzle K-major core matrices of 8 cells x
// 16 bytes: LBO 160 bytes, SBO 960 bytes).  The matrix of an offset's K-part
// (hi and lo, 88 rows) comes by one bulk copy into a 4-stage ring; its rows
// 88..127 are read from whatever follows the block in shared memory (the lo
// block, the next stage or a pad) and only feed TMEM lanes >= 88, which hold
// no local component and are never read.
// Split precision: x = hi + lo in BF16, three MMAs per K-step (hi.hi, hi.lo,
// lo.hi), FP32 accumulation in TMEM, the two issuers' accumulators added in
// FP32 and converted once at write-out (FP64 operations are the narrow pipe
// of this part).
//
// Kernel shape 3 runs the first K-part only: the columns >= 48 reach only
// the local rows of rank <= p - 6 (9 of the 128 rows at p = 8), so the second
// K-part's tiles would be mostly padding; those products (86 per pair at
// p = 8) run afterwards as FP32 FMAs on the CUDA cores (fmm_m2l_rest.cu).
//
// Roles: warp 0 lane 0 issues the slab loads and warp 7 lane 0 the matrix
// copies (separately, so that the next slab is requested as soon as its
// buffer is free); lane 0 of warps 1 and 6 issue tcgen05.mma, each into its
// own accumulator of N columns, taking the matrix blocks alternately; warps
// 2..5 drain TMEM (each reads its lane quadrant) and write L through a
// shared-memory transpose.  Every wait is bounded and reports a timeout
// through an error word.
#include <cuda.h>
#include <cuda_bf16.h>

#include "fmm_internal.h"
#include "fmm_tc_common.cuh"

namespace fmm {

constexpr int TT_KP = 6;                          // 16-byte chunks (8 BF16 columns) per K-part
constexpr int TT_G = 11;                          // 8-row groups of local components stored (88 rows)
constexpr int TT_GB = TT_G * TT_KP * 128;         // 8448: one hi or lo block of a K-part
constexpr int TT_BLK = 2 * TT_GB;                 // hi + lo block of one offset's K-part
constexpr int TT_OVR = (16 - TT_G) * TT_KP * 128; // 3840: bytes an M = 128 operand reads past a block
constexpr int TT_NST = 4;                         // matrix stages
constexpr int TT_NISS = 2;                        // MMA-issuing warps (divides TT_NST)
constexpr int TT_I = 10;                          // slab cells along x
constexpr int TT_SBO = TT_KP * TT_I * 16;         // 960: slab bytes per cell row (y)

static __host__ __device__ constexpr int tt_slab_bytes(int ty) { return (ty + 2) * TT_SBO; }
static __host__ __device__ constexpr int tt_smem(int ty) {
    return 4 * tt_slab_bytes(ty) + TT_NST * TT_BLK + TT_OVR + 256 + 1024;
}

int tct_np(int p) { return (ncoef_of(p, 1) + 8 * TT_KP - 1) / (8 * TT_KP); }
size_t tct_bytes() { return (size_t)343 * 2 * TT_BLK; }
int tct_ty(int l) { return l >= 6 ? 32 : 16; }   // tile rows: the class grid has 2^(l-1) cells per axis

constexpr int TT_THREADS = 256;

template <int TY>
__global__ void __launch_bounds__(TT_THREADS, 1)
k_m2l_tc_t(const __grid_constant__ TcMaps maps, int l, int np, int npt, int nrows,
           const unsigned char* __restrict__ Kmat, double* __restrict__ Lt, int64_t ncell, int* __restrict__ err,
           float* __restrict__ Lt32) {
    constexpr int N = 8 * TY;
    constexpr int SLB = tt_slab_bytes(TY);
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* ring = smem + 4 * SLB;
    uint64_t* bars = (uint64_t*)(ring + TT_NST * TT_BLK + TT_OVR);
    uint64_t* sfull = bars;        // [2]
    uint64_t* sempty = bars + 2;   // [2]
    uint64_t* bfull = bars + 4;    // [4]
    uint64_t* bempty = bars + 8;   // [4]
    uint64_t* done = bars + 12;
    uint32_t* tslot = (uint32_t*)(bars + 13);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int hs = 1 << (l - 1);
    const int nti = hs / 8, ntj = hs / TY;
    const int tpc = nti * ntj * hs;
    const int cls = blockIdx.x / tpc, t = blockIdx.x % tpc;
    const int ti = t % nti, tj = (t / nti) % ntj, tk = t / (nti * ntj);
    const int cx = cls & 1, cy = (cls >> 1) & 1, cz = cls >> 2;

    if (threadIdx.x == 0) {
        for (int b = 0; b < 2; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&sfull[b])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&sempty[b])), "r"(TT_NISS));
        }
        for (int b = 0; b < TT_NST; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bfull[b])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bempty[b])));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(done)), "r"(TT_NISS));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(TT_NISS * N));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;

    if ((warp == 0 || warp == 7) && lane == 0) {
        // ---------------- producers: slabs (warp 0), matrices (warp 7) ----------------
        const bool slabs = warp == 0;
        int sl = 0, bt = 0;
        bool ok = true;
        for (int sc = 0; sc < 8 && ok; ++sc) {
            const int sx = sc & 1, sy = (sc >> 1) & 1, sz = sc >> 2;
            for (int dz = -1; dz <= 1 && ok; ++dz) {
                if (tk + dz < 0 || tk + dz >= hs) continue;   // plane outside the grid: no sources
                const int oz = 2 * dz + sz - cz;
                for (int pt = 0; pt < npt && ok; ++pt) {
                    const int buf = sl & 1;
                    ++sl;
                    if (slabs) {
                    if (!(ok = mbar_wait(smem_u32(&sempty[buf]), ((uint32_t)((sl - 1) >> 1) & 1u) ^ 1u, err, 21))) break;
                    const uint32_t fb = smem_u32(&sfull[buf]);
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(2 * SLB)
                                 : "memory");
                    unsigned char* st = smem + buf * 2 * SLB;
                    const int c1 = 8 * ti - 1, c2 = TT_KP * pt, c3 = TY * tj - 1, c4 = tk + dz;
                    asm volatile(
                        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                        " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(smem_u32(st)),
                        "l"((uint64_t)&maps.hi[sc]), "r"(0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(fb)
                        : "memory");
                    asm volatile(
                        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                        " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(smem_u32(st + SLB)),
                        "l"((uint64_t)&maps.lo[sc]), "r"(0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(fb)
                        : "memory");
                    continue;
                    }
                    for (int dy = -1; dy <= 1 && ok; ++dy) {
                        const int oy = 2 * dy + sy - cy;
                        for (int dx = -1; dx <= 1; ++dx) {
                            const int ox = 2 * dx + sx - cx;
                            if (ox >= -1 && ox <= 1 && oy >= -1 && oy <= 1 && oz >= -1 && oz <= 1) continue;
                            const int bs = bt % TT_NST;
                            if (!(ok = mbar_wait(smem_u32(&bempty[bs]), ((uint32_t)(bt / TT_NST) & 1u) ^ 1u, err,
                                                 22)))
                                break;
                            const uint32_t bb = smem_u32(&bfull[bs]);
                            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bb),
                                         "r"(TT_BLK)
                                         : "memory");
                            const int ridx = (3 - oz) * 49 + (3 - oy) * 7 + (3 - ox);   // r = -o
                            const unsigned char* kb = Kmat + ((int64_t)ridx * np + pt) * TT_BLK;
                            asm volatile(
                                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
                                "[%3];" ::"r"(smem_u32(ring + bs * TT_BLK)),
                                "l"((uint64_t)kb), "r"(TT_BLK), "r"(bb)
                                : "memory");
                            ++bt;
                        }
                    }
                }
            }
        }
        // drain: every issued copy has landed before the CTA may exit
        if (slabs)
            for (int k = sl > 2 ? sl - 2 : 0; k < sl; ++k)
                mbar_wait(smem_u32(&sfull[k & 1]), (uint32_t)(k >> 1) & 1u, err, 23);
        else
            for (int k = bt > TT_NST ? bt - TT_NST : 0; k < bt; ++k)
                mbar_wait(smem_u32(&bfull[k % TT_NST]), (uint32_t)(k / TT_NST) & 1u, err, 23);
    } else if ((warp == 1 || warp == 6) && lane == 0) {
        // ---------------- MMA issuers ----------------
        const int w = warp == 1 ? 0 : 1;
        const uint32_t dcol = tmem + (uint32_t)(w * N);
        const uint32_t idesc = make_idesc(0, 128, N);
        int sl = 0, bt = 0;
        bool ok = true, first = true;
        for (int sc = 0; sc < 8 && ok; ++sc) {
            const int sx = sc & 1, sy = (sc >> 1) & 1, sz = sc >> 2;
            for (int dz = -1; dz <= 1 && ok; ++dz) {
                if (tk + dz < 0 || tk + dz >= hs) continue;
                const int oz = 2 * dz + sz - cz;
                for (int pt = 0; pt < npt && ok; ++pt) {
                    const int buf = sl & 1;
                    if (!(ok = mbar_wait(smem_u32(&sfull[buf]), (uint32_t)(sl >> 1) & 1u, err, 24))) break;
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t sbase = smem_u32(smem + buf * 2 * SLB);
                    for (int dy = -1; dy <= 1 && ok; ++dy) {
                        const int oy = 2 * dy + sy - cy;
                        for (int dx = -1; dx <= 1; ++dx) {
                            const int ox = 2 * dx + sx - cx;
                            if (ox >= -1 && ox <= 1 && oy >= -1 && oy <= 1 && oz >= -1 && oz <= 1) continue;
                            const int mine = bt % TT_NISS == w;
                            const int bs = bt % TT_NST;
                            ++bt;
                            if (!mine) continue;
                            if (!(ok = mbar_wait(smem_u32(&bfull[bs]), (uint32_t)((bt - 1) / TT_NST) & 1u, err, 25)))
                                break;
                            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                            const uint32_t abase = smem_u32(ring + bs * TT_BLK);
                            const uint32_t boff = (uint32_t)((dy + 1) * TT_SBO + (dx + 1) * 16);
                            // K-step 0 descriptors; a K-step adds 256 bytes (A) or 320 bytes (B), i.e. 16
                            // or 20 in the address field (no carry: shared addresses < 2^18)
                            const uint64_t ah = make_desc(abase, 128, TT_KP * 128);
                            const uint64_t al = make_desc(abase + TT_GB, 128, TT_KP * 128);
                            const uint64_t bh = make_desc(sbase + boff, TT_I * 16, TT_SBO);
                            const uint64_t bl = make_desc(sbase + SLB + boff, TT_I * 16, TT_SBO);
                            tc_mma<0>(dcol, ah, bh, idesc, first ? 0u : 1u);
#pragma unroll
                            for (int ks = 1; ks < TT_KP / 2; ++ks) tc_mma<0>(dcol, ah + 16 * ks, bh + 20 * ks, idesc, 1u);
#pragma unroll
                            for (int ks = 0; ks < TT_KP / 2; ++ks) tc_mma<0>(dcol, ah + 16 * ks, bl + 20 * ks, idesc, 1u);
#pragma unroll
                            for (int ks = 0; ks < TT_KP / 2; ++ks) tc_mma<0>(dcol, al + 16 * ks, bh + 20 * ks, idesc, 1u);
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
        // ---------------- epilogue: TMEM (two accumulators) -> FP64 L ----------------
        bool ok = true;
        if (lane == 0) ok = mbar_wait(smem_u32(done), 0u, err, 26);
        ok = __shfl_sync(0xffffffffu, ok, 0);
        __syncwarp();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int q = warp & 3;
        const int n = q * 32 + lane;   // local component of this thread's TMEM lane
        // a 32 x 33 FP32 tile per warp in the slab buffers (free: every copy
        // has been consumed by the MMAs behind `done`)
        float* tile = (float*)smem + (warp - 2) * 32 * 33;
        if (q * 32 < nrows) {
            const int64_t h3 = (int64_t)hs * hs * hs;
            const int64_t tbase = (int64_t)cls * h3 + ((int64_t)tk * hs + TY * tj) * hs + 8 * ti;
            const int rmax = min(32, nrows - q * 32);   // rows of this quadrant holding local components
#pragma unroll 1
            for (int cb = 0; cb < N / 32; ++cb) {
                const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(cb * 32);
                uint32_t v0[32], v1[32];
                tmem_ld32(ta, v0);
                tmem_ld32(ta + (uint32_t)N, v1);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int e = 0; e < 32; ++e)
                    tile[lane * 33 + e] = __uint_as_float(v0[e]) + __uint_as_float(v1[e]);
                __syncwarp();
                // lane = cell (x, y) = (col % 8, col / 8) of the tile, col = 32 cb + lane
                const int col = cb * 32 + lane;
                const int64_t cell = tbase + (int64_t)(col >> 3) * hs + (col & 7);
                if (ok)
                    for (int r = 0; r < rmax; ++r) {
                        if (Lt32) Lt32[(int64_t)(q * 32 + r) * ncell + cell] = tile[r * 33 + lane];
                        else Lt[(int64_t)(q * 32 + r) * ncell + cell] = (double)tile[r * 33 + lane];
                    }
                __syncwarp();
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TT_NISS * N));
    }
}

// A operand of every offset r (343) and K-part: Kt_r(n, m) = D_{n+m}(r)/m!
// for local component n (row) and reduced multipole component m (column),
// zero outside |n| + |m| <= p and in the padding, split into BF16 hi/lo.
// Block of (r, part): hi then lo, each [group 0..10][16-byte column chunk
// 0..5][row 0..7][16 bytes].  One thread per (r, part, group, chunk, row).
__global__ void k_tct_build(int p, int nc, int np, const double* __restrict__ Dtab, unsigned char* __restrict__ B) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)343 * np * TT_G * TT_KP * 8) return;
    const int rr = (int)(t % 8), c = (int)((t / 8) % TT_KP), g = (int)((t / (8 * TT_KP)) % TT_G);
    const int pt = (int)((t / (8 * TT_KP * TT_G)) % np);
    const int r = (int)(t / ((int64_t)8 * TT_KP * TT_G * np));
    const int n = 8 * g + rr, ns = ns_of(p);
    __align__(16) __nv_bfloat16 vh[8], vl[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        const int m = 8 * TT_KP * pt + 8 * c + e;
        double v = 0.0;
        if (n < nc && m < nc) {
            const int nx = c_tl_idx[n][0], ny = c_tl_idx[n][1], nz = c_tl_idx[n][2];
            const int mx = c_tl_idx[m][0], my = c_tl_idx[m][1], mz = c_tl_idx[m][2];
            if (nx + ny + nz + mx + my + mz <= p)
                v = Dtab[(int64_t)r * ns + pos_sym(nx + mx, ny + my, nz + mz)] * c_invfact[mx] * c_invfact[my] *
                    c_invfact[mz];
        }
        vh[e] = __double2bfloat16(v);
        vl[e] = __double2bfloat16(v - (double)__bfloat162float(vh[e]));
    }
    const int64_t off = ((int64_t)r * np + pt) * TT_BLK + g * (TT_KP * 128) + c * 128 + rr * 16;
    *(uint4*)(B + off) = *(const uint4*)vh;
    *(uint4*)(B + off + TT_GB) = *(const uint4*)vl;
}

int tct_build(int p, const double* Dtab, void* B, cudaStream_t s) {
    const int np = tct_np(p);
    if (np < 1 || np > 2) return -1;
    const int64_t tot = (int64_t)343 * np * TT_G * TT_KP * 8;
    k_tct_build<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(p, ncoef_of(p, 1), np, Dtab, (unsigned char*)B);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

// Box of the slab loads of level l: (8 + 2) x (TY + 2) x 1 cells, one K-part.
void tct_box(int l, unsigned (&box)[5]) {
    box[0] = 8;   // BF16 elements of a 16-byte chunk
    box[1] = TT_I;
    box[2] = TT_KP;
    box[3] = (unsigned)(tct_ty(l) + 2);
    box[4] = 1;
}

template <int TY>
static int tct_launch(int l, int np, int npt, int nc, const TcMaps& maps, const void* B, double* Lt, int64_t ncell,
                      int* err, cudaStream_t s, float* Lt32) {
    const int hs = 1 << (l - 1);
    const int smem = tt_smem(TY);
    if (cudaFuncSetAttribute(k_m2l_tc_t<TY>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
        return -2;
    const int tpc = (hs / 8) * (hs / TY) * hs;
    k_m2l_tc_t<TY><<<(unsigned)(8 * tpc), TT_THREADS, smem, s>>>(maps, l, np, npt, nc, (const unsigned char*)B, Lt,
                                                                 ncell, err, Lt32);
    count_launch();
    return 0;
}

// M2L of tensor-core level l (>= 5) with this kernel; the hi/lo operand
// tiles of the level must be in place (k_tc_split_m).  first_part_only:
// only the multipole columns 0..47 (the first K-part) on the tensor cores;
// the columns >= 48 are left to k_m2l_rest (kernel shape 3).
int tct_m2l_level(int p, int l, int first_part_only, const void* maps, const void* B, double* Lt, int* err,
                  cudaStream_t s, float* Lt32) {
    const int hs = 1 << (l - 1);
    const int ty = tct_ty(l);
    if (hs < 16 || hs % ty != 0) return -1;
    const int np = tct_np(p);
    if (np < 1 || np > 2) return -1;
    const int64_t ncell = (int64_t)8 * hs * hs * hs;
    const TcMaps& m = ((const TcLevelMaps*)maps)->tall;
    const int nc = ncoef_of(p, 1);
    const int npt = first_part_only ? 1 : np;
    const int rc = ty == 32 ? tct_launch<32>(l, np, npt, nc, m, B, Lt, ncell, err, s, Lt32)
                            : tct_launch<16>(l, np, npt, nc, m, B, Lt, ncell, err, s, Lt32);
    if (rc != 0) return rc;
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

}  // namespace fmm
