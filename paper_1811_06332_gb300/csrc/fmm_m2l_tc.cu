// Offset-grouped M2L on the 5th-generation tensor cores (Eq. M2L regrouped).
//
// On a uniform level, every target cell of one parity class sees the same
// 189 integer offsets o, and all pairs with one offset share one matrix
//     Kt_o(n, m) = D_{n+m}(-o)/m!      (cell units, |n| + |m| <= p)
// so M2L is a sum of dense products  Lt[T, :] += Mt[T + o, :] . Kt_o^T.
// Per CTA: a tile of 128 target cells (a brick of 8 x 4 x 4 in one class)
// accumulates over all 189 offsets in TMEM:
//     D[128 cells x 96] += A_o[128 cells x 96] . B_o[96 x 96]^T
// with A_o the source multipoles (reduced traceless representative, padded
// 81 -> 96) fetched by a 5-D TMA tensor load whose out-of-range part is
// zero-filled (grid boundary), and B_o the precomputed matrix fetched by a
// bulk copy.  Split precision: x = hi + lo in BF16, three MMAs per K-step
// (hi.hi + hi.lo + lo.hi), FP32 accumulation in TMEM, FP64 write-out.
//
// Roles: warp 0 lane 0 issues copies, warp 1 owns TMEM and lane 0 issues
// tcgen05.mma, warps 2..5 drain TMEM (each reads its lane quadrant).
// Stages form a 3-deep mbarrier ring; every wait is bounded and reports a
// timeout through an error word instead of hanging.
#include <cstdlib>
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include "fmm_internal.h"

namespace fmm {

constexpr int TC_K = 96;                       // padded multipole components (K)
constexpr int TC_N = 96;                       // padded local components (N)
constexpr int TC_CH = TC_K / 8;                // 16-byte chunks along K
constexpr int TC_NCH = TC_N / 16;              // N-chunks of 16 local components
constexpr int TC_A_BYTES = 128 * TC_K * 2;     // 24576
constexpr int TC_BMAX = TC_N * TC_K * 2;       // 18432: bound on one packed matrix
constexpr int TC_STAGES = 3;
constexpr int TC_TMEM_COLS = 128;
constexpr long TC_SPIN = 1L << 24;             // bounded waits

// The matrix of one offset is block-triangular in rank (|n| + |m| <= p), so
// local components are processed in N-chunks of 16: chunk j (rows 16j..16j+15,
// lowest rank a_j) only multiplies multipole components of rank <= p - a_j,
// i.e. the first kch[j] K-steps of 16.  Chunk j's packed block holds 16 rows
// x 16 kch[j] columns in the K-major core-matrix layout (SBO = 256 kch[j]).
struct TcChunks {
    int cw;             // chunk width (local components per chunk, N of one MMA)
    int nch;            // chunks holding real rows
    int kch[TC_NCH];    // K-steps of chunk j
    int boff[TC_NCH];   // byte offset of chunk j inside a packed matrix
    int bbytes;         // bytes of one packed matrix (hi or lo)
    int nst;            // pipeline stages that fit in shared memory (2 or 3)
};

struct TcMaps {
    CUtensorMap hi[8];
    CUtensorMap lo[8];
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* err, int code) {
    for (long it = 0; it < TC_SPIN; ++it) {
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
__device__ __forceinline__ uint64_t make_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version
    return d;                // layout type 0: no swizzle
}

// Instruction descriptor: kind::f16, BF16 x BF16 -> F32, both K-major.
__host__ __device__ constexpr uint32_t make_idesc_bf16(int M, int N) {
    return (1u << 4)                       // D format F32
           | (1u << 7)                     // A format BF16
           | (1u << 10)                    // B format BF16
           | ((uint32_t)(N >> 3) << 17)    // N
           | ((uint32_t)(M >> 4) << 24);   // M
}

__device__ __forceinline__ int floor_half(int v) { return v >= 0 ? v / 2 : -((1 - v) / 2); }

__global__ void __launch_bounds__(192, 1)
k_m2l_tc(const __grid_constant__ TcMaps maps, const TcChunks ch, int l, int nrows,
         const __nv_bfloat16* __restrict__ Kmat, double* __restrict__ Lt, int64_t ncell, int* __restrict__ err) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int TC_STAGE = 2 * TC_A_BYTES + 2 * ch.bbytes;   // bbytes is a multiple of 1024
    uint64_t* bars = (uint64_t*)(smem + ch.nst * TC_STAGE);
    uint64_t* full = bars;                 // [TC_STAGES]
    uint64_t* empty = bars + TC_STAGES;    // [TC_STAGES]
    uint64_t* done = bars + 2 * TC_STAGES;
    uint32_t* tslot = (uint32_t*)(bars + 2 * TC_STAGES + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int hs = 1 << (l - 1);
    const int nti = hs / 8, ntj = hs / 4;
    const int tpc = nti * ntj * (hs / 4);
    const int cls = blockIdx.x / tpc, t = blockIdx.x % tpc;
    const int ti = t % nti, tj = (t / nti) % ntj, tk = t / (nti * ntj);
    const int cx = cls & 1, cy = (cls >> 1) & 1, cz = cls >> 2;

    if (threadIdx.x == 0) {
        for (int s = 0; s < ch.nst; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full[s])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[s])));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(done)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(TC_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;

    if (warp == 0 && lane == 0) {
        // ---------------- producer ----------------
        int it = 0;
        bool ok = true;
        for (int u = 0; u < 216 && ok; ++u) {
            const int ox = -2 - cx + u % 6, oy = -2 - cy + (u / 6) % 6, oz = -2 - cz + u / 36;
            if (ox >= -1 && ox <= 1 && oy >= -1 && oy <= 1 && oz >= -1 && oz <= 1) continue;
            const int s = it % ch.nst;
            const uint32_t ph = (uint32_t)(it / ch.nst) & 1u;
            if (!(ok = mbar_wait(smem_u32(&empty[s]), ph ^ 1u, err, 1))) break;
            const uint32_t fb = smem_u32(&full[s]);
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(TC_STAGE) : "memory");
            const int scls = ((cx + ox) & 1) | (((cy + oy) & 1) << 1) | (((cz + oz) & 1) << 2);
            const int c1 = 8 * ti + floor_half(cx + ox), c3 = 4 * tj + floor_half(cy + oy),
                      c4 = 4 * tk + floor_half(cz + oz);
            unsigned char* st = smem + s * TC_STAGE;
            const CUtensorMap* mh = &maps.hi[scls];
            const CUtensorMap* ml = &maps.lo[scls];
            asm volatile(
                "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(smem_u32(st)),
                "l"((uint64_t)mh), "r"(0), "r"(c1), "r"(0), "r"(c3), "r"(c4), "r"(fb)
                : "memory");
            asm volatile(
                "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(smem_u32(st + TC_A_BYTES)),
                "l"((uint64_t)ml), "r"(0), "r"(c1), "r"(0), "r"(c3), "r"(c4), "r"(fb)
                : "memory");
            const int ridx = (3 - oz) * 49 + (3 - oy) * 7 + (3 - ox);   // r = target - source = -o
            const unsigned char* kb = (const unsigned char*)Kmat + (int64_t)ridx * 2 * ch.bbytes;
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                             smem_u32(st + 2 * TC_A_BYTES)),
                         "l"((uint64_t)kb), "r"(2 * ch.bbytes), "r"(fb)
                         : "memory");
            ++it;
        }
        // drain: every issued stage has landed before the CTA may exit
        const int first = it > ch.nst ? it - ch.nst : 0;
        for (int k = first; k < it; ++k)
            mbar_wait(smem_u32(&full[k % ch.nst]), (uint32_t)(k / ch.nst) & 1u, err, 2);
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer ----------------
        const uint32_t idesc = make_idesc_bf16(128, ch.cw);
        int it = 0;
        bool ok = true;
        for (int u = 0; u < 216; ++u) {
            const int ox = -2 - cx + u % 6, oy = -2 - cy + (u / 6) % 6, oz = -2 - cz + u / 36;
            if (ox >= -1 && ox <= 1 && oy >= -1 && oy <= 1 && oz >= -1 && oz <= 1) continue;
            const int s = it % ch.nst;
            const uint32_t ph = (uint32_t)(it / ch.nst) & 1u;
            if (!(ok = mbar_wait(smem_u32(&full[s]), ph, err, 3))) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t base = smem_u32(smem + s * TC_STAGE);
            const uint32_t a_addr[2] = {base, base + TC_A_BYTES};
            const uint32_t b_addr[2] = {base + 2 * TC_A_BYTES, base + 2 * TC_A_BYTES + ch.bbytes};
            for (int j = 0; j < ch.nch; ++j) {
                const uint32_t dcol = tmem + (uint32_t)(ch.cw * j);
                const uint32_t sbo = 256u * ch.kch[j];
#pragma unroll
                for (int pass = 0; pass < 3; ++pass) {
                    const int ia = pass == 2 ? 1 : 0, ib = pass == 1 ? 1 : 0;   // hi.hi, hi.lo, lo.hi
                    for (int ks = 0; ks < ch.kch[j]; ++ks) {
                        const uint64_t ad = make_desc(a_addr[ia] + ks * 256, 128, TC_CH * 128);
                        const uint64_t bd = make_desc(b_addr[ib] + ch.boff[j] + ks * 256, 128, sbo);
                        const uint32_t acc = (it > 0 || pass > 0 || ks > 0) ? 1u : 0u;
                        asm volatile(
                            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dcol),
                            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                            : "memory");
                    }
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&empty[s]))
                         : "memory");
            ++it;
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(done))
                     : "memory");
        (void)ok;
    } else if (warp >= 2) {
        // ---------------- epilogue: TMEM -> FP64 L ----------------
        bool ok = true;
        if (lane == 0) ok = mbar_wait(smem_u32(done), 0u, err, 4);
        ok = __shfl_sync(0xffffffffu, ok, 0);
        __syncwarp();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int q = warp & 3;
        const int row = q * 32 + lane;
        const int i = row & 7, j = (row >> 3) & 3, k = row >> 5;
        const int64_t h3 = (int64_t)hs * hs * hs;
        const int64_t tg = (int64_t)cls * h3 + ((int64_t)(4 * tk + k) * hs + (4 * tj + j)) * hs + (8 * ti + i);
#pragma unroll
        for (int cb = 0; cb < TC_N / 32; ++cb) {
            uint32_t v[32];
            const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(cb * 32);
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
                "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                  "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
                  "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
                  "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                : "r"(ta));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (ok) {
#pragma unroll
                for (int e = 0; e < 32; ++e) {
                    const int n = cb * 32 + e;
                    if (n < nrows) Lt[(int64_t)n * ncell + tg] = (double)__uint_as_float(v[e]);
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS));
    }
}

// ---------------------------------------------------------------------------
// Operand preparation
// ---------------------------------------------------------------------------
// Multipoles of one level (FP64, [ncoef][ncell], parity-class numbering) ->
// BF16 hi/lo in the TMA layout [class][k][j][chunk][i][8] (components padded
// to 96).  One thread per (cell, chunk).
__global__ void k_tc_split_m(int l, int nc, const double* __restrict__ M, __nv_bfloat16* __restrict__ hi,
                             __nv_bfloat16* __restrict__ lo) {
    const int hs = 1 << (l - 1);
    const int64_t h3 = (int64_t)hs * hs * hs, ncell = 8 * h3;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ncell * TC_CH) return;
    const int c = (int)(t / ncell);
    const int64_t idx = t % ncell;
    const int cls = (int)(idx / h3);
    const int64_t lin = idx % h3;
    const int i = (int)(lin % hs), j = (int)((lin / hs) % hs), k = (int)(lin / ((int64_t)hs * hs));
    __align__(16) __nv_bfloat16 vh[8], vl[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        const int m = 8 * c + e;
        const double x = m < nc ? M[(int64_t)m * ncell + idx] : 0.0;
        const __nv_bfloat16 h = __double2bfloat16(x);
        vh[e] = h;
        vl[e] = __double2bfloat16(x - (double)__bfloat162float(h));
    }
    const int64_t o = ((((int64_t)cls * hs + k) * hs + j) * TC_CH + c) * hs + i;
    *(uint4*)(hi + o * 8) = *(const uint4*)vh;
    *(uint4*)(lo + o * 8) = *(const uint4*)vl;
}

// Kt_r(n, m) = D_{n+m}(r)/m! (traceless basis, reduced multipole columns),
// zero outside |n| + |m| <= p and in the padding, split into BF16 hi/lo and
// stored per offset as N-chunks: chunk j = rows 16j..16j+15 by 16 kch[j]
// columns, K-major core-matrix layout, byte (r/8)*256 kch[j] + (m/8)*128 +
// (r%8)*16 + (m%8)*2 inside the chunk.  One thread per (offset, row, column
// group of 8).
__global__ void k_tc_build_b(int p, int nc, const TcChunks ch, const double* __restrict__ Dtab,
                             __nv_bfloat16* __restrict__ B) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)343 * TC_N * TC_CH) return;
    const int r = (int)(t / (TC_N * TC_CH));
    const int n = (int)((t / TC_CH) % TC_N), c = (int)(t % TC_CH);
    const int j = n / ch.cw, rr = n % ch.cw;
    if (j >= ch.nch || c >= 2 * ch.kch[j]) return;
    const int ns = ns_of(p);
    __align__(16) __nv_bfloat16 vh[8], vl[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        const int m = 8 * c + e;
        double v = 0.0;
        if (n < nc && m < nc) {
            const int nx = c_tl_idx[n][0], ny = c_tl_idx[n][1], nz = c_tl_idx[n][2];
            const int mx = c_tl_idx[m][0], my = c_tl_idx[m][1], mz = c_tl_idx[m][2];
            if (nx + ny + nz + mx + my + mz <= p)
                v = Dtab[(int64_t)r * ns + pos_sym(nx + mx, ny + my, nz + mz)] * c_invfact[mx] * c_invfact[my] *
                    c_invfact[mz];
        }
        const __nv_bfloat16 h = __double2bfloat16(v);
        vh[e] = h;
        vl[e] = __double2bfloat16(v - (double)__bfloat162float(h));
    }
    const int64_t boff = ch.boff[j] + (rr / 8) * 256 * ch.kch[j] + c * 128 + (rr % 8) * 16;   // bytes
    unsigned char* bh = (unsigned char*)B + (int64_t)r * 2 * ch.bbytes;
    *(uint4*)(bh + boff) = *(const uint4*)vh;
    *(uint4*)(bh + ch.bbytes + boff) = *(const uint4*)vl;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

int tc_supported(int p, int basis) { return basis == 1 && p >= 1 && ncoef_of(p, basis) <= TC_K; }
size_t tc_b_bytes() { return (size_t)343 * 2 * TC_BMAX; }

// Chunk width: the N of one MMA.  Wider chunks issue fewer, larger MMAs;
// narrower ones skip more of the zero triangle.  FMM_TC_CHUNK (16, 32, 48 or
// 96) overrides the default for tuning.
static int tc_chunk_width() {
    static int cw = 0;
    if (!cw) {
        cw = 32;
        if (const char* e = getenv("FMM_TC_CHUNK")) {
            const int v = atoi(e);
            if (v == 16 || v == 32 || v == 48 || v == 96) cw = v;
        }
    }
    return cw;
}

static TcChunks tc_chunks(int p) {
    TcChunks c;
    const int nc = ncoef_of(p, 1);
    c.cw = tc_chunk_width();
    c.nch = (nc + c.cw - 1) / c.cw;
    int off = 0;
    for (int j = 0; j < TC_NCH; ++j) {
        c.kch[j] = 0;
        c.boff[j] = off;
        if (j < c.nch) {
            const int r0 = c.cw * j;
            const int a = fmm_tl_idx[r0][0] + fmm_tl_idx[r0][1] + fmm_tl_idx[r0][2];   // lowest rank in chunk
            const int cols = (p - a + 1) * (p - a + 1);
            c.kch[j] = (cols + 15) / 16;
            off += 32 * c.cw * c.kch[j];
        }
    }
    c.bbytes = (off + 1023) / 1024 * 1024;
    c.nst = TC_STAGES * (2 * TC_A_BYTES + 2 * c.bbytes) + 1280 <= 227 * 1024 ? TC_STAGES : 2;
    return c;
}

size_t tc_m_elems(int l) { return l < 1 ? 0 : ((size_t)8 << (3 * (l - 1))) * TC_K; }

int tc_build_b(int p, const double* Dtab, void* B, cudaStream_t s) {
    const int64_t tot = (int64_t)343 * TC_N * TC_CH;
    if (cudaMemsetAsync(B, 0, tc_b_bytes(), s) != cudaSuccess) return -2;
    k_tc_build_b<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(p, ncoef_of(p, 1), tc_chunks(p), Dtab,
                                                               (__nv_bfloat16*)B);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

// Encodes the 16 tensor maps (8 classes x hi/lo) of one level.
// Tensor dims (innermost first): e (8), i (hs), chunk (12), j (hs), k (hs).
int tc_encode_maps(int l, void* hi, void* lo, void* out_maps) {
    if (!g_encode) {
        cudaDriverEntryPointQueryResult q;
        void* fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return -2;
        g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    }
    TcMaps* maps = (TcMaps*)out_maps;
    const cuuint64_t hs = (cuuint64_t)1 << (l - 1);
    const cuuint64_t dims[5] = {8, hs, (cuuint64_t)TC_CH, hs, hs};
    const cuuint64_t strides[4] = {16, hs * 16, (cuuint64_t)TC_CH * hs * 16, hs * TC_CH * hs * 16};
    const cuuint32_t box[5] = {8, 8, (cuuint32_t)TC_CH, 4, 4};
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    const size_t cls_elems = (size_t)hs * hs * hs * TC_K;
    for (int c = 0; c < 8; ++c) {
        for (int h = 0; h < 2; ++h) {
            void* base = (char*)(h ? lo : hi) + c * cls_elems * sizeof(__nv_bfloat16);
            CUresult r = g_encode(h ? &maps->lo[c] : &maps->hi[c], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, base, dims,
                                  strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                  CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) return -1;
        }
    }
    return 0;
}
size_t tc_maps_bytes() { return sizeof(TcMaps); }

int tc_m2l_level(int p, int l, const double* M, void* hi, void* lo, const void* maps, const void* B, double* Lt,
                 int* err, cudaStream_t s) {
    const int hs = 1 << (l - 1);
    if (hs < 8) return -1;
    const int64_t ncell = (int64_t)8 * hs * hs * hs;
    const int nc = ncoef_of(p, 1);
    const int64_t tot = ncell * TC_CH;
    k_tc_split_m<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(l, nc, M, (__nv_bfloat16*)hi, (__nv_bfloat16*)lo);
    count_launch();
    const TcChunks ch = tc_chunks(p);
    const int smem = ch.nst * (2 * TC_A_BYTES + 2 * ch.bbytes) + 1024 + 256;
    if (cudaFuncSetAttribute(k_m2l_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) return -2;
    const int tpc = (hs / 8) * (hs / 4) * (hs / 4);
    k_m2l_tc<<<(unsigned)(8 * tpc), 192, smem, s>>>(*(const TcMaps*)maps, ch, l, nc, (const __nv_bfloat16*)B, Lt,
                                                    ncell, err);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

}  // namespace fmm
