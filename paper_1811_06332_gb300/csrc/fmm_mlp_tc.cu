// Inference of the order-choosing MLP on the 5th-generation tensor cores.
//
// Each CTA (128 threads, persistent over tiles) takes 128 M2L pairs per
// tile, one pair per thread (= one TMEM lane).  The four layers are four
// dense products with FP32 accumulation in TMEM:
//     D[128 x 64] = A[128 x 16] . W1^T      (features, BF16, padded 12 -> 16)
//     D[128 x 64] = A[128 x 64] . W2^T      (h1 in BF16), then W3 the same way
//     D[128 x 16] = A[128 x 64] . W4^T      (9 outputs padded to 16)
// Between layers every thread reads its TMEM row (tcgen05.ld), adds the
// bias, applies ReLU, rounds to BF16 and writes its row of the next A
// operand into shared memory; one thread issues the MMAs and commits them
// to an mbarrier that everyone waits on (bounded).  Operands use the
// K-major, no-swizzle core-matrix layout (8 rows x 16 bytes per core
// matrix): byte (r/8)*SBO + (k/8)*128 + (r%8)*16 + (k%8)*2, SBO = K/8*128.
#include <cuda_bf16.h>
#include <cstring>

#include "fmm_learn.h"

namespace fmm {

constexpr int MT_W1 = 0;        // 64 x 16 BF16: 2048 B
constexpr int MT_W2 = 2048;     // 64 x 64: 8192 B
constexpr int MT_W3 = 10240;    // 64 x 64: 8192 B
constexpr int MT_W4 = 18432;    // 16 x 64: 2048 B
constexpr int MT_F = 20480;     // floats: b1[64] b2[64] b3[64] b4[16] mu[16] sd[16]
constexpr int MT_A = 22528;     // A tile, 128 x 64 BF16: 16384 B
constexpr int MT_BAR = MT_A + 16384;
constexpr int MT_SMEM = MT_BAR + 64 + 1024;   // + alignment slack
constexpr long MT_SPIN = 1L << 24;
constexpr int MT_TMEM_COLS = 64;

static_assert(MLP_DEV_BYTES == MT_F + 1024, "device weight block");

__device__ __forceinline__ uint32_t mt_smem(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool mt_wait(uint32_t bar, uint32_t parity) {
    for (long it = 0; it < MT_SPIN; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ uint64_t mt_desc(uint32_t addr, uint32_t sbo) {
    uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((128u >> 4) & 0x3FFFu) << 16;   // LBO: next core matrix along K
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;    // SBO: next 8-row group
    d |= (uint64_t)1 << 46;
    return d;
}

__host__ __device__ constexpr uint32_t mt_idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// issue ksteps MMAs (K = 16 each) into TMEM column 0 and commit to bar
__device__ __forceinline__ void mt_issue(uint32_t tmem, uint32_t a, uint32_t asbo, uint32_t b, uint32_t bsbo,
                                         int ksteps, uint32_t idesc, uint32_t bar) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    for (int ks = 0; ks < ksteps; ++ks) {
        const uint64_t ad = mt_desc(a + 256u * ks, asbo), bd = mt_desc(b + 256u * ks, bsbo);
        const uint32_t acc = ks > 0 ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
            : "memory");
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void mt_ld32(uint32_t ta, float* out) {
    uint32_t v[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
          "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(ta));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int e = 0; e < 32; ++e) out[e] = __uint_as_float(v[e]);
}

__device__ __forceinline__ void mt_ld16(uint32_t ta, float* out) {
    uint32_t v[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(ta));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int e = 0; e < 16; ++e) out[e] = __uint_as_float(v[e]);
}

// half (32 columns, c0 = 0 or 4 chunks of 8) of row r of the next A operand
// (K = 64) from FP32 values: bias, ReLU, BF16
__device__ __forceinline__ void mt_store_hidden(unsigned char* sA, int r, const float* acc, const float* bias, int c0) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        __align__(16) __nv_bfloat16 h[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) h[e] = __float2bfloat16_rn(fmaxf(acc[8 * c + e] + bias[8 * c + e], 0.f));
        *(uint4*)(sA + (r >> 3) * 1024 + (c0 + c) * 128 + (r & 7) * 16) = *(const uint4*)h;
    }
}

// MODE 0: features read from feat[n][12], predictions written to pred[n][9].
// MODE 1: features of the plan's M2L pairs, the chosen order (lowest p in
//         2..pmax whose prediction is <= thr - log10(K_B)/2, else pmax)
//         written to porder.
template <int MODE>
__global__ void __launch_bounds__(128)
k_mlp_tc(int64_t n, const unsigned char* __restrict__ wdev, const float* __restrict__ feat, float* __restrict__ pred,
         const int* __restrict__ ptgt, const int* __restrict__ msrc, const int4* __restrict__ ic, float scale,
         const float* __restrict__ nodeF, const float* __restrict__ nodeK, float thr, int pmax,
         signed char* __restrict__ porder, int* __restrict__ err) {
    extern __shared__ unsigned char mt_raw[];
    unsigned char* sm = (unsigned char*)(((uintptr_t)mt_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* sA = sm + MT_A;
    const float* sF = (const float*)(sm + MT_F);
    uint64_t* bar = (uint64_t*)(sm + MT_BAR);
    uint32_t* tslot = (uint32_t*)(sm + MT_BAR + 8);
    const int tid = threadIdx.x, warp = tid >> 5;

    for (int i = tid; i < MLP_DEV_BYTES / 16; i += 128) ((uint4*)sm)[i] = ((const uint4*)wdev)[i];
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mt_smem(bar)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(mt_smem(tslot)),
                     "r"(MT_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // weights: generic stores -> tensor core reads
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);   // this warp's lane quadrant
    const uint32_t a_s = mt_smem(sA), w_s = mt_smem(sm), b_s = mt_smem(bar);
    const float *b1 = sF, *b2 = sF + 64, *b3 = sF + 128, *b4 = sF + 192, *mu = sF + 208, *sd = sF + 224;
    uint32_t phase = 0;
    bool ok = true;
    for (int64_t tile = blockIdx.x; (int64_t)tile * 128 < n; tile += gridDim.x) {
        const int64_t k = tile * 128 + tid;
        const bool valid = k < n;
        // ---- features -> BF16 row of A (K = 16)
        float f[FMM_MLP_NF];
        if (valid) {
            if (MODE == 0) {
                for (int j = 0; j < FMM_MLP_NF; ++j) f[j] = feat[k * FMM_MLP_NF + j];
            } else {
                pair_features(msrc[k], ptgt[k], ic, scale, nodeF, f);
            }
        }
        {
            __align__(16) __nv_bfloat16 z[16];
#pragma unroll
            for (int j = 0; j < 16; ++j)
                z[j] = __float2bfloat16_rn((valid && j < FMM_MLP_NF) ? (f[j] - mu[j]) / sd[j] : 0.f);
            *(uint4*)(sA + (tid >> 3) * 256 + (tid & 7) * 16) = *(const uint4*)&z[0];
            *(uint4*)(sA + (tid >> 3) * 256 + 128 + (tid & 7) * 16) = *(const uint4*)&z[8];
        }
        float acc[32];
        for (int layer = 0; layer < 4; ++layer) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
            if (tid == 0) {
                if (layer == 0) mt_issue(tmem, a_s, 256, w_s + MT_W1, 256, 1, mt_idesc(128, 64), b_s);
                else if (layer == 1) mt_issue(tmem, a_s, 1024, w_s + MT_W2, 1024, 4, mt_idesc(128, 64), b_s);
                else if (layer == 2) mt_issue(tmem, a_s, 1024, w_s + MT_W3, 1024, 4, mt_idesc(128, 64), b_s);
                else mt_issue(tmem, a_s, 1024, w_s + MT_W4, 1024, 4, mt_idesc(128, 16), b_s);
            }
            const bool got = mt_wait(b_s, phase);
            ok = __syncthreads_and(got) != 0;
            if (!ok) break;
            phase ^= 1u;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (layer < 3) {
                const float* bias = layer == 0 ? b1 : layer == 1 ? b2 : b3;
                mt_ld32(trow, acc);            // columns 0..31
                mt_store_hidden(sA, tid, acc, bias, 0);
                mt_ld32(trow + 32, acc);       // columns 32..63
                mt_store_hidden(sA, tid, acc, bias + 32, 4);
            } else {
                mt_ld16(trow, acc);
            }
        }
        if (!ok) break;
        if (valid) {
            float y[FMM_MLP_NOUT];
#pragma unroll
            for (int j = 0; j < FMM_MLP_NOUT; ++j) y[j] = acc[j] + b4[j];
            if (MODE == 0) {
                for (int j = 0; j < FMM_MLP_NOUT; ++j) pred[k * FMM_MLP_NOUT + j] = y[j];
            } else {
                // budget per pair: target / sqrt(K_B), K_B the M2L pairs on the
                // target's ancestor chain (nodeK = log10 K_B)
                const float tk = thr - 0.5f * nodeK[ptgt[k]];
                int p = pmax;
                for (int q = pmax; q >= 2; --q)
                    if (y[q - 2] <= tk) p = q;
                porder[k] = (signed char)p;
            }
        }
    }
    if (!ok) {
        if (tid == 0) atomicExch(err, 11);
        mt_wait(b_s, phase);   // bounded: let an MMA still in flight finish before TMEM is freed
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(MT_TMEM_COLS));
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static uint16_t bf16_rne(float v) {
    uint32_t u;
    std::memcpy(&u, &v, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}

static void put_bf16(unsigned char* base, int sbo, int r, int k, float v) {
    const uint16_t h = bf16_rne(v);
    std::memcpy(base + (r / 8) * sbo + (k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2, &h, 2);
}

void mlp_pack_device(const float* blob, unsigned char* out) {
    std::memset(out, 0, MLP_DEV_BYTES);
    const MlpView P(blob + FMM_MLP_OFF_PAR);
    for (int u = 0; u < 64; ++u)
        for (int k = 0; k < 16; ++k) put_bf16(out + MT_W1, 256, u, k, k < FMM_MLP_NF ? P.W1[u * FMM_MLP_NF + k] : 0.f);
    for (int u = 0; u < 64; ++u)
        for (int k = 0; k < 64; ++k) {
            put_bf16(out + MT_W2, 1024, u, k, P.W2[u * 64 + k]);
            put_bf16(out + MT_W3, 1024, u, k, P.W3[u * 64 + k]);
        }
    for (int u = 0; u < 16; ++u)
        for (int k = 0; k < 64; ++k) put_bf16(out + MT_W4, 1024, u, k, u < FMM_MLP_NOUT ? P.W4[u * 64 + k] : 0.f);
    float* F = (float*)(out + MT_F);
    for (int u = 0; u < 64; ++u) { F[u] = P.b1[u]; F[64 + u] = P.b2[u]; F[128 + u] = P.b3[u]; }
    for (int u = 0; u < 16; ++u) {
        F[192 + u] = u < FMM_MLP_NOUT ? P.b4[u] : 0.f;
        F[208 + u] = u < FMM_MLP_NF ? blob[FMM_MLP_OFF_MU + u] : 0.f;
        F[224 + u] = u < FMM_MLP_NF ? blob[FMM_MLP_OFF_SD + u] : 1.f;
    }
}

static int mt_grid(int64_t n, int sms) {
    const int64_t tiles = (n + 127) / 128;
    const int64_t g = (int64_t)sms * 5;   // 5 CTAs per SM: 40 KB shared memory and 72 registers each
    return (int)(tiles < g ? tiles : g);
}

int mlp_predict_dev(const unsigned char* wdev, int64_t n, const float* feat, float* pred, int sms, int* err,
                    cudaStream_t s) {
    if (n <= 0) return 0;
    k_mlp_tc<0><<<mt_grid(n, sms), 128, MT_SMEM, s>>>(n, wdev, feat, pred, nullptr, nullptr, nullptr, 0.f, nullptr,
                                                      nullptr, 0.f, 0, nullptr, err);
    count_launch();
    return 0;
}

int mlp_orders_dev(const unsigned char* wdev, AdState* a, float thr, int pmax, int sms, int* err, cudaStream_t s) {
    if (a->nm2l <= 0) return 0;
    k_mlp_tc<1><<<mt_grid(a->nm2l, sms), 128, MT_SMEM, s>>>(a->nm2l, wdev, nullptr, nullptr, a->ptgt, a->msrc, a->ic,
                                                            a->scale32, a->nodeF, a->nodeK, thr, pmax, a->porder,
                                                            err);
    count_launch();
    return 0;
}

}  // namespace fmm
