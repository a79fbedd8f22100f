// Learned per-pair M2L order: network shape, parameter layout, the pair
// feature function shared by the feature kernel and the tensor-core
// inference kernel, and the host entry points (fmm_learn.cu, fmm_mlp_tc.cu).
#pragma once
#include "fmm_gb300.h"
#include "fmm_adaptive.h"

namespace fmm {

constexpr int FMM_MLP_H = 64;
constexpr int FMM_MLP_OFF_MU = 8;
constexpr int FMM_MLP_OFF_SD = 8 + FMM_MLP_NF;
constexpr int FMM_MLP_OFF_PAR = 8 + 2 * FMM_MLP_NF;
constexpr int FMM_MLP_NPAR = FMM_MLP_NBLOB - FMM_MLP_OFF_PAR;
static_assert(FMM_MLP_NPAR == 64 * 11 + 64 + 2 * (64 * 64 + 64) + 9 * 64 + 9, "parameter count");

// trainable parameters in blob order: W1 (64x11, row-major), b1, W2 (64x64),
// b2, W3 (64x64), b3, W4 (9x64), b4
struct MlpView {
    const float *W1, *b1, *W2, *b2, *W3, *b3, *W4, *b4;
    __host__ __device__ explicit MlpView(const float* p)
        : W1(p), b1(p + 704), W2(p + 768), b2(p + 4864), W3(p + 4928), b3(p + 9024), W4(p + 9088), b4(p + 9664) {}
};

// parameter t -> layer l (1..4), output row u, input column j (-1: bias)
__host__ __device__ inline void mlp_param_index(int t, int& l, int& u, int& j) {
    if (t < 704) { l = 1; u = t / 11; j = t % 11; }
    else if (t < 768) { l = 1; u = t - 704; j = -1; }
    else if (t < 4864) { l = 2; u = (t - 768) / 64; j = (t - 768) % 64; }
    else if (t < 4928) { l = 2; u = t - 4864; j = -1; }
    else if (t < 9024) { l = 3; u = (t - 4928) / 64; j = (t - 4928) % 64; }
    else if (t < 9088) { l = 3; u = t - 9024; j = -1; }
    else if (t < 9664) { l = 4; u = (t - 9088) / 64; j = (t - 9088) % 64; }
    else { l = 4; u = t - 9664; j = -1; }
}

__host__ __device__ inline double c_fact_small(int j) { return j <= 1 ? 1.0 : j == 2 ? 2.0 : j == 3 ? 6.0 : 24.0; }

// Features of the M2L pair (source A, target B) from per-node data:
// nodeF[8c..8c+7] = (shape_1..shape_4, ln n_c, r_c, 0, 0) and the integer
// centres ic (offset d = (ic_B - ic_A) * scale).
__device__ __forceinline__ void pair_features(int A, int B, const int4* __restrict__ ic, float scale,
                                              const float* __restrict__ nodeF, float* f) {
    const int4 ia = ic[A], ib = ic[B];
    const float dx = (float)(ib.x - ia.x) * scale, dy = (float)(ib.y - ia.y) * scale,
                dz = (float)(ib.z - ia.z) * scale;
    const float dn = sqrtf(dx * dx + dy * dy + dz * dz);
    const float4* nf = (const float4*)nodeF;
    const float4 a0 = nf[2 * A], a1 = nf[2 * A + 1], b0 = nf[2 * B], b1 = nf[2 * B + 1];
    const float ar = fmaxf(a1.y / dn, 1e-6f), br = fmaxf(b1.y / dn, 1e-6f);
    f[0] = logf(ar + br);
    f[1] = logf(ar);
    f[2] = logf(br);
    f[3] = a0.x; f[4] = a0.y; f[5] = a0.z; f[6] = a0.w;
    f[7] = b0.x; f[8] = b0.y;
    f[9] = a1.x;
    f[10] = b1.x;
}

// fmm_learn.cu
int ad_node_features(AdState* a, cudaStream_t s);
int ad_pair_targets_launch(int nn, int npair, const int* off, int* ptgt, cudaStream_t s);
int ad_pair_features(AdState* a, float* feat, cudaStream_t s);
int ad_pair_labels(AdState* a, double* lab, cudaStream_t s);
int mlp_grad_host(const float* blob, int64_t n, const float* feat, const float* lab, float* loss_out, float* grad_out,
                  cudaStream_t s);
int mlp_train_host(float* blob, int64_t n, const float* feat, const float* lab, const int* order, int epochs,
                   int batch, float lr, int fit_moments, float* loss_out, cudaStream_t s);

// fmm_mlp_tc.cu
constexpr int MLP_DEV_BYTES = 20480 + 1024;   // packed BF16 weights + FP32 biases, mu, sd
void mlp_pack_device(const float* blob, unsigned char* out /* MLP_DEV_BYTES */);
int mlp_predict_dev(const unsigned char* wdev, int64_t n, const float* feat, float* pred, int sms, int* err,
                    cudaStream_t s);
int mlp_orders_dev(const unsigned char* wdev, AdState* a, float thr, int pmax, int sms, int* err, cudaStream_t s);

}  // namespace fmm
