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
// offsets of the parameter blocks inside the trainable parameters
constexpr int MLP_W1 = 0, MLP_B1 = 64 * FMM_MLP_NF, MLP_W2 = MLP_B1 + 64, MLP_B2 = MLP_W2 + 64 * 64,
              MLP_W3 = MLP_B2 + 64, MLP_B3 = MLP_W3 + 64 * 64, MLP_W4 = MLP_B3 + 64, MLP_B4 = MLP_W4 + 9 * 64;
static_assert(FMM_MLP_NPAR == MLP_B4 + 9, "parameter count");
constexpr float FMM_MLP_VERSION = 2.f;

// trainable parameters in blob order: W1 (64xNF, row-major), b1, W2 (64x64),
// b2, W3 (64x64), b3, W4 (9x64), b4
struct MlpView {
    const float *W1, *b1, *W2, *b2, *W3, *b3, *W4, *b4;
    __host__ __device__ explicit MlpView(const float* p)
        : W1(p + MLP_W1), b1(p + MLP_B1), W2(p + MLP_W2), b2(p + MLP_B2), W3(p + MLP_W3), b3(p + MLP_B3),
          W4(p + MLP_W4), b4(p + MLP_B4) {}
};

// parameter t -> layer l (1..4), output row u, input column j (-1: bias)
__host__ __device__ inline void mlp_param_index(int t, int& l, int& u, int& j) {
    if (t < MLP_B1) { l = 1; u = t / FMM_MLP_NF; j = t % FMM_MLP_NF; }
    else if (t < MLP_W2) { l = 1; u = t - MLP_B1; j = -1; }
    else if (t < MLP_B2) { l = 2; u = (t - MLP_W2) / 64; j = (t - MLP_W2) % 64; }
    else if (t < MLP_W3) { l = 2; u = t - MLP_B2; j = -1; }
    else if (t < MLP_B3) { l = 3; u = (t - MLP_W3) / 64; j = (t - MLP_W3) % 64; }
    else if (t < MLP_W4) { l = 3; u = t - MLP_B3; j = -1; }
    else if (t < MLP_B4) { l = 4; u = (t - MLP_W4) / 64; j = (t - MLP_W4) % 64; }
    else { l = 4; u = t - MLP_B4; j = -1; }
}

__host__ __device__ inline double c_fact_small(int j) { return j <= 1 ? 1.0 : j == 2 ? 2.0 : j == 3 ? 6.0 : 24.0; }

// Features of the M2L pair (source A, target B) from per-node data:
// nodeF[8c..8c+7] = (shape_1..shape_4, ln n_c, r_c, T_c, |M_c,0|) and the
// integer centres ic (offset d = (ic_B - ic_A) * scale).
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
    f[11] = logf(fmaxf(b1.z > 0.f ? a1.w / (dn * dn) / b1.z : 0.f, 1e-12f));
}

// fmm_learn.cu
int ad_node_features(AdState* a, cudaStream_t s);
int ad_pair_targets_launch(int nn, int npair, const int* off, int* ptgt, cudaStream_t s);
int ad_pair_features(AdState* a, float* feat, cudaStream_t s);
int ad_pair_labels(AdState* a, double* lab, const double* atx, const double* aty, const double* atz, cudaStream_t s);
int ad_far_estimate(AdState* a, cudaStream_t s);
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
