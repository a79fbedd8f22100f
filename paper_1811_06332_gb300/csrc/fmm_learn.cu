// Learned per-pair M2L order (an addition to the paper, which fixes one
// order per run): per-pair features and FP64 truncation-error labels of an
// adaptive plan's M2L list, and an FP32 trainer (forward, backward, Adam)
// for the 11 -> 64 -> 64 -> 64 -> 9 ReLU network that predicts the log10
// force error of a pair's M2L at orders 2..10.
//
// Features of a pair (source A, target B, d = z_B - z_A):
//   a = max(r_A/|d|, 1e-6), b = max(r_B/|d|, 1e-6)
//   f0 = ln(a + b) (the MAC ratio of App. C), f1 = ln a, f2 = ln b,
//   f3..f6 = ln max(|M_A^(j)| / (|M_A,0| r_A^j), 1e-6), j = 1..4,
//   f7..f8 = the same for M_B, j = 1..2,  f9 = ln min(n_A, 1024),
//   f10 = ln min(n_B, 1024),
//   f11 = ln max(g_AB / T_B, 1e-12), g_AB = |M_A,0|/|d|^2 and T_B the sum of
//         g over the M2L lists of B and of all its ancestors,
// with |M^(j)|^2 = sum_{|m|=j} j!/m! M_m^2 (Frobenius norm of the rank-j
// symmetric tensor; a ratio with a zero denominator counts as 0).
// Label of a pair at order p: log10 max(e_p, 1e-12), e_p the error of the
// force of the pair's order-p M2L + L2P (Eqs. M2L, L2P) at up to 64 target
// particles of B (all when n_B <= 64, else sorted positions
// b_B + floor(j n_B/64)) against the direct sum over A's particles, relative
// to the total force at those particles.
#include "fmm_adaptive.h"
#include "fmm_learn.h"

namespace fmm {

// ---------------------------------------------------------------------------
// node data: shape terms of the multipole (ranks 1..4), ln count, radius
// ---------------------------------------------------------------------------
// (multipoles of FP32 plans are stored in the cell's scaled units,
// Mt_m = M_m / h^|m|: the ratio then uses r / h in place of r)
__global__ void k_node_feat(int nn, int ld, const double* __restrict__ Mn, const double* __restrict__ rad,
                            const int* __restrict__ nb, const int* __restrict__ ne, const int* __restrict__ lev,
                            int scaled, double side, float* __restrict__ nodeF) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nn) return;
    const double* M = Mn + (int64_t)c * ld;
    const double m0 = fabs(M[0]), r = scaled ? rad[c] * ldexp(1.0 / side, lev[c]) : rad[c];
    float out[8];
    double rj = 1.0;
    for (int j = 1; j <= 4; ++j) {
        rj *= r;
        double s = 0.0;
        const int b = ns_of(j - 1), e = ns_of(j);
        for (int t = b; t < e; ++t) {
            const double mult = (double)c_fact_small(j) * c_invfact[c_sym_idx[t][0]] * c_invfact[c_sym_idx[t][1]] *
                                c_invfact[c_sym_idx[t][2]];
            s += mult * M[t] * M[t];
        }
        double g = 0.0;
        if (m0 > 0.0 && r > 0.0) g = sqrt(s) / (m0 * rj);
        out[j - 1] = (float)log(g > 1e-6 ? g : 1e-6);
    }
    out[4] = logf((float)min(ne[c] - nb[c], 1024));   // counts saturate at 1024
    out[5] = (float)rad[c];
    out[6] = 0.f;           // T_c, set by the far-field estimate
    out[7] = (float)m0;     // |M_0| (the same in scaled units)
    float4* o = (float4*)(nodeF + 8 * (int64_t)c);
    o[0] = make_float4(out[0], out[1], out[2], out[3]);
    o[1] = make_float4(out[4], out[5], out[6], out[7]);
}

// far-field magnitude estimate: S_c = sum over c's M2L list of |M_A,0|/|d|^2,
// then T_c = sum of S over c and its ancestors (written to nodeF slot 6)
__global__ void k_far_sum(int nn, const int* __restrict__ off, const int* __restrict__ src,
                          const int4* __restrict__ ic, float scale, const float* __restrict__ nodeF,
                          float* __restrict__ S, float* __restrict__ K) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nn) return;
    const int4 it = ic[c];
    float acc = 0.f;
    for (int k = off[c]; k < off[c + 1]; ++k) {
        const int A = src[k];
        const int4 ia = ic[A];
        const float dx = (float)(it.x - ia.x) * scale, dy = (float)(it.y - ia.y) * scale,
                    dz = (float)(it.z - ia.z) * scale;
        acc += nodeF[8 * (int64_t)A + 7] / (dx * dx + dy * dy + dz * dz);
    }
    S[c] = acc;
    K[c] = (float)(off[c + 1] - off[c]);
}
// (also K_c = number of M2L pairs of c and its ancestors, stored as log10 max(K_c, 1))
__global__ void k_far_down(int nn, const int* __restrict__ parent, const float* __restrict__ S,
                           const float* __restrict__ K, float* __restrict__ nodeF, float* __restrict__ nodeK) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nn) return;
    float t = 0.f, kk = 0.f;
    for (int a = c; a >= 0; a = parent[a]) { t += S[a]; kk += K[a]; }
    nodeF[8 * (int64_t)c + 6] = t;
    nodeK[c] = log10f(fmaxf(kk, 1.f));
}

// M2L pair index -> its target (CSR rows expanded)
__global__ void k_pair_target(int nn, const int* __restrict__ off, int* __restrict__ ptgt) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nn) return;
    for (int k = off[c]; k < off[c + 1]; ++k) ptgt[k] = c;
}

__global__ void k_pair_features(int npair, const int* __restrict__ ptgt, const int* __restrict__ msrc,
                                const int4* __restrict__ ic, float scale, const float* __restrict__ nodeF,
                                float* __restrict__ feat) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= npair) return;
    float f[FMM_MLP_NF];
    pair_features(msrc[k], ptgt[k], ic, scale, nodeF, f);
    for (int j = 0; j < FMM_MLP_NF; ++j) feat[(int64_t)k * FMM_MLP_NF + j] = f[j];
}

// ---------------------------------------------------------------------------
// FP64 labels, one warp per pair
// ---------------------------------------------------------------------------
// Full symmetric D_k(r), |k| <= p (Eq. traceless grad), by the recurrence
//   |r|^2 D_k = -[(2k_i - 1) r_i D_{k-e_i} + sum_{j != i} 2 k_j r_j D_{k-e_j}
//                + (k_i - 1)^2 D_{k-2e_i} + sum_{j != i} k_j (k_j - 1) D_{k-2e_j}],
// i the first axis with k_i > 0; lanes split each rank.
static __device__ void dtensor_warp(int p, const double r[3], double* D, int lane) {
    const double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2], ir2 = 1.0 / r2;
    if (lane == 0) D[0] = 1.0 / sqrt(r2);
    __syncwarp();
    for (int j = 1; j <= p; ++j) {
        const int base = ns_of(j - 1), cnt = (j + 1) * (j + 2) / 2;
        for (int t = lane; t < cnt; t += 32) {
            const int s = base + t;
            const int k[3] = {c_sym_idx[s][0], c_sym_idx[s][1], c_sym_idx[s][2]};
            const int i = k[0] > 0 ? 0 : (k[1] > 0 ? 1 : 2);
            double acc = 0.0;
            for (int a = 0; a < 3; ++a) {
                if (k[a] == 0) continue;
                int km[3] = {k[0], k[1], k[2]};
                km[a] -= 1;
                acc += (a == i ? 2.0 * k[a] - 1.0 : 2.0 * k[a]) * r[a] * D[pos_sym(km[0], km[1], km[2])];
                if (k[a] >= 2) {
                    km[a] -= 1;
                    acc += (a == i ? (double)(k[a] - 1) * (k[a] - 1) : (double)k[a] * (k[a] - 1)) *
                           D[pos_sym(km[0], km[1], km[2])];
                }
            }
            D[s] = -acc * ir2;
        }
        __syncwarp();
    }
}

constexpr int LBL_P = 10;
constexpr int LBL_NS = 286;   // ns(10)

template <int WARPS>
__global__ void __launch_bounds__(WARPS * 32)
k_pair_labels(int npair, const int* __restrict__ ptgt, const int* __restrict__ msrc, const double* __restrict__ zc,
              const int* __restrict__ nb, const int* __restrict__ ne, const double* __restrict__ xs,
              const double* __restrict__ ys, const double* __restrict__ zs, const double* __restrict__ qs,
              const double* __restrict__ Mn, int ld, const double* __restrict__ atx,
              const double* __restrict__ aty, const double* __restrict__ atz, double* __restrict__ lab) {
    __shared__ double sM[WARPS][LBL_NS], sD[WARPS][LBL_NS], sL[WARPS][LBL_NS];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int k = blockIdx.x * WARPS + w;
    if (k >= npair) return;
    const int A = msrc[k], B = ptgt[k];
    const double d[3] = {zc[3 * B] - zc[3 * A], zc[3 * B + 1] - zc[3 * A + 1], zc[3 * B + 2] - zc[3 * A + 2]};
    for (int s = lane; s < LBL_NS; s += 32)
        sM[w][s] = Mn[(int64_t)A * ld + s] * c_invfact[c_sym_idx[s][0]] * c_invfact[c_sym_idx[s][1]] *
                   c_invfact[c_sym_idx[s][2]];
    dtensor_warp(LBL_P, d, sD[w], lane);
    // targets of this lane (two at most) and their exact field
    const int bB = nb[B], nB = ne[B] - nb[B];
    const int ny = nB <= 64 ? nB : 64;
    double rb[2][3], g[2][3];
    bool act[2];
    double tot = 0.0;   // squared total force at this lane's targets
    for (int u = 0; u < 2; ++u) {
        const int j = lane + 32 * u;
        act[u] = j < ny;
        g[u][0] = g[u][1] = g[u][2] = 0.0;
        rb[u][0] = rb[u][1] = rb[u][2] = 0.0;
        if (!act[u]) continue;
        const int sp = bB + (nB <= 64 ? j : (int)((int64_t)j * nB / 64));
        tot += atx[sp] * atx[sp] + aty[sp] * aty[sp] + atz[sp] * atz[sp];
        const double y[3] = {xs[sp], ys[sp], zs[sp]};
        for (int c = 0; c < 3; ++c) rb[u][c] = y[c] - zc[3 * B + c];
        for (int a = nb[A]; a < ne[A]; ++a) {
            const double dx = xs[a] - y[0], dy = ys[a] - y[1], dz = zs[a] - y[2];
            const double r2 = dx * dx + dy * dy + dz * dz;
            const double ir = 1.0 / sqrt(r2), ir3 = ir * ir * ir;
            g[u][0] += qs[a] * dx * ir3;
            g[u][1] += qs[a] * dy * ir3;
            g[u][2] += qs[a] * dz * ir3;
        }
    }
    const double den = warp_sum(tot);
    for (int p = 2; p <= LBL_P; ++p) {
        __syncwarp();
        // Eq. M2L at order p: L_n = sum_{|m| <= p-|n|} M_m/m! D_{n+m}
        for (int n = lane; n < ns_of(p); n += 32) {
            const int nx = c_sym_idx[n][0], ny2 = c_sym_idx[n][1], nz = c_sym_idx[n][2];
            const int mcount = ns_of(p - nx - ny2 - nz);
            double v = 0.0;
            for (int m = 0; m < mcount; ++m)
                v += sM[w][m] * sD[w][pos_sym(nx + c_sym_idx[m][0], ny2 + c_sym_idx[m][1], nz + c_sym_idx[m][2])];
            sL[w][n] = v;
        }
        __syncwarp();
        // Eq. L2P gradient at order p: dPhi/dx_i = sum_{|k| <= p-1} rb^k/k! L_{k+e_i}
        double num = 0.0;
        for (int u = 0; u < 2; ++u) {
            if (!act[u]) continue;
            double px[LBL_P + 1], py[LBL_P + 1], pz[LBL_P + 1];
            px[0] = py[0] = pz[0] = 1.0;
            for (int e = 1; e < p; ++e) {
                px[e] = px[e - 1] * rb[u][0] / e;
                py[e] = py[e - 1] * rb[u][1] / e;
                pz[e] = pz[e - 1] * rb[u][2] / e;
            }
            double gx = 0.0, gy = 0.0, gz = 0.0;
            const int nk = ns_of(p - 1);
            for (int s = 0; s < nk; ++s) {
                const int kx = c_sym_idx[s][0], ky = c_sym_idx[s][1], kz = c_sym_idx[s][2];
                const double wgt = px[kx] * py[ky] * pz[kz];
                gx += wgt * sL[w][pos_sym(kx + 1, ky, kz)];
                gy += wgt * sL[w][pos_sym(kx, ky + 1, kz)];
                gz += wgt * sL[w][pos_sym(kx, ky, kz + 1)];
            }
            num += (gx - g[u][0]) * (gx - g[u][0]) + (gy - g[u][1]) * (gy - g[u][1]) +
                   (gz - g[u][2]) * (gz - g[u][2]);
        }
        num = warp_sum(num);
        if (lane == 0) {
            const double e = den > 0.0 ? sqrt(num / den) : 0.0;
            lab[(int64_t)k * FMM_MLP_NOUT + (p - 2)] = log10(e > 1e-12 ? e : 1e-12);
        }
    }
}

// ---------------------------------------------------------------------------
// FP32 trainer
// ---------------------------------------------------------------------------
// feature mean and standard deviation (FP64 sums), one block per feature
__global__ void k_mlp_moments(int64_t n, const float* __restrict__ feat, float* __restrict__ mu,
                              float* __restrict__ sd) {
    __shared__ double s1[256], s2[256];
    const int f = blockIdx.x;
    double a = 0.0, b = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += 256) {
        const double v = feat[i * FMM_MLP_NF + f];
        a += v;
        b += v * v;
    }
    s1[threadIdx.x] = a;
    s2[threadIdx.x] = b;
    __syncthreads();
    for (int o = 128; o; o >>= 1) {
        if (threadIdx.x < o) { s1[threadIdx.x] += s1[threadIdx.x + o]; s2[threadIdx.x] += s2[threadIdx.x + o]; }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double m = s1[0] / (double)n;
        double var = s2[0] / (double)n - m * m;
        const double s = var > 0.0 ? sqrt(var) : 0.0;
        mu[f] = (float)m;
        sd[f] = s > 1e-6 ? (float)s : 1.0f;
    }
}

// Forward and backward of one sample per thread for the batch rows
// order[0..nb); stores the layer inputs (Z0, H1..H3) and the output-side
// gradients of every layer (G1..G4) for the parameter-gradient kernel.
// Loss: mean over the batch and the 9 outputs of (y - t)^2.
__global__ void k_mlp_fb(int nb, int64_t n, const int* __restrict__ order, const float* __restrict__ feat,
                         const float* __restrict__ lab, const float* __restrict__ prm, const float* __restrict__ mu,
                         const float* __restrict__ sd, float* __restrict__ Z0, float* __restrict__ H,
                         float* __restrict__ G, float* __restrict__ G4, float* __restrict__ loss) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nb) return;
    int64_t i = order ? order[s] : s;
    const bool valid = i >= 0 && i < n;   // an index outside the data contributes nothing
    if (!valid) i = 0;
    const MlpView P(prm);
    float z0[FMM_MLP_NF], h[3][FMM_MLP_H], y[FMM_MLP_NOUT];
    for (int f = 0; f < FMM_MLP_NF; ++f) {
        z0[f] = (feat[i * FMM_MLP_NF + f] - mu[f]) / sd[f];
        Z0[(int64_t)s * FMM_MLP_NF + f] = z0[f];
    }
    for (int u = 0; u < FMM_MLP_H; ++u) {
        float a = P.b1[u];
        for (int f = 0; f < FMM_MLP_NF; ++f) a = fmaf(P.W1[u * FMM_MLP_NF + f], z0[f], a);
        h[0][u] = fmaxf(a, 0.f);
    }
    for (int l = 1; l < 3; ++l) {
        const float* W = l == 1 ? P.W2 : P.W3;
        const float* b = l == 1 ? P.b2 : P.b3;
        for (int u = 0; u < FMM_MLP_H; ++u) {
            float a = b[u];
            for (int j = 0; j < FMM_MLP_H; ++j) a = fmaf(W[u * FMM_MLP_H + j], h[l - 1][j], a);
            h[l][u] = fmaxf(a, 0.f);
        }
    }
    float sq = 0.f;
    const float gscale = 2.0f / ((float)nb * FMM_MLP_NOUT);
    for (int k = 0; k < FMM_MLP_NOUT; ++k) {
        float a = P.b4[k];
        for (int j = 0; j < FMM_MLP_H; ++j) a = fmaf(P.W4[k * FMM_MLP_H + j], h[2][j], a);
        const float r = valid ? a - lab[i * FMM_MLP_NOUT + k] : 0.f;
        sq += r * r;
        y[k] = gscale * r;   // dL/dy
        G4[(int64_t)s * FMM_MLP_NOUT + k] = y[k];
    }
    atomicAdd(loss, sq / ((float)nb * FMM_MLP_NOUT));
    for (int l = 0; l < 3; ++l)
        for (int u = 0; u < FMM_MLP_H; ++u) H[((int64_t)l * nb + s) * FMM_MLP_H + u] = h[l][u];
    // backward: g3 = (W4^T dy) * [h3 > 0], g2 = (W3^T g3) * [h2 > 0], g1 = (W2^T g2) * [h1 > 0]
    float gnext[FMM_MLP_H], gcur[FMM_MLP_H];
    for (int j = 0; j < FMM_MLP_H; ++j) {
        float a = 0.f;
        for (int k = 0; k < FMM_MLP_NOUT; ++k) a = fmaf(P.W4[k * FMM_MLP_H + j], y[k], a);
        gcur[j] = h[2][j] > 0.f ? a : 0.f;
        G[((int64_t)2 * nb + s) * FMM_MLP_H + j] = gcur[j];
    }
    for (int l = 2; l >= 1; --l) {
        const float* W = l == 2 ? P.W3 : P.W2;
        for (int j = 0; j < FMM_MLP_H; ++j) {
            float a = 0.f;
            for (int u = 0; u < FMM_MLP_H; ++u) a = fmaf(W[u * FMM_MLP_H + j], gcur[u], a);
            gnext[j] = h[l - 1][j] > 0.f ? a : 0.f;
        }
        for (int j = 0; j < FMM_MLP_H; ++j) {
            gcur[j] = gnext[j];
            G[((int64_t)(l - 1) * nb + s) * FMM_MLP_H + j] = gcur[j];
        }
    }
}

// Parameter gradients summed over the batch, one thread per parameter:
// dW_l[u][j] = sum_s G_l[s][u] X_l[s][j], db_l[u] = sum_s G_l[s][u],
// X_1 = Z0, X_2 = H1, X_3 = H2, X_4 = H3.
__global__ void k_mlp_grad(int nb, const float* __restrict__ Z0, const float* __restrict__ H,
                           const float* __restrict__ G, const float* __restrict__ G4, float* __restrict__ grad) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= FMM_MLP_NPAR) return;
    int l, u, j;   // layer 1..4, output row, input column (-1: bias)
    mlp_param_index(t, l, u, j);
    const int nin = l == 1 ? FMM_MLP_NF : FMM_MLP_H;
    const int nout = l == 4 ? FMM_MLP_NOUT : FMM_MLP_H;
    const float* Gl = l == 4 ? G4 : G + (int64_t)(l - 1) * nb * FMM_MLP_H;
    const float* X = l == 1 ? Z0 : H + (int64_t)(l - 2) * nb * FMM_MLP_H;
    float a = 0.f;
    for (int s = 0; s < nb; ++s) {
        const float gv = Gl[(int64_t)s * nout + u];
        a = fmaf(gv, j < 0 ? 1.f : X[(int64_t)s * nin + j], a);
    }
    grad[t] = a;
}

// Adam: m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
// theta -= lr (m/(1-b1^t)) / (sqrt(v/(1-b2^t)) + eps)
__global__ void k_mlp_adam(float* __restrict__ prm, const float* __restrict__ grad, float* __restrict__ m,
                           float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= FMM_MLP_NPAR) return;
    const float g = grad[t];
    const float mm = b1 * m[t] + (1.f - b1) * g;
    const float vv = b2 * v[t] + (1.f - b2) * g * g;
    m[t] = mm;
    v[t] = vv;
    prm[t] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
int ad_node_features(AdState* a, cudaStream_t s) {
    if (a->nn <= 0) return 0;
    k_node_feat<<<(a->nn + 255) / 256, 256, 0, s>>>(a->nn, a->nc, a->M, a->rad, a->nb, a->ne, a->lev,
                                                    a->pos32 ? 1 : 0, a->side, a->nodeF);
    count_launch();
    return 0;
}

int ad_pair_targets_launch(int nn, int npair, const int* off, int* ptgt, cudaStream_t s) {
    if (npair <= 0 || nn <= 0) return 0;
    k_pair_target<<<(nn + 255) / 256, 256, 0, s>>>(nn, off, ptgt);
    count_launch();
    return 0;
}

__global__ void k_iota(int n, int* __restrict__ a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = i;
}
int ad_iota(int n, int* a, cudaStream_t s) {
    if (n <= 0) return 0;
    k_iota<<<(n + 255) / 256, 256, 0, s>>>(n, a);
    count_launch();
    return 0;
}

__global__ void k_order_keys(int n, const signed char* __restrict__ porder, uint64_t* __restrict__ key,
                             int* __restrict__ val) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    key[k] = (uint64_t)(unsigned char)porder[k];
    val[k] = k;
}
int ad_order_keys(int n, const signed char* porder, uint64_t* key, int* val, cudaStream_t s) {
    if (n <= 0) return 0;
    k_order_keys<<<(n + 255) / 256, 256, 0, s>>>(n, porder, key, val);
    count_launch();
    return 0;
}

// pairs sorted by order (stable, so targets stay ascending inside an order):
// bsrc = their sources, bcnt[q * nn + t] = pairs of target t at order q,
// from the segment boundaries of the key (q, t)
__global__ void k_bucket_csr(int n, int nn, const uint64_t* __restrict__ key, const int* __restrict__ val,
                             const int* __restrict__ ptgt, const int* __restrict__ msrc, int* __restrict__ bsrc,
                             int* __restrict__ bcnt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int k = val[i];
    bsrc[i] = msrc[k];
    const int64_t kk = (int64_t)key[i] * nn + ptgt[k];
    const bool first = i == 0 || ((int64_t)key[i - 1] * nn + ptgt[val[i - 1]]) != kk;
    const bool last = i == n - 1 || ((int64_t)key[i + 1] * nn + ptgt[val[i + 1]]) != kk;
    if (first) atomicAdd(&bcnt[kk], -i);
    if (last) atomicAdd(&bcnt[kk], i + 1);
}
int ad_bucket_csr(int n, int nn, const uint64_t* key, const int* val, const int* ptgt, const int* msrc, int* bsrc,
                  int* bcnt, cudaStream_t s) {
    if (n <= 0) return 0;
    k_bucket_csr<<<(n + 255) / 256, 256, 0, s>>>(n, nn, key, val, ptgt, msrc, bsrc, bcnt);
    count_launch();
    return 0;
}

int ad_far_estimate(AdState* a, cudaStream_t s) {
    if (a->nn <= 0) return 0;
    k_far_sum<<<(a->nn + 255) / 256, 256, 0, s>>>(a->nn, a->moff, a->msrc, a->ic, a->scale32, a->nodeF, a->fsum,
                                                  a->fsum + a->nn);
    k_far_down<<<(a->nn + 255) / 256, 256, 0, s>>>(a->nn, a->parent, a->fsum, a->fsum + a->nn, a->nodeF, a->nodeK);
    count_launch();
    count_launch();
    return 0;
}

int ad_pair_features(AdState* a, float* feat, cudaStream_t s) {
    if (a->nm2l <= 0) return 0;
    k_pair_features<<<(a->nm2l + 255) / 256, 256, 0, s>>>(a->nm2l, a->ptgt, a->msrc, a->ic, a->scale32, a->nodeF,
                                                          feat);
    count_launch();
    return 0;
}

int ad_pair_labels(AdState* a, double* lab, const double* atx, const double* aty, const double* atz, cudaStream_t s) {
    if (a->nm2l <= 0) return 0;
    constexpr int W = 4;
    k_pair_labels<W><<<(a->nm2l + W - 1) / W, W * 32, 0, s>>>(a->nm2l, a->ptgt, a->msrc, a->zc, a->nb, a->ne, a->xs,
                                                             a->ys, a->zs, a->qs, a->M, a->nc, atx, aty, atz, lab);
    count_launch();
    return 0;
}

// One pass of forward + backward over n samples (rows order[0..n) or 0..n),
// leaving the gradient in grad (device) and the loss in loss (device).
static void mlp_batch(int n, int64_t ntot, const int* order, const float* feat, const float* lab, const float* prm,
                      const float* mu, const float* sd, float* scratch, float* grad, float* loss, cudaStream_t s) {
    float* Z0 = scratch;
    float* H = Z0 + (int64_t)n * FMM_MLP_NF;
    float* G = H + (int64_t)3 * n * FMM_MLP_H;
    float* G4 = G + (int64_t)3 * n * FMM_MLP_H;
    k_mlp_fb<<<(n + 127) / 128, 128, 0, s>>>(n, ntot, order, feat, lab, prm, mu, sd, Z0, H, G, G4, loss);
    k_mlp_grad<<<(FMM_MLP_NPAR + 255) / 256, 256, 0, s>>>(n, Z0, H, G, G4, grad);
    count_launch();
    count_launch();
}

static size_t mlp_scratch_floats(int n) {
    return (size_t)n * (FMM_MLP_NF + 6 * FMM_MLP_H + FMM_MLP_NOUT);
}

int mlp_grad_host(const float* blob, int64_t n, const float* feat, const float* lab, float* loss_out, float* grad_out,
                  cudaStream_t s) {
    float *d_blob = nullptr, *d_scr = nullptr, *d_grad = nullptr, *d_loss = nullptr;
    int rc = 0;
    if (cudaMalloc(&d_blob, FMM_MLP_NBLOB * 4) != cudaSuccess ||
        cudaMalloc(&d_scr, mlp_scratch_floats((int)n) * 4) != cudaSuccess ||
        cudaMalloc(&d_grad, FMM_MLP_NPAR * 4) != cudaSuccess || cudaMalloc(&d_loss, 4) != cudaSuccess) {
        rc = -3;
    } else {
        cudaMemcpyAsync(d_blob, blob, FMM_MLP_NBLOB * 4, cudaMemcpyHostToDevice, s);
        cudaMemsetAsync(d_loss, 0, 4, s);
        mlp_batch((int)n, n, nullptr, feat, lab, d_blob + FMM_MLP_OFF_PAR, d_blob + FMM_MLP_OFF_MU,
                  d_blob + FMM_MLP_OFF_SD, d_scr, d_grad, d_loss, s);
        cudaMemcpyAsync(grad_out, d_grad, FMM_MLP_NPAR * 4, cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(loss_out, d_loss, 4, cudaMemcpyDeviceToHost, s);
        if (cudaStreamSynchronize(s) != cudaSuccess) rc = -2;
    }
    cudaFree(d_blob); cudaFree(d_scr); cudaFree(d_grad); cudaFree(d_loss);
    return rc;
}

int mlp_train_host(float* blob, int64_t n, const float* feat, const float* lab, const int* order, int epochs,
                   int batch, float lr, int fit_moments, float* loss_out, cudaStream_t s) {
    const int B = batch;
    float *d_blob = nullptr, *d_scr = nullptr, *d_grad = nullptr, *d_loss = nullptr, *d_m = nullptr, *d_v = nullptr;
    int rc = 0;
    const int nbatch = (int)((n + B - 1) / B);
    if (cudaMalloc(&d_blob, FMM_MLP_NBLOB * 4) != cudaSuccess ||
        cudaMalloc(&d_scr, mlp_scratch_floats(B) * 4) != cudaSuccess ||
        cudaMalloc(&d_grad, FMM_MLP_NPAR * 4) != cudaSuccess ||
        cudaMalloc(&d_loss, (size_t)(epochs > 0 ? epochs : 1) * 4) != cudaSuccess ||
        cudaMalloc(&d_m, FMM_MLP_NPAR * 4) != cudaSuccess || cudaMalloc(&d_v, FMM_MLP_NPAR * 4) != cudaSuccess) {
        rc = -3;
    } else {
        cudaMemcpyAsync(d_blob, blob, FMM_MLP_NBLOB * 4, cudaMemcpyHostToDevice, s);
        cudaMemsetAsync(d_m, 0, FMM_MLP_NPAR * 4, s);
        cudaMemsetAsync(d_v, 0, FMM_MLP_NPAR * 4, s);
        cudaMemsetAsync(d_loss, 0, (size_t)(epochs > 0 ? epochs : 1) * 4, s);
        if (fit_moments) {
            k_mlp_moments<<<FMM_MLP_NF, 256, 0, s>>>(n, feat, d_blob + FMM_MLP_OFF_MU, d_blob + FMM_MLP_OFF_SD);
            count_launch();
        }
        const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
        int64_t t = 0;
        for (int e = 0; e < epochs; ++e) {
            for (int bi = 0; bi < nbatch; ++bi) {
                const int64_t r0 = (int64_t)bi * B;
                const int nb = (int)((n - r0) < B ? (n - r0) : B);
                ++t;
                mlp_batch(nb, n, order + r0, feat, lab, d_blob + FMM_MLP_OFF_PAR, d_blob + FMM_MLP_OFF_MU,
                          d_blob + FMM_MLP_OFF_SD, d_scr, d_grad, d_loss + e, s);
                const float c1 = (float)(1.0 - pow((double)b1, (double)t));
                const float c2 = (float)(1.0 - pow((double)b2, (double)t));
                k_mlp_adam<<<(FMM_MLP_NPAR + 255) / 256, 256, 0, s>>>(d_blob + FMM_MLP_OFF_PAR, d_grad, d_m, d_v, lr,
                                                                     b1, b2, eps, c1, c2);
                count_launch();
            }
        }
        cudaMemcpyAsync(blob, d_blob, FMM_MLP_NBLOB * 4, cudaMemcpyDeviceToHost, s);
        if (loss_out && epochs > 0) cudaMemcpyAsync(loss_out, d_loss, (size_t)epochs * 4, cudaMemcpyDeviceToHost, s);
        if (cudaStreamSynchronize(s) != cudaSuccess) rc = -2;
        if (loss_out)
            for (int e = 0; e < epochs; ++e) loss_out[e] /= (float)nbatch;   // mean batch loss of the epoch
    }
    cudaFree(d_blob); cudaFree(d_scr); cudaFree(d_grad); cudaFree(d_loss); cudaFree(d_m); cudaFree(d_v);
    return rc;
}

}  // namespace fmm
