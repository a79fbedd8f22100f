// L2P at leaves and the P2P near field.
#include "fmm_internal.h"

namespace fmm {

// ---------------------------------------------------------------------------
// L2P at the leaves (scaled units): Phi = (1/h) sum_k rho^k/k! Lt_k,
// dPhi/dx_i = (1/h^2) sum_k rho^k/k! Lt_{k+e_i}, rho = (x - z_leaf)/h.
// Writes pot = -Phi, acc = +grad Phi into caller order via perm (overwrite).
// One warp per leaf, lanes over the leaf's particles.
// ---------------------------------------------------------------------------
template <int WARPS>
__global__ void __launch_bounds__(WARPS * 32)
k_l2p_leaf(int p, int basis, int depth, int64_t nleaf, const int* __restrict__ start,
           const double* __restrict__ xs, const double* __restrict__ ys, const double* __restrict__ zs,
           const int* __restrict__ perm, const double* __restrict__ Lt, const double* __restrict__ expand,
           DevOffsets off, double* __restrict__ pot, double* __restrict__ ax, double* __restrict__ ay,
           double* __restrict__ az) {
    __shared__ double sX[WARPS][FMM_NS_MAX], sA[WARPS][FMM_NT_MAX];
    __shared__ double sP[WARPS][32][3][FMM_PMAX + 1];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t c = (int64_t)blockIdx.x * WARPS + w;
    if (c >= nleaf) return;
    const int b = start[c], e = start[c + 1];
    if (b == e) return;
    const int ns = ns_of(p), nc = ncoef_of(p, basis);
    if (basis) {
        for (int t = lane; t < nc; t += 32) sA[w][t] = Lt[(int64_t)t * nleaf + c];
        __syncwarp();
        expand_tl_warp(p, sA[w], sX[w], expand, off, lane);
    } else {
        for (int s = lane; s < ns; s += 32) sX[w][s] = Lt[(int64_t)s * nleaf + c];
    }
    __syncwarp();
    int ix, iy, iz;
    cell_coords(depth, c, ix, iy, iz);
    const double inv_h = (double)(1 << depth), h = 1.0 / inv_h;
    const double cx = (ix + 0.5) * h, cy = (iy + 0.5) * h, cz = (iz + 0.5) * h;
    for (int a0 = b; a0 < e; a0 += 32) {
        const int a = a0 + lane;
        if (a < e) {
            double rr[3] = {(xs[a] - cx) * inv_h, (ys[a] - cy) * inv_h, (zs[a] - cz) * inv_h};
            for (int d = 0; d < 3; ++d) {
                double v = 1.0;
                sP[w][lane][d][0] = 1.0;
                for (int k = 1; k <= p; ++k) { v *= rr[d]; sP[w][lane][d][k] = v * c_invfact[k]; }
            }
            double ph = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
            for (int s = 0; s < ns; ++s) {
                const int kx = c_sym_idx[s][0], ky = c_sym_idx[s][1], kz = c_sym_idx[s][2];
                const double wgt = sP[w][lane][0][kx] * sP[w][lane][1][ky] * sP[w][lane][2][kz];
                ph += wgt * sX[w][s];
                if (kx + ky + kz < p) {
                    gx += wgt * sX[w][pos_sym(kx + 1, ky, kz)];
                    gy += wgt * sX[w][pos_sym(kx, ky + 1, kz)];
                    gz += wgt * sX[w][pos_sym(kx, ky, kz + 1)];
                }
            }
            const int o = perm[a];
            pot[o] = -ph * inv_h;
            ax[o] = gx * inv_h * inv_h;
            ay[o] = gy * inv_h * inv_h;
            az[o] = gz * inv_h * inv_h;
        }
    }
}

int launch_l2p_leaf(int p, int basis, int depth, int64_t nleaf, const int* start, const double* xs,
                    const double* ys, const double* zs, const int* perm, const double* Lt, const DevTables& T,
                    double* pot, double* ax, double* ay, double* az, cudaStream_t s) {
    constexpr int WARPS = 2;
    k_l2p_leaf<WARPS><<<(unsigned)((nleaf + WARPS - 1) / WARPS), WARPS * 32, 0, s>>>(
        p, basis, depth, nleaf, start, xs, ys, zs, perm, Lt, T.expand, T.offsets(), pot, ax, ay, az);
    count_launch();
    return 0;
}

// Zero far field (trees too shallow for M2L): overwrite outputs with 0.
__global__ void k_zero4(int64_t n, double* a, double* b, double* c, double* d) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) { a[i] = 0.0; b[i] = 0.0; c[i] = 0.0; d[i] = 0.0; }
}
int launch_zero4(int64_t n, double* a, double* b, double* c, double* d, cudaStream_t s) {
    if (n <= 0) return 0;
    k_zero4<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, a, b, c, d);
    count_launch();
    return 0;
}

// ---------------------------------------------------------------------------
// P2P near field over adjacent leaves (App. C), self excluded, accumulated
// into caller order via perm.  One block per target leaf; sources staged in
// shared memory; positions taken relative to the target leaf centre so that
// the FP32 variant keeps relative accuracy.
// ---------------------------------------------------------------------------
template <typename T, int NT>
__global__ void __launch_bounds__(NT)
k_p2p_leaf(int depth, int64_t nleaf, const int* __restrict__ start, const double* __restrict__ xs,
           const double* __restrict__ ys, const double* __restrict__ zs, const double* __restrict__ qs,
           const int* __restrict__ perm, double* __restrict__ pot, double* __restrict__ ax,
           double* __restrict__ ay, double* __restrict__ az) {
    __shared__ T sx[NT], sy[NT], sz[NT], sq[NT];
    __shared__ int sid[NT];
    const int64_t c = blockIdx.x;
    const int b = start[c], e = start[c + 1];
    if (b == e) return;
    const int side = 1 << depth;
    int ix, iy, iz;
    cell_coords(depth, c, ix, iy, iz);
    const double h = 1.0 / side;
    const double cx = (ix + 0.5) * h, cy = (iy + 0.5) * h, cz = (iz + 0.5) * h;
    for (int t0 = b; t0 < e; t0 += NT) {
        const int ti = t0 + threadIdx.x;
        const bool act = ti < e;
        const T xi = act ? T(xs[ti] - cx) : T(0), yi = act ? T(ys[ti] - cy) : T(0), zi = act ? T(zs[ti] - cz) : T(0);
        T ph = 0, gx = 0, gy = 0, gz = 0;
#pragma unroll 1
        for (int jz = iz - 1; jz <= iz + 1; ++jz) {
            if (jz < 0 || jz >= side) continue;
#pragma unroll 1
            for (int jy = iy - 1; jy <= iy + 1; ++jy) {
                if (jy < 0 || jy >= side) continue;
#pragma unroll 1
                for (int jx = ix - 1; jx <= ix + 1; ++jx) {
                    if (jx < 0 || jx >= side) continue;
                    const int64_t S = cell_index(depth, jx, jy, jz);
                    const int sb = start[S], se = start[S + 1];
                    for (int s0 = sb; s0 < se; s0 += NT) {
                        __syncthreads();
                        const int sj = s0 + threadIdx.x;
                        if (sj < se) {
                            sx[threadIdx.x] = T(xs[sj] - cx);
                            sy[threadIdx.x] = T(ys[sj] - cy);
                            sz[threadIdx.x] = T(zs[sj] - cz);
                            sq[threadIdx.x] = T(qs[sj]);
                            sid[threadIdx.x] = sj;
                        }
                        __syncthreads();
                        const int cnt = min(NT, se - s0);
                        if (act) {
                            for (int k = 0; k < cnt; ++k) {
                                const T dx = sx[k] - xi, dy = sy[k] - yi, dz = sz[k] - zi;
                                const T r2 = dx * dx + dy * dy + dz * dz;
                                if (sid[k] == ti || r2 == T(0)) continue;
                                const T ir = fmm_rsqrt(r2);
                                const T qir = sq[k] * ir;
                                const T qir3 = qir * ir * ir;
                                ph += qir;
                                gx += qir3 * dx; gy += qir3 * dy; gz += qir3 * dz;
                            }
                        }
                    }
                }
            }
        }
        if (act) {
            const int o = perm[ti];
            pot[o] -= (double)ph;
            ax[o] += (double)gx;
            ay[o] += (double)gy;
            az[o] += (double)gz;
        }
    }
}

int launch_p2p_leaf(int prec, int depth, int64_t nleaf, const int* start, const double* xs, const double* ys,
                    const double* zs, const double* qs, const int* perm, double* pot, double* ax, double* ay,
                    double* az, cudaStream_t s) {
    if (nleaf <= 0) return 0;
    if (prec == 0)
        k_p2p_leaf<double, 64><<<(unsigned)nleaf, 64, 0, s>>>(depth, nleaf, start, xs, ys, zs, qs, perm, pot, ax,
                                                              ay, az);
    else
        k_p2p_leaf<float, 64><<<(unsigned)nleaf, 64, 0, s>>>(depth, nleaf, start, xs, ys, zs, qs, perm, pot, ax,
                                                             ay, az);
    count_launch();
    return 0;
}

}  // namespace fmm
