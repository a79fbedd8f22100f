// General-shift M2M, L2L, L2P (operator-level entry points) and the FP64
// direct sum.
#include "fmm_internal.h"

namespace fmm {

// ---------------------------------------------------------------------------
// General-shift M2M (Eq. M2M / M2M part 2):  Y_n = sum_{k<=n} n!/(k!(n-k)!)
// (-delta)^{n-k} X_k, traceless: Mbar = D[Y].  Public (Mbar) format.
// One warp per item.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128)
k_m2m_general(int p, int basis, int64_t n, const double* __restrict__ Mc, const double* __restrict__ delta,
              double* __restrict__ Mp, const double* __restrict__ detr, const double* __restrict__ expand,
              DevOffsets off) {
    __shared__ double sX[4][FMM_NS_MAX], sY[4][FMM_NS_MAX], sA[4][FMM_NT_MAX];
    __shared__ double sP[4][3][FMM_PMAX + 1];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * 4 + w;
    if (i >= n) return;
    const int ns = ns_of(p), nc = ncoef_of(p, basis);
    if (basis) {
        for (int t = lane; t < nc; t += 32) sA[w][t] = Mc[(int64_t)t * n + i];
        __syncwarp();
        expand_tl_warp(p, sA[w], sX[w], expand, off, lane);
    } else {
        for (int s = lane; s < ns; s += 32) sX[w][s] = Mc[(int64_t)s * n + i];
    }
    if (lane < 3) {
        const double md = -delta[(int64_t)lane * n + i];
        double v = 1.0;
        sP[w][lane][0] = 1.0;
        for (int k = 1; k <= p; ++k) { v *= md; sP[w][lane][k] = v; }
    }
    __syncwarp();
    for (int s = lane; s < ns; s += 32) {
        const int nx = c_sym_idx[s][0], ny = c_sym_idx[s][1], nz = c_sym_idx[s][2];
        double v = 0.0;
        for (int kx = 0; kx <= nx; ++kx)
            for (int ky = 0; ky <= ny; ++ky)
                for (int kz = 0; kz <= nz; ++kz)
                    v += c_binom[nx][kx] * c_binom[ny][ky] * c_binom[nz][kz] * sP[w][0][nx - kx] *
                         sP[w][1][ny - ky] * sP[w][2][nz - kz] * sX[w][pos_sym(kx, ky, kz)];
        sY[w][s] = v;
    }
    __syncwarp();
    if (!basis) {
        for (int s = lane; s < ns; s += 32) Mp[(int64_t)s * n + i] += sY[w][s];
        return;
    }
    for (int t = lane; t < nc; t += 32) {
        const int nx = c_tl_idx[t][0], nz = c_tl_idx[t][2];
        const int j = c_tl_idx[t][0] + c_tl_idx[t][1] + nz;
        const int cols = (j + 1) * (j + 2) / 2;
        const int row = (j - nx) * (j - nx + 1) / 2 + nz;
        const double* R = detr + off.detr[j] + row * cols;
        const double* Ys = &sY[w][ns_of(j - 1)];
        double v = 0.0;
        for (int s = 0; s < cols; ++s) v += R[s] * Ys[s];
        Mp[(int64_t)t * n + i] += v;
    }
}

int launch_m2m_general(int p, int basis, int64_t n, const double* Mc, const double* delta, double* Mp,
                       const DevTables& T, cudaStream_t s) {
    if (n <= 0) return 0;
    k_m2m_general<<<(unsigned)((n + 3) / 4), 128, 0, s>>>(p, basis, n, Mc, delta, Mp, T.detr, T.expand,
                                                          T.offsets());
    count_launch();
    return 0;
}

// ---------------------------------------------------------------------------
// General-shift L2L (Eq. L2L): Y_n = sum_{|k|<=p-|n|} delta^k/k! X_{n+k};
// and L2P (Eq. L2P): Phi = sum_k rb^k/k! X_k, dPhi/dx_i = sum_k rb^k/k! X_{k+e_i}.
// One warp per item, public storage.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128)
k_l2l_general(int p, int basis, int64_t n, const double* __restrict__ Lp, const double* __restrict__ delta,
              double* __restrict__ Lc, const double* __restrict__ expand, DevOffsets off) {
    __shared__ double sX[4][FMM_NS_MAX], sA[4][FMM_NT_MAX];
    __shared__ double sP[4][3][FMM_PMAX + 1];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * 4 + w;
    if (i >= n) return;
    const int ns = ns_of(p), nc = ncoef_of(p, basis);
    if (basis) {
        for (int t = lane; t < nc; t += 32) sA[w][t] = Lp[(int64_t)t * n + i];
        __syncwarp();
        expand_tl_warp(p, sA[w], sX[w], expand, off, lane);
    } else {
        for (int s = lane; s < ns; s += 32) sX[w][s] = Lp[(int64_t)s * n + i];
    }
    if (lane < 3) {
        const double d = delta[(int64_t)lane * n + i];
        double v = 1.0;
        sP[w][lane][0] = 1.0;
        for (int k = 1; k <= p; ++k) { v *= d; sP[w][lane][k] = v * c_invfact[k]; }
    }
    __syncwarp();
    for (int o = lane; o < nc; o += 32) {
        int nx, ny, nz;
        if (basis) { nx = c_tl_idx[o][0]; ny = c_tl_idx[o][1]; nz = c_tl_idx[o][2]; }
        else { nx = c_sym_idx[o][0]; ny = c_sym_idx[o][1]; nz = c_sym_idx[o][2]; }
        const int rem = p - nx - ny - nz;
        double v = 0.0;
        for (int kx = 0; kx <= rem; ++kx)
            for (int ky = 0; ky <= rem - kx; ++ky)
                for (int kz = 0; kz <= rem - kx - ky; ++kz)
                    v += sP[w][0][kx] * sP[w][1][ky] * sP[w][2][kz] * sX[w][pos_sym(nx + kx, ny + ky, nz + kz)];
        Lc[(int64_t)o * n + i] += v;
    }
}

int launch_l2l_general(int p, int basis, int64_t n, const double* Lp, const double* delta, double* Lc,
                       const DevTables& T, cudaStream_t s) {
    if (n <= 0) return 0;
    k_l2l_general<<<(unsigned)((n + 3) / 4), 128, 0, s>>>(p, basis, n, Lp, delta, Lc, T.expand, T.offsets());
    count_launch();
    return 0;
}

__global__ void __launch_bounds__(128)
k_l2p_general(int p, int basis, int64_t n, const double* __restrict__ L, const double* __restrict__ rb,
              double* __restrict__ out, const double* __restrict__ expand, DevOffsets off) {
    __shared__ double sX[4][FMM_NS_MAX], sA[4][FMM_NT_MAX];
    __shared__ double sP[4][3][FMM_PMAX + 1];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * 4 + w;
    if (i >= n) return;
    const int ns = ns_of(p), nc = ncoef_of(p, basis);
    if (basis) {
        for (int t = lane; t < nc; t += 32) sA[w][t] = L[(int64_t)t * n + i];
        __syncwarp();
        expand_tl_warp(p, sA[w], sX[w], expand, off, lane);
    } else {
        for (int s = lane; s < ns; s += 32) sX[w][s] = L[(int64_t)s * n + i];
    }
    if (lane < 3) {
        const double d = rb[(int64_t)lane * n + i];
        double v = 1.0;
        sP[w][lane][0] = 1.0;
        for (int k = 1; k <= p; ++k) { v *= d; sP[w][lane][k] = v * c_invfact[k]; }
    }
    __syncwarp();
    double ph = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
    for (int s = lane; s < ns; s += 32) {
        const int kx = c_sym_idx[s][0], ky = c_sym_idx[s][1], kz = c_sym_idx[s][2];
        const double wgt = sP[w][0][kx] * sP[w][1][ky] * sP[w][2][kz];
        ph += wgt * sX[w][s];
        if (kx + ky + kz < p) {
            gx += wgt * sX[w][pos_sym(kx + 1, ky, kz)];
            gy += wgt * sX[w][pos_sym(kx, ky + 1, kz)];
            gz += wgt * sX[w][pos_sym(kx, ky, kz + 1)];
        }
    }
    ph = warp_sum(ph); gx = warp_sum(gx); gy = warp_sum(gy); gz = warp_sum(gz);
    if (lane == 0) {
        out[i] = ph; out[n + i] = gx; out[2 * n + i] = gy; out[3 * n + i] = gz;
    }
}

int launch_l2p_general(int p, int basis, int64_t n, const double* L, const double* rb, double* out,
                       const DevTables& T, cudaStream_t s) {
    if (n <= 0) return 0;
    k_l2p_general<<<(unsigned)((n + 3) / 4), 128, 0, s>>>(p, basis, n, L, rb, out, T.expand, T.offsets());
    count_launch();
    return 0;
}

// ---------------------------------------------------------------------------
// FP64 direct sum (Eq. PhiAB), shared-memory tiles of sources.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
k_direct(int64_t n, const double* __restrict__ x, const double* __restrict__ y, const double* __restrict__ z,
         const double* __restrict__ q, int64_t nt, const int64_t* __restrict__ targets, double* __restrict__ pot,
         double* __restrict__ ax, double* __restrict__ ay, double* __restrict__ az) {
    __shared__ double sx[256], sy[256], sz[256], sq[256];
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool act = t < nt;
    const int64_t i = act ? (targets ? targets[t] : t) : 0;
    const double xi = act ? x[i] : 0.0, yi = act ? y[i] : 0.0, zi = act ? z[i] : 0.0;
    double ph = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
    for (int64_t b = 0; b < n; b += 256) {
        const int64_t j = b + threadIdx.x;
        __syncthreads();
        if (j < n) { sx[threadIdx.x] = x[j]; sy[threadIdx.x] = y[j]; sz[threadIdx.x] = z[j]; sq[threadIdx.x] = q[j]; }
        __syncthreads();
        const int cnt = (int)min((int64_t)256, n - b);
        for (int k = 0; k < cnt; ++k) {
            if (b + k == i) continue;
            const double dx = sx[k] - xi, dy = sy[k] - yi, dz = sz[k] - zi;
            const double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 == 0.0) continue;
            const double ir = 1.0 / sqrt(r2);
            const double qir3 = sq[k] * ir * ir * ir;
            ph += sq[k] * ir;
            gx += qir3 * dx; gy += qir3 * dy; gz += qir3 * dz;
        }
    }
    if (act) { pot[t] = -ph; ax[t] = gx; ay[t] = gy; az[t] = gz; }
}

int launch_direct(int64_t n, const double* x, const double* y, const double* z, const double* q, int64_t nt,
                  const int64_t* targets, double* pot, double* ax, double* ay, double* az, cudaStream_t s) {
    if (nt <= 0) return 0;
    k_direct<<<(unsigned)((nt + 255) / 256), 256, 0, s>>>(n, x, y, z, q, nt, targets, pot, ax, ay, az);
    count_launch();
    return 0;
}

}  // namespace fmm
