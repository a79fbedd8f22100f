// General-shift M2M, L2L, L2P (operator-level entry points, FP64 or FP32
// storage and arithmetic) and the FP64 direct sum.
#include <algorithm>
#include <cmath>
#include <vector>

#include "fmm_internal.h"

namespace fmm {

template <typename T>
static const T* gtab(const double* d, const float* f);
template <>
const double* gtab<double>(const double* d, const float*) { return d; }
template <>
const float* gtab<float>(const double*, const float* f) { return f; }

// Rebuilds the full symmetric polytensor X from independent traceless
// components A (trace condition, App. B); lanes stride the output.
template <typename T>
__device__ __forceinline__ void expand_tl_warp_t(int p, const T* A, T* X, const T* expand, const DevOffsets& off,
                                                 int lane) {
    const int ns = ns_of(p);
    for (int s = lane; s < ns; s += 32) {
        const int nx = c_sym_idx[s][0], ny = c_sym_idx[s][1], nz = c_sym_idx[s][2];
        const int j = nx + ny + nz;
        const int row = (j - nx) * (j - nx + 1) / 2 + nz;
        const T* E = expand + off.expand[j] + row * (2 * j + 1);
        T v = T(0);
        for (int t = 0; t < 2 * j + 1; ++t) v += E[t] * A[j * j + t];
        X[s] = v;
    }
}

// ---------------------------------------------------------------------------
// General-shift M2M (Eq. M2M / M2M part 2):  Y_n = sum_{k<=n} n!/(k!(n-k)!)
// (-delta)^{n-k} X_k, traceless: Mbar = D[Y].  Public (Mbar) format.
// One warp per item; T is the storage and arithmetic type.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(128)
k_m2m_general(int p, int basis, int64_t n, const T* __restrict__ Mc, const double* __restrict__ delta,
              T* __restrict__ Mp, const T* __restrict__ detr, const T* __restrict__ expand, DevOffsets off) {
    __shared__ T sX[4][FMM_NS_MAX], sY[4][FMM_NS_MAX], sA[4][FMM_NT_MAX];
    __shared__ T sP[4][3][FMM_PMAX + 1];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * 4 + w;
    if (i >= n) return;
    const int ns = ns_of(p), nc = ncoef_of(p, basis);
    if (basis) {
        for (int t = lane; t < nc; t += 32) sA[w][t] = Mc[(int64_t)t * n + i];
        __syncwarp();
        expand_tl_warp_t<T>(p, sA[w], sX[w], expand, off, lane);
    } else {
        for (int s = lane; s < ns; s += 32) sX[w][s] = Mc[(int64_t)s * n + i];
    }
    if (lane < 3) {
        const T md = T(-delta[(int64_t)lane * n + i]);
        T v = T(1);
        sP[w][lane][0] = T(1);
        for (int k = 1; k <= p; ++k) { v *= md; sP[w][lane][k] = v; }
    }
    __syncwarp();
    for (int s = lane; s < ns; s += 32) {
        const int nx = c_sym_idx[s][0], ny = c_sym_idx[s][1], nz = c_sym_idx[s][2];
        T v = T(0);
        for (int kx = 0; kx <= nx; ++kx)
            for (int ky = 0; ky <= ny; ++ky)
                for (int kz = 0; kz <= nz; ++kz)
                    v += T(c_binom[nx][kx] * c_binom[ny][ky] * c_binom[nz][kz]) * sP[w][0][nx - kx] *
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
        const T* R = detr + off.detr[j] + row * cols;
        const T* Ys = &sY[w][ns_of(j - 1)];
        T v = T(0);
        for (int s = 0; s < cols; ++s) v += R[s] * Ys[s];
        Mp[(int64_t)t * n + i] += v;
    }
}

int launch_m2m_general(int prec, int p, int basis, int64_t n, const void* Mc, const double* delta, void* Mp,
                       const DevTables& T, cudaStream_t s) {
    if (n <= 0) return 0;
    const unsigned g = (unsigned)((n + 3) / 4);
    if (prec == 0)
        k_m2m_general<double><<<g, 128, 0, s>>>(p, basis, n, (const double*)Mc, delta, (double*)Mp,
                                                gtab<double>(T.detr, T.detr32), gtab<double>(T.expand, T.expand32),
                                                T.offsets());
    else
        k_m2m_general<float><<<g, 128, 0, s>>>(p, basis, n, (const float*)Mc, delta, (float*)Mp,
                                               gtab<float>(T.detr, T.detr32), gtab<float>(T.expand, T.expand32),
                                               T.offsets());
    count_launch();
    return 0;
}

// ---------------------------------------------------------------------------
// General-shift L2L (Eq. L2L): Y_n = sum_{|k|<=p-|n|} delta^k/k! X_{n+k};
// and L2P (Eq. L2P): Phi = sum_k rb^k/k! X_k, dPhi/dx_i = sum_k rb^k/k! X_{k+e_i}.
// One warp per item, public storage; T is the storage and arithmetic type.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(128)
k_l2l_general(int p, int basis, int64_t n, const T* __restrict__ Lp, const double* __restrict__ delta,
              T* __restrict__ Lc, const T* __restrict__ expand, DevOffsets off) {
    __shared__ T sX[4][FMM_NS_MAX], sA[4][FMM_NT_MAX];
    __shared__ T sP[4][3][FMM_PMAX + 1];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * 4 + w;
    if (i >= n) return;
    const int ns = ns_of(p), nc = ncoef_of(p, basis);
    if (basis) {
        for (int t = lane; t < nc; t += 32) sA[w][t] = Lp[(int64_t)t * n + i];
        __syncwarp();
        expand_tl_warp_t<T>(p, sA[w], sX[w], expand, off, lane);
    } else {
        for (int s = lane; s < ns; s += 32) sX[w][s] = Lp[(int64_t)s * n + i];
    }
    if (lane < 3) {
        const T d = T(delta[(int64_t)lane * n + i]);
        T v = T(1);
        sP[w][lane][0] = T(1);
        for (int k = 1; k <= p; ++k) { v *= d; sP[w][lane][k] = v * T(c_invfact[k]); }
    }
    __syncwarp();
    for (int o = lane; o < nc; o += 32) {
        int nx, ny, nz;
        if (basis) { nx = c_tl_idx[o][0]; ny = c_tl_idx[o][1]; nz = c_tl_idx[o][2]; }
        else { nx = c_sym_idx[o][0]; ny = c_sym_idx[o][1]; nz = c_sym_idx[o][2]; }
        const int rem = p - nx - ny - nz;
        T v = T(0);
        for (int kx = 0; kx <= rem; ++kx)
            for (int ky = 0; ky <= rem - kx; ++ky)
                for (int kz = 0; kz <= rem - kx - ky; ++kz)
                    v += sP[w][0][kx] * sP[w][1][ky] * sP[w][2][kz] * sX[w][pos_sym(nx + kx, ny + ky, nz + kz)];
        Lc[(int64_t)o * n + i] += v;
    }
}

int launch_l2l_general(int prec, int p, int basis, int64_t n, const void* Lp, const double* delta, void* Lc,
                       const DevTables& T, cudaStream_t s) {
    if (n <= 0) return 0;
    const unsigned g = (unsigned)((n + 3) / 4);
    if (prec == 0)
        k_l2l_general<double><<<g, 128, 0, s>>>(p, basis, n, (const double*)Lp, delta, (double*)Lc,
                                                gtab<double>(T.expand, T.expand32), T.offsets());
    else
        k_l2l_general<float><<<g, 128, 0, s>>>(p, basis, n, (const float*)Lp, delta, (float*)Lc,
                                               gtab<float>(T.expand, T.expand32), T.offsets());
    count_launch();
    return 0;
}

template <typename T>
__device__ __forceinline__ T warp_sum_t(T v) {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename T>
__global__ void __launch_bounds__(128)
k_l2p_general(int p, int basis, int64_t n, const T* __restrict__ L, const double* __restrict__ rb,
              T* __restrict__ out, const T* __restrict__ expand, DevOffsets off) {
    __shared__ T sX[4][FMM_NS_MAX], sA[4][FMM_NT_MAX];
    __shared__ T sP[4][3][FMM_PMAX + 1];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * 4 + w;
    if (i >= n) return;
    const int ns = ns_of(p), nc = ncoef_of(p, basis);
    if (basis) {
        for (int t = lane; t < nc; t += 32) sA[w][t] = L[(int64_t)t * n + i];
        __syncwarp();
        expand_tl_warp_t<T>(p, sA[w], sX[w], expand, off, lane);
    } else {
        for (int s = lane; s < ns; s += 32) sX[w][s] = L[(int64_t)s * n + i];
    }
    if (lane < 3) {
        const T d = T(rb[(int64_t)lane * n + i]);
        T v = T(1);
        sP[w][lane][0] = T(1);
        for (int k = 1; k <= p; ++k) { v *= d; sP[w][lane][k] = v * T(c_invfact[k]); }
    }
    __syncwarp();
    T ph = T(0), gx = T(0), gy = T(0), gz = T(0);
    for (int s = lane; s < ns; s += 32) {
        const int kx = c_sym_idx[s][0], ky = c_sym_idx[s][1], kz = c_sym_idx[s][2];
        const T wgt = sP[w][0][kx] * sP[w][1][ky] * sP[w][2][kz];
        ph += wgt * sX[w][s];
        if (kx + ky + kz < p) {
            gx += wgt * sX[w][pos_sym(kx + 1, ky, kz)];
            gy += wgt * sX[w][pos_sym(kx, ky + 1, kz)];
            gz += wgt * sX[w][pos_sym(kx, ky, kz + 1)];
        }
    }
    ph = warp_sum_t(ph); gx = warp_sum_t(gx); gy = warp_sum_t(gy); gz = warp_sum_t(gz);
    if (lane == 0) {
        out[i] = ph; out[n + i] = gx; out[2 * n + i] = gy; out[3 * n + i] = gz;
    }
}

int launch_l2p_general(int prec, int p, int basis, int64_t n, const void* L, const double* rb, void* out,
                       const DevTables& T, cudaStream_t s) {
    if (n <= 0) return 0;
    const unsigned g = (unsigned)((n + 3) / 4);
    if (prec == 0)
        k_l2p_general<double><<<g, 128, 0, s>>>(p, basis, n, (const double*)L, rb, (double*)out,
                                                gtab<double>(T.expand, T.expand32), T.offsets());
    else
        k_l2p_general<float><<<g, 128, 0, s>>>(p, basis, n, (const float*)L, rb, (float*)out,
                                               gtab<float>(T.expand, T.expand32), T.offsets());
    count_launch();
    return 0;
}

// ---------------------------------------------------------------------------
// Fused traceless M2M (Eq. Detracer2, Sec. 2.1): the shift inserted into the
// detracer and regrouped by multipole component q; with j = n + 2k - 2m - q
//   Mbar'_n = sum_q Mbar_q sum_j c_{n,q,j} (-delta)^j,
//   c_{n,q,j} = 1/((2n-1)!! q!) sum_{m <= floor(n/2), |k| = |m|} f_{n,m} (|m|!/k!) (j+q)!/j!
// (the regrouping that reproduces D[shift]).  The coefficients are a table of
// (c, q, j) terms per output row, built once per order on the host; one warp
// per item, lanes over the output rows, FP64.
// ---------------------------------------------------------------------------
struct FusedTerm {
    double c;
    uint16_t q;            // symmetric position of the multipole component
    uint8_t jx, jy, jz, pad;
};

__global__ void __launch_bounds__(128)
k_m2m_fused(int p, int64_t n, const double* __restrict__ Mc, const double* __restrict__ delta,
            double* __restrict__ Mp, const double* __restrict__ expand, DevOffsets off,
            const int* __restrict__ toff, const FusedTerm* __restrict__ terms) {
    __shared__ double sX[4][FMM_NS_MAX], sA[4][FMM_NT_MAX];
    __shared__ double sP[4][3][FMM_PMAX + 1];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * 4 + w;
    if (i >= n) return;
    const int nt = nt_of(p);
    for (int t = lane; t < nt; t += 32) sA[w][t] = Mc[(int64_t)t * n + i];
    __syncwarp();
    expand_tl_warp_t<double>(p, sA[w], sX[w], expand, off, lane);
    if (lane < 3) {
        const double md = -delta[(int64_t)lane * n + i];
        double v = 1.0;
        sP[w][lane][0] = 1.0;
        for (int k = 1; k <= p; ++k) { v *= md; sP[w][lane][k] = v; }
    }
    __syncwarp();
    for (int t = lane; t < nt; t += 32) {
        double v = 0.0;
        for (int e = toff[t]; e < toff[t + 1]; ++e) {
            const FusedTerm T = terms[e];
            v += T.c * sX[w][T.q] * sP[w][0][T.jx] * sP[w][1][T.jy] * sP[w][2][T.jz];
        }
        Mp[(int64_t)t * n + i] += v;
    }
}

// Host: the term table of order p (rows in traceless order).
static void fused_table(int p, std::vector<int>& toff, std::vector<FusedTerm>& terms) {
    auto fact = [](int k) { double f = 1; for (int i = 2; i <= k; ++i) f *= i; return f; };
    auto mf = [&](int a, int b, int c) { return fact(a) * fact(b) * fact(c); };
    auto dfo = [](int k) { double v = 1; for (int i = 2 * k - 1; i > 1; i -= 2) v *= i; return v; };
    const int nt = nt_of(p), ns = ns_of(p);
    toff.assign(1, 0);
    terms.clear();
    std::vector<double> acc;
    for (int t = 0; t < nt; ++t) {
        const unsigned char* nn = fmm_tl_idx[t];
        const int n[3] = {nn[0], nn[1], nn[2]}, an = n[0] + n[1] + n[2];
        for (int iq = 0; iq < ns; ++iq) {
            const unsigned char* qq = fmm_sym_idx[iq];
            const int q[3] = {qq[0], qq[1], qq[2]};
            if (q[0] + q[1] + q[2] > an) continue;
            // accumulate c_{n,q,j} over (m, k) for each j (indexed by j's symmetric position)
            acc.assign(ns, 0.0);
            for (int mx = 0; mx <= n[0] / 2; ++mx)
                for (int my = 0; my <= n[1] / 2; ++my)
                    for (int mz = 0; mz <= n[2] / 2; ++mz) {
                        const int mm = mx + my + mz;
                        double f = dfo(an - mm) * mf(n[0], n[1], n[2]) /
                                   (std::ldexp(1.0, mm) * mf(mx, my, mz) * mf(n[0] - 2 * mx, n[1] - 2 * my, n[2] - 2 * mz));
                        if (mm & 1) f = -f;
                        for (int kx = 0; kx <= mm; ++kx)
                            for (int ky = 0; ky <= mm - kx; ++ky) {
                                const int kz = mm - kx - ky;
                                const int j[3] = {n[0] + 2 * kx - 2 * mx - q[0], n[1] + 2 * ky - 2 * my - q[1],
                                                  n[2] + 2 * kz - 2 * mz - q[2]};
                                if (j[0] < 0 || j[1] < 0 || j[2] < 0) continue;
                                acc[pos_sym(j[0], j[1], j[2])] += f * fact(mm) / mf(kx, ky, kz) *
                                                                 mf(j[0] + q[0], j[1] + q[1], j[2] + q[2]) /
                                                                 mf(j[0], j[1], j[2]);
                            }
                    }
            const double sc = 1.0 / (dfo(an) * mf(q[0], q[1], q[2]));
            for (int ij = 0; ij < ns; ++ij) {
                if (acc[ij] == 0.0) continue;
                FusedTerm T;
                T.c = acc[ij] * sc;
                T.q = (uint16_t)iq;
                T.jx = fmm_sym_idx[ij][0];
                T.jy = fmm_sym_idx[ij][1];
                T.jz = fmm_sym_idx[ij][2];
                T.pad = 0;
                terms.push_back(T);
            }
        }
        toff.push_back((int)terms.size());
    }
}

int launch_m2m_fused(int p, int64_t n, const double* Mc, const double* delta, double* Mp, const DevTables& T,
                     cudaStream_t s) {
    // term tables per device and order, uploaded once
    static int* d_off[64][FMM_PMAX + 1];
    static FusedTerm* d_terms[64][FMM_PMAX + 1];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return -2;
    if (!d_off[dev][p]) {
        std::vector<int> toff;
        std::vector<FusedTerm> terms;
        fused_table(p, toff, terms);
        int* o = nullptr;
        FusedTerm* tm = nullptr;
        if (cudaMalloc(&o, toff.size() * sizeof(int)) != cudaSuccess ||
            cudaMalloc(&tm, (terms.size() + 1) * sizeof(FusedTerm)) != cudaSuccess) {
            cudaFree(o);
            return -3;
        }
        if (cudaMemcpy(o, toff.data(), toff.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
            (!terms.empty() &&
             cudaMemcpy(tm, terms.data(), terms.size() * sizeof(FusedTerm), cudaMemcpyHostToDevice) != cudaSuccess))
            return -2;
        d_off[dev][p] = o;
        d_terms[dev][p] = tm;
    }
    if (n <= 0) return 0;
    k_m2m_fused<<<(unsigned)((n + 3) / 4), 128, 0, s>>>(p, n, Mc, delta, Mp, T.expand, T.offsets(), d_off[dev][p],
                                                         d_terms[dev][p]);
    count_launch();
    return 0;
}

// number of (c, q, j) terms of the fused table of order p (host)
int m2m_fused_terms(int p) {
    std::vector<int> toff;
    std::vector<FusedTerm> terms;
    fused_table(p, toff, terms);
    return (int)terms.size();
}

// ---------------------------------------------------------------------------
// FP64 direct sum (Eq. PhiAB), shared-memory tiles of sources.  A block
// takes 256 targets and the sources of its slice blockIdx.y of gridDim.y;
// with one slice it writes the result, with several it writes its partial
// sums to part[slice][4][nt], which k_direct_sum adds in slice order (the
// result does not depend on scheduling).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
k_direct(int64_t n, const double* __restrict__ x, const double* __restrict__ y, const double* __restrict__ z,
         const double* __restrict__ q, int64_t nt, const int64_t* __restrict__ targets, double* __restrict__ pot,
         double* __restrict__ ax, double* __restrict__ ay, double* __restrict__ az, double* __restrict__ part) {
    __shared__ double sx[256], sy[256], sz[256], sq[256];
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool act = t < nt;
    const int64_t i = act ? (targets ? targets[t] : t) : 0;
    const double xi = act ? x[i] : 0.0, yi = act ? y[i] : 0.0, zi = act ? z[i] : 0.0;
    // the slice: whole tiles of 256 sources
    const int64_t ntile = (n + 255) / 256, per = (ntile + gridDim.y - 1) / gridDim.y;
    const int64_t s0 = (int64_t)blockIdx.y * per * 256, s1 = min(n, s0 + per * 256);
    double ph = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
    for (int64_t b = s0; b < s1; b += 256) {
        const int64_t j = b + threadIdx.x;
        __syncthreads();
        if (j < s1) { sx[threadIdx.x] = x[j]; sy[threadIdx.x] = y[j]; sz[threadIdx.x] = z[j]; sq[threadIdx.x] = q[j]; }
        __syncthreads();
        const int cnt = (int)min((int64_t)256, s1 - b);
        for (int k = 0; k < cnt; ++k) {
            const double dx = sx[k] - xi, dy = sy[k] - yi, dz = sz[k] - zi;
            const double r2 = dx * dx + dy * dy + dz * dz;
            // the self pair and coincident pairs contribute 0
            const double ir = (b + k != i && r2 > 0.0) ? fmm_rsqrt(r2) : 0.0;
            const double qir3 = sq[k] * ir * ir * ir;
            ph += sq[k] * ir;
            gx += qir3 * dx; gy += qir3 * dy; gz += qir3 * dz;
        }
    }
    if (!act) return;
    if (gridDim.y == 1) {
        pot[t] = -ph; ax[t] = gx; ay[t] = gy; az[t] = gz;
    } else {
        double* o = part + (int64_t)blockIdx.y * 4 * nt;
        o[t] = ph; o[nt + t] = gx; o[2 * nt + t] = gy; o[3 * nt + t] = gz;
    }
}

__global__ void k_direct_sum(int64_t nt, int nsl, const double* __restrict__ part, double* __restrict__ pot,
                             double* __restrict__ ax, double* __restrict__ ay, double* __restrict__ az) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    double ph = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
    for (int k = 0; k < nsl; ++k) {
        const double* o = part + (int64_t)k * 4 * nt;
        ph += o[t]; gx += o[nt + t]; gy += o[2 * nt + t]; gz += o[3 * nt + t];
    }
    pot[t] = -ph; ax[t] = gx; ay[t] = gy; az[t] = gz;
}

int launch_direct(int64_t n, const double* x, const double* y, const double* z, const double* q, int64_t nt,
                  const int64_t* targets, double* pot, double* ax, double* ay, double* az, cudaStream_t s) {
    if (nt <= 0) return 0;
    const int64_t nbx = (nt + 255) / 256, ntile = (n + 255) / 256;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // slices of the sources so that about 4 blocks per SM run
    int64_t nsl = (4 * (int64_t)sms + nbx - 1) / nbx;
    nsl = std::max<int64_t>(1, std::min<int64_t>({nsl, 64, ntile}));
    double* part = nullptr;
    if (nsl > 1 && cudaMallocAsync((void**)&part, sizeof(double) * 4 * nt * nsl, s) != cudaSuccess) {
        cudaGetLastError();
        nsl = 1;   // no scratch: one slice
    }
    k_direct<<<dim3((unsigned)nbx, (unsigned)nsl), 256, 0, s>>>(n, x, y, z, q, nt, targets, pot, ax, ay, az, part);
    count_launch();
    if (nsl > 1) {
        k_direct_sum<<<(unsigned)nbx, 256, 0, s>>>(nt, (int)nsl, part, pot, ax, ay, az);
        count_launch();
        cudaFreeAsync(part, s);
    }
    return 0;
}

}  // namespace fmm
