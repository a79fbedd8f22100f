// Leaf kernels of the uniform-octree FMM, specialised per order p and per
// arithmetic type (double for FMM_FP64, float for the reduced-precision
// forms; expansions are stored in FP64 either way):
//   P2M (Eq. P2M):   A_m = sum_a q_a (-(x_a - z)/h)^m, then SYM: Mt = A,
//                    TRACELESS: Mt = reduced representative of D[A];
//   L2P (Eq. L2P):   Phi = (1/h) sum_k rho^k/k! Lt_k,
//                    dPhi/dx_i = (1/h^2) sum_k rho^k/k! Lt_{k+e_i};
//   P2P (near field over adjacent leaves, self excluded).
#include "fmm_internal.h"

namespace fmm {

// ---------------------------------------------------------------------------
// 16-byte shared-memory access helpers (P2M power tables, L2P columns)
// ---------------------------------------------------------------------------
// padded length (a multiple of 16 bytes); offset of column (kx, ky) in the
// column-nested layout of a symmetric tensor of rank <= P
template <typename T>
__host__ __device__ constexpr int pad16(int len) {
    return (len + (int)(16 / sizeof(T)) - 1) / (int)(16 / sizeof(T)) * (int)(16 / sizeof(T));
}
template <int P, typename T>
__host__ __device__ constexpr int nested_col_off(int kx, int ky) {
    int off = 0;
    for (int x = 0; x <= P; ++x)
        for (int y = 0; y <= P - x; ++y) {
            if (x == kx && y == ky) return off;
            off += pad16<T>(P + 1 - x - y);
        }
    return off;
}
// loads n (compile-time after unrolling) consecutive coefficients from a 16-byte aligned shared address
template <typename T, int N>
__device__ __forceinline__ void load16(const T* __restrict__ src, T (&dst)[N]) {
    if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int q = 0; q < (N + 3) / 4; ++q) {
            const float4 v = reinterpret_cast<const float4*>(src)[q];
            if (4 * q + 0 < N) dst[4 * q + 0] = v.x;
            if (4 * q + 1 < N) dst[4 * q + 1] = v.y;
            if (4 * q + 2 < N) dst[4 * q + 2] = v.z;
            if (4 * q + 3 < N) dst[4 * q + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int q = 0; q < (N + 1) / 2; ++q) {
            const double2 v = reinterpret_cast<const double2*>(src)[q];
            if (2 * q + 0 < N) dst[2 * q + 0] = v.x;
            if (2 * q + 1 < N) dst[2 * q + 1] = v.y;
        }
    }
}
// ---------------------------------------------------------------------------
// P2M: one warp per leaf.  Particles are staged 32 at a time together with
// the powers of their offsets (one particle per lane); lane c owns the column
// (nx, ny) of multi-indices and adds q x^nx y^ny z^j for every j of the
// column, one fused product per component and particle.
// ---------------------------------------------------------------------------
template <int P, typename T, int WARPS>
__global__ void __launch_bounds__(WARPS * 32)
k_p2m_leaf(int basis, int depth, int64_t nleaf, const int* __restrict__ start, const double* __restrict__ xs,
           const double* __restrict__ ys, const double* __restrict__ zs, const double* __restrict__ qs,
           double* __restrict__ M, const T* __restrict__ reduce, DevOffsets off,
           const float4* __restrict__ pos32, float* __restrict__ msym, float* __restrict__ M32) {
    constexpr int NS = (P + 1) * (P + 2) * (P + 3) / 6;
    constexpr int NCOL = (P + 1) * (P + 2) / 2;
    // powers per axis; FP32 rows padded to 16 bytes for vector loads (FP64 rows
    // unpadded: at p = 10 padding would pass the 48 KB of static shared memory)
    constexpr int PP = sizeof(T) == 4 ? pad16<T>(P + 1) : P + 1;
    __shared__ T sx[WARPS][32], sy[WARPS][32], sz[WARPS][32], sq[WARPS][32];
    __shared__ __align__(16) T sPw[WARPS][32][3][PP];
    __shared__ T sA[WARPS][NS];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t c = (int64_t)blockIdx.x * WARPS + w;
    if (c >= nleaf) return;
    // the leaf centre in FP64 only for the FP64 coordinates; the FP32 path
    // scales by the exact power of two in FP32 (an FP64 operation costs a
    // warp 16 cycles of this part's narrow FP64 pipe)
    const float inv_hf = (float)(1 << depth);
    double inv_h = 0.0, cx = 0.0, cy = 0.0, cz = 0.0;
    if (!pos32) {
        int ix, iy, iz;
        cell_coords(depth, c, ix, iy, iz);
        inv_h = (double)(1 << depth);
        const double h = 1.0 / inv_h;
        cx = (ix + 0.5) * h; cy = (iy + 0.5) * h; cz = (iz + 0.5) * h;
    }
    const int b = start[c], e = start[c + 1];
    // columns of this lane: col = lane + 32*k -> (nx, ny)
    constexpr int KC = (NCOL + 31) / 32;
    T acc[KC][P + 1];
#pragma unroll
    for (int k = 0; k < KC; ++k)
#pragma unroll
        for (int j = 0; j <= P; ++j) acc[k][j] = T(0);
    int cnx[KC], cny[KC];
#pragma unroll
    for (int k = 0; k < KC; ++k) {
        int col = lane + 32 * k, nx = 0;
        while (nx <= P && col >= P + 1 - nx) { col -= P + 1 - nx; ++nx; }
        cnx[k] = nx;
        cny[k] = col;
    }
    for (int a0 = b; a0 < e; a0 += 32) {
        const int a = a0 + lane;
        __syncwarp();
        if (a < e) {
            if (pos32) {   // FP32 offsets from the leaf centre
                const float4 v = pos32[a];
                sx[w][lane] = T(-v.x * inv_hf);
                sy[w][lane] = T(-v.y * inv_hf);
                sz[w][lane] = T(-v.z * inv_hf);
                sq[w][lane] = T(v.w);
            } else {
                sx[w][lane] = T((cx - xs[a]) * inv_h);   // -(x_a - z)/h
                sy[w][lane] = T((cy - ys[a]) * inv_h);
                sz[w][lane] = T((cz - zs[a]) * inv_h);
                sq[w][lane] = T(qs[a]);
            }
        }
        // powers of the staged offsets, one (particle, axis) per lane: sPw[i][d][j] = r_d^j
        const int cnt = min(32, e - a0);
        if (lane < cnt) {
            const T r[3] = {sx[w][lane], sy[w][lane], sz[w][lane]};
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                T v = T(1);
#pragma unroll
                for (int j = 0; j <= P; ++j) { sPw[w][lane][d][j] = v; v *= r[d]; }
            }
        }
        __syncwarp();
        for (int i = 0; i < cnt; ++i) {
            const T qa = sq[w][i];
            T zp[P + 1];   // the particle's z powers (same address across the warp)
            if constexpr (sizeof(T) == 4) {
                load16<T, P + 1>(sPw[w][i][2], zp);   // 16-byte loads
            } else {
#pragma unroll
                for (int j = 0; j <= P; ++j) zp[j] = sPw[w][i][2][j];
            }
#pragma unroll
            for (int k = 0; k < KC; ++k) {
                if (lane + 32 * k < NCOL) {
                    // q x^nx y^ny, then the column's z powers: one product per
                    // component.  FP32: all P + 1 z powers, unconditionally (the
                    // sums past the column's rank are never stored; a product costs
                    // less than the per-lane test that would skip it); FP64 skips
                    // them, its FMAs being the costly part
                    const T wgt = qa * sPw[w][i][0][cnx[k]] * sPw[w][i][1][cny[k]];
                    const int rem = P - cnx[k] - cny[k];
#pragma unroll
                    for (int j = 0; j <= P; ++j)
                        if (sizeof(T) == 4 || j <= rem) acc[k][j] = fma(wgt, zp[j], acc[k][j]);
                }
            }
        }
    }
    __syncwarp();
#pragma unroll
    for (int k = 0; k < KC; ++k) {
        if (lane + 32 * k < NCOL) {
            const int rem = P - cnx[k] - cny[k];
#pragma unroll
            for (int j = 0; j <= P; ++j)
                if (j <= rem) sA[w][pos_sym(cnx[k], cny[k], j)] = acc[k][j];
        }
    }
    __syncwarp();
    if (!basis) {
        for (int s = lane; s < NS; s += 32) {
            M[(int64_t)s * nleaf + c] = (double)sA[w][s];
            if (M32) M32[(int64_t)s * nleaf + c] = float(sA[w][s]);
        }
        return;
    }
    if (msym) {
        // the symmetric moments, leaf-major (NS padded to 4 per leaf), for
        // k_p2m_reduce: one thread per leaf there instead of this warp's
        // rank-imbalanced rows
        constexpr int NSP = (NS + 3) / 4 * 4;
        for (int s = lane; s < NSP; s += 32) msym[c * NSP + s] = s < NS ? float(sA[w][s]) : 0.f;
        return;
    }
    // reduced representative, in the arithmetic type (FP32 tables for the FP32 form)
    constexpr int NT = (P + 1) * (P + 1);
    for (int t = lane; t < NT; t += 32) {
        const int j = c_tl_idx[t][0] + c_tl_idx[t][1] + c_tl_idx[t][2];
        const int cols = (j + 1) * (j + 2) / 2;
        const T* R = reduce + off.reduce[j] + (t - j * j) * cols;
        const T* As = &sA[w][ns_of(j - 1)];
        T v = T(0);
        for (int s = 0; s < cols; ++s) v += R[s] * As[s];
        M[(int64_t)t * nleaf + c] = (double)v;
        if (M32) M32[(int64_t)t * nleaf + c] = float(v);
    }
}

// ---------------------------------------------------------------------------
// L2P: one half-warp per leaf (two leaves per warp), lanes over particles.
// The expansion (full symmetric, dependent traceless components rebuilt)
// sits in shared memory in a column-nested layout: column (kx, ky) holds
// L[kx, ky, 0..P-kx-ky] contiguously from a 16-byte aligned offset, so a
// lane reads a column with 16-byte loads (the lanes of a half read the same
// address at the same time).  Nested sums
// Phi = sum_kx ax[kx] sum_ky ay[ky] sum_kz az[kz] L[kx,ky,kz].
// ---------------------------------------------------------------------------
// the column sums of one (kx, ky): potential and the three gradient components
template <int P, typename T, int KX, int KY>
__device__ __forceinline__ void l2p_column(const T* __restrict__ Ln, const T (&fz)[P + 1], T& s_p, T& s_gx, T& s_gy,
                                           T& s_gz) {
    constexpr int LEN = P + 1 - KX - KY;
    T c0[LEN];
    load16<T, LEN>(Ln + nested_col_off<P, T>(KX, KY), c0);
    s_p = T(0);
#pragma unroll
    for (int kz = 0; kz < LEN; ++kz) s_p = fma(fz[kz], c0[kz], s_p);
    s_gx = s_gy = s_gz = T(0);
    if constexpr (LEN > 1) {
        T c1[LEN - 1], c2[LEN - 1];
        load16<T, LEN - 1>(Ln + nested_col_off<P, T>(KX + 1, KY), c1);
        load16<T, LEN - 1>(Ln + nested_col_off<P, T>(KX, KY + 1), c2);
#pragma unroll
        for (int kz = 0; kz < LEN - 1; ++kz) {
            s_gx = fma(fz[kz], c1[kz], s_gx);
            s_gy = fma(fz[kz], c2[kz], s_gy);
            s_gz = fma(fz[kz], c0[kz + 1], s_gz);
        }
    }
}
template <int P, typename T, int KX, int KY>
__device__ __forceinline__ void l2p_row(const T* __restrict__ Ln, const T (&fy)[P + 1], const T (&fz)[P + 1],
                                        T& sx_p, T& sx_gx, T& sx_gy, T& sx_gz) {
    if constexpr (KY <= P - KX) {
        T s_p, s_gx, s_gy, s_gz;
        l2p_column<P, T, KX, KY>(Ln, fz, s_p, s_gx, s_gy, s_gz);
        sx_p = fma(fy[KY], s_p, sx_p);
        sx_gx = fma(fy[KY], s_gx, sx_gx);
        sx_gy = fma(fy[KY], s_gy, sx_gy);
        sx_gz = fma(fy[KY], s_gz, sx_gz);
        l2p_row<P, T, KX, KY + 1>(Ln, fy, fz, sx_p, sx_gx, sx_gy, sx_gz);
    }
}
template <int P, typename T, int KX>
__device__ __forceinline__ void l2p_all(const T* __restrict__ Ln, const T (&fx)[P + 1], const T (&fy)[P + 1],
                                        const T (&fz)[P + 1], T& ph, T& gx, T& gy, T& gz) {
    if constexpr (KX <= P) {
        T sx_p = T(0), sx_gx = T(0), sx_gy = T(0), sx_gz = T(0);
        l2p_row<P, T, KX, 0>(Ln, fy, fz, sx_p, sx_gx, sx_gy, sx_gz);
        ph = fma(fx[KX], sx_p, ph);
        gx = fma(fx[KX], sx_gx, gx);
        gy = fma(fx[KX], sx_gy, gy);
        gz = fma(fx[KX], sx_gz, gz);
        l2p_all<P, T, KX + 1>(Ln, fx, fy, fz, ph, gx, gy, gz);
    }
}

template <int P, typename T, int WARPS>
__global__ void __launch_bounds__(WARPS * 32)
k_l2p_leaf2(int basis, int depth, int64_t nleaf, const int* __restrict__ start, const double* __restrict__ xs,
            const double* __restrict__ ys, const double* __restrict__ zs, const int* __restrict__ perm,
            const double* __restrict__ Lt, const T* __restrict__ expand, DevOffsets off,
            double* __restrict__ pot, double* __restrict__ ax, double* __restrict__ ay, double* __restrict__ az,
            const float4* __restrict__ pos32, const float* __restrict__ Lt32) {
    constexpr int NS = (P + 1) * (P + 2) * (P + 3) / 6;
    constexpr int NN = nested_col_off<P, T>(P + 1, 0);   // nested layout size (a multiple of 16 bytes)
    __shared__ T sA[WARPS][2][NS];
    __shared__ __align__(16) T sN[WARPS][2][NN];
    // two leaves per warp, one per half-warp (leaves hold ~16 particles)
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, h = lane >> 4, hl = lane & 15;
    const int64_t c = ((int64_t)blockIdx.x * WARPS + w) * 2 + h;
    const bool valid = c < nleaf;
    const int b = valid ? start[c] : 0, e = valid ? start[c + 1] : 0;
    if (basis) {
        constexpr int NT = (P + 1) * (P + 1);
        for (int t = hl; t < NT; t += 16)
            if (valid) sA[w][h][t] = Lt32 ? T(Lt32[(int64_t)t * nleaf + c]) : T(Lt[(int64_t)t * nleaf + c]);
        __syncwarp();
        for (int s = hl; s < NS; s += 16) {
            if (!valid) continue;
            const int nx = c_sym_idx[s][0], ny = c_sym_idx[s][1], nz = c_sym_idx[s][2];
            const int j = nx + ny + nz;
            const int row = (j - nx) * (j - nx + 1) / 2 + nz;
            const T* E = expand + off.expand[j] + row * (2 * j + 1);
            T v = T(0);
            for (int t = 0; t < 2 * j + 1; ++t) v += E[t] * sA[w][h][j * j + t];
            sN[w][h][nested_col_off<P, T>(nx, ny) + nz] = v;
        }
    } else {
        for (int s = hl; s < NS; s += 16)
            if (valid)
                sN[w][h][nested_col_off<P, T>(c_sym_idx[s][0], c_sym_idx[s][1]) + c_sym_idx[s][2]] =
                    Lt32 ? T(Lt32[(int64_t)s * nleaf + c]) : T(Lt[(int64_t)s * nleaf + c]);
    }
    __syncwarp();
    if (!valid || b == e) return;
    const float inv_hf = (float)(1 << depth);   // exact
    const double inv_h = (double)(1 << depth);
    double cx = 0.0, cy = 0.0, cz = 0.0;
    if (!pos32) {
        int ix, iy, iz;
        cell_coords(depth, c, ix, iy, iz);
        const double hc = 1.0 / inv_h;
        cx = (ix + 0.5) * hc; cy = (iy + 0.5) * hc; cz = (iz + 0.5) * hc;
    }
    const T* Ln = sN[w][h];
    for (int a0 = b; a0 < e; a0 += 16) {
        const int a = a0 + hl;
        if (a >= e) break;
        T rx, ry, rz;
        if (pos32) {
            const float4 v = pos32[a];
            rx = T(v.x * inv_hf); ry = T(v.y * inv_hf); rz = T(v.z * inv_hf);
        } else {
            rx = T((xs[a] - cx) * inv_h); ry = T((ys[a] - cy) * inv_h); rz = T((zs[a] - cz) * inv_h);
        }
        T fx[P + 1], fy[P + 1], fz[P + 1];
        fx[0] = fy[0] = fz[0] = T(1);
#pragma unroll
        for (int k = 1; k <= P; ++k) {
            fx[k] = fx[k - 1] * rx * T(1.0 / k);
            fy[k] = fy[k - 1] * ry * T(1.0 / k);
            fz[k] = fz[k - 1] * rz * T(1.0 / k);
        }
        T ph = 0, gx = 0, gy = 0, gz = 0;
        l2p_all<P, T, 0>(Ln, fx, fy, fz, ph, gx, gy, gz);
        const int o = perm[a];
        if constexpr (sizeof(T) == 4) {
            // scaling by powers of two, exact in FP32 (outside FP32's
            // subnormal range), then one conversion each
            pot[o] = (double)(-ph * inv_hf);
            ax[o] = (double)(gx * inv_hf * inv_hf);
            ay[o] = (double)(gy * inv_hf * inv_hf);
            az[o] = (double)(gz * inv_hf * inv_hf);
        } else {
            pot[o] = -(double)ph * inv_h;
            ax[o] = (double)gx * inv_h * inv_h;
            ay[o] = (double)gy * inv_h * inv_h;
            az[o] = (double)gz * inv_h * inv_h;
        }
    }
}

// ---------------------------------------------------------------------------
// P2P: one warp per target leaf.  Targets of a pass are spread over lane
// groups (tp = next power of two >= targets, G = 32/tp groups), each group
// takes every G-th staged source, and the groups are summed by shuffles.
// ---------------------------------------------------------------------------
template <typename T, int WARPS>
__global__ void __launch_bounds__(WARPS * 32)
k_p2p_leaf2(int depth, int64_t nleaf, const int* __restrict__ start, const double* __restrict__ xs,
            const double* __restrict__ ys, const double* __restrict__ zs, const double* __restrict__ qs,
            const int* __restrict__ perm, double* __restrict__ pot, double* __restrict__ ax,
            double* __restrict__ ay, double* __restrict__ az) {
    __shared__ T sx[WARPS][32], sy[WARPS][32], sz[WARPS][32], sq[WARPS][32];
    __shared__ int sid[WARPS][32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t c = (int64_t)blockIdx.x * WARPS + w;
    if (c >= nleaf) return;
    const int b = start[c], e = start[c + 1];
    if (b == e) return;
    const int side = 1 << depth;
    int ix, iy, iz;
    cell_coords(depth, c, ix, iy, iz);
    const double h = 1.0 / side;
    const double cx = (ix + 0.5) * h, cy = (iy + 0.5) * h, cz = (iz + 0.5) * h;
    for (int t0 = b; t0 < e; t0 += 32) {
        const int tn = min(32, e - t0);
        int tp = 1;
        while (tp < tn) tp <<= 1;
        const int G = 32 / tp, grp = lane / tp, tl = lane % tp;
        const int ti = t0 + tl;
        const bool act = tl < tn;
        const T xi = act ? T(xs[ti] - cx) : T(0), yi = act ? T(ys[ti] - cy) : T(0), zi = act ? T(zs[ti] - cz) : T(0);
        T ph = 0, gx = 0, gy = 0, gz = 0;
#pragma unroll 1
        for (int nb = 0; nb < 27; ++nb) {
            const int jx = ix - 1 + nb % 3, jy = iy - 1 + (nb / 3) % 3, jz = iz - 1 + nb / 9;
            if (jx < 0 || jy < 0 || jz < 0 || jx >= side || jy >= side || jz >= side) continue;
            const int64_t S = cell_index(depth, jx, jy, jz);
            const int sb = start[S], se = start[S + 1];
            for (int s0 = sb; s0 < se; s0 += 32) {
                __syncwarp();
                const int sj = s0 + lane;
                if (sj < se) {
                    sx[w][lane] = T(xs[sj] - cx);
                    sy[w][lane] = T(ys[sj] - cy);
                    sz[w][lane] = T(zs[sj] - cz);
                    sq[w][lane] = T(qs[sj]);
                    sid[w][lane] = sj;
                }
                __syncwarp();
                const int cnt = min(32, se - s0);
                if (act) {
                    for (int k = grp; k < cnt; k += G) {
                        const T dx = sx[w][k] - xi, dy = sy[w][k] - yi, dz = sz[w][k] - zi;
                        const T r2 = dx * dx + dy * dy + dz * dz;
                        // the self pair and coincident pairs contribute 0
                        const T ir = (sid[w][k] != ti && r2 > T(0)) ? fmm_rsqrt(r2) : T(0);
                        const T qir = sq[w][k] * ir;
                        const T qir3 = qir * ir * ir;
                        ph += qir;
                        gx += qir3 * dx; gy += qir3 * dy; gz += qir3 * dz;
                    }
                }
            }
        }
        for (int o = tp; o < 32; o <<= 1) {
            ph += __shfl_xor_sync(0xffffffffu, ph, o);
            gx += __shfl_xor_sync(0xffffffffu, gx, o);
            gy += __shfl_xor_sync(0xffffffffu, gy, o);
            gz += __shfl_xor_sync(0xffffffffu, gz, o);
        }
        if (act && grp == 0) {
            const int o = perm[ti];
            pot[o] -= (double)ph;
            ax[o] += (double)gx;
            ay[o] += (double)gy;
            az[o] += (double)gz;
        }
    }
}

template <typename T>
static const T* tab_of(const double* d, const float* f);
template <>
const double* tab_of<double>(const double* d, const float*) { return d; }
template <>
const float* tab_of<float>(const double*, const float* f) { return f; }

// rank J of k_p2m_reduce (RO: offset of its rows in the map, S0: of its
// moments), then the next rank; every bound is a compile-time constant
template <int P, int J, int RO, int S0>
__device__ __forceinline__ void p2m_reduce_rank(const float* sR, const float* a, double* M, float* M32,
                                                int64_t nleaf, int64_t c) {
    if constexpr (J <= P) {
        constexpr int cols = (J + 1) * (J + 2) / 2;
        // the rank's moments by 16-byte loads of the aligned span around them
        constexpr int A0 = S0 / 4 * 4, A1 = (S0 + cols + 3) / 4 * 4;
        float v[A1 - A0];
#pragma unroll
        for (int k = 0; k < A1 - A0; k += 4) {
            const float4 q = *(const float4*)(a + A0 + k);
            v[k] = q.x; v[k + 1] = q.y; v[k + 2] = q.z; v[k + 3] = q.w;
        }
        float m[cols];
#pragma unroll
        for (int k = 0; k < cols; ++k) m[k] = v[S0 - A0 + k];
#pragma unroll 1
        for (int u = 0; u < 2 * J + 1; ++u) {
            const float* R = sR + RO + u * cols;
            float v = 0.f;
#pragma unroll
            for (int k = 0; k < cols; ++k) v = fmaf(R[k], m[k], v);
            M[(int64_t)(J * J + u) * nleaf + c] = (double)v;
            if (M32) M32[(int64_t)(J * J + u) * nleaf + c] = v;
        }
        p2m_reduce_rank<P, J + 1, RO + (2 * J + 1) * cols, S0 + cols>(sR, a, M, M32, nleaf, c);
    }
}

// Reduced traceless representative of the leaves' symmetric moments (FP32
// form), one thread per leaf: row t of rank j is the dot product of the
// exact map's row with the rank-j moments, summed in the order of the
// warp-per-leaf form (so the result is the same bit for bit); the map sits in
// shared memory and every thread of a warp reads the same entry.
template <int P>
__global__ void __launch_bounds__(128)
k_p2m_reduce(int64_t nleaf, const float* __restrict__ msym, const float* __restrict__ reduce, DevOffsets off,
             double* __restrict__ M, float* __restrict__ M32) {
    constexpr int NS = (P + 1) * (P + 2) * (P + 3) / 6, NSP = (NS + 3) / 4 * 4;
    constexpr int RT = [] {
        int t = 0;
        for (int j = 0; j <= P; ++j) t += (2 * j + 1) * (j + 1) * (j + 2) / 2;
        return t;
    }();
    __shared__ float sR[RT];
    {
        int o = 0;
        for (int j = 0; j <= P; ++j) {
            const int sz = (2 * j + 1) * (j + 1) * (j + 2) / 2;
            for (int i = threadIdx.x; i < sz; i += blockDim.x) sR[o + i] = reduce[off.reduce[j] + i];
            o += sz;
        }
    }
    __syncthreads();
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nleaf) return;
    p2m_reduce_rank<P, 0, 0, 0>(sR, msym + c * NSP, M, M32, nleaf, c);
}

template <int P, typename T>
static void p2m_leaf_p(int basis, int depth, int64_t nleaf, const int* start, const double* xs, const double* ys,
                       const double* zs, const double* qs, double* M, const DevTables& Tb, cudaStream_t s,
                       const float4* pos32, float* msym, float* M32) {
    constexpr int W = 4;
    const bool split = sizeof(T) == 4 && basis && msym;
    k_p2m_leaf<P, T, W><<<(unsigned)((nleaf + W - 1) / W), W * 32, 0, s>>>(basis, depth, nleaf, start, xs, ys, zs,
                                                                           qs, M, tab_of<T>(Tb.reduce, Tb.reduce32),
                                                                           Tb.offsets(), pos32,
                                                                           split ? msym : nullptr, M32);
    if (split) {
        k_p2m_reduce<P><<<(unsigned)((nleaf + 127) / 128), 128, 0, s>>>(nleaf, msym, Tb.reduce32, Tb.offsets(), M,
                                                                        M32);
        count_launch();
    }
}
template <int P, typename T>
static void l2p_leaf_p(int basis, int depth, int64_t nleaf, const int* start, const double* xs, const double* ys,
                       const double* zs, const int* perm, const double* Lt, const DevTables& Tb, double* pot,
                       double* ax, double* ay, double* az, cudaStream_t s, const float4* pos32, const float* Lt32) {
    constexpr int W = 4;
    k_l2p_leaf2<P, T, W><<<(unsigned)((nleaf + 2 * W - 1) / (2 * W)), W * 32, 0, s>>>(
        basis, depth, nleaf, start, xs, ys, zs, perm, Lt, tab_of<T>(Tb.expand, Tb.expand32), Tb.offsets(), pot, ax,
        ay, az, pos32, Lt32);
}

#define FMM_P_SWITCH(P_, CALL) \
    switch (P_) {              \
        case 0: CALL(0); break; case 1: CALL(1); break; case 2: CALL(2); break; case 3: CALL(3); break; \
        case 4: CALL(4); break; case 5: CALL(5); break; case 6: CALL(6); break; case 7: CALL(7); break; \
        case 8: CALL(8); break; case 9: CALL(9); break; default: CALL(10); break; }

int launch_p2m_leaf(int prec, int p, int basis, int depth, int64_t nleaf, const int* start, const double* xs,
                    const double* ys, const double* zs, const double* qs, double* M, const DevTables& Tb,
                    cudaStream_t s, const float4* pos32, float* msym, float* M32) {
    if (nleaf <= 0) return 0;
#define C64(P) p2m_leaf_p<P, double>(basis, depth, nleaf, start, xs, ys, zs, qs, M, Tb, s, nullptr, nullptr, nullptr)
#define C32(P) p2m_leaf_p<P, float>(basis, depth, nleaf, start, xs, ys, zs, qs, M, Tb, s, pos32, msym, M32)
    if (prec == 0) { FMM_P_SWITCH(p, C64) } else { FMM_P_SWITCH(p, C32) }
#undef C64
#undef C32
    count_launch();
    return 0;
}

int launch_l2p_leaf2(int prec, int p, int basis, int depth, int64_t nleaf, const int* start, const double* xs,
                     const double* ys, const double* zs, const int* perm, const double* Lt, const DevTables& Tb,
                     double* pot, double* ax, double* ay, double* az, cudaStream_t s, const float4* pos32,
                     const float* Lt32) {
    if (nleaf <= 0) return 0;
#define C64(P) l2p_leaf_p<P, double>(basis, depth, nleaf, start, xs, ys, zs, perm, Lt, Tb, pot, ax, ay, az, s, nullptr, \
                                     nullptr)
#define C32(P) l2p_leaf_p<P, float>(basis, depth, nleaf, start, xs, ys, zs, perm, Lt, Tb, pot, ax, ay, az, s, pos32, \
                                    Lt32)
    if (prec == 0) { FMM_P_SWITCH(p, C64) } else { FMM_P_SWITCH(p, C32) }
#undef C64
#undef C32
    count_launch();
    return 0;
}

int launch_p2p_leaf2(int prec, int depth, int64_t nleaf, const int* start, const double* xs, const double* ys,
                     const double* zs, const double* qs, const int* perm, double* pot, double* ax, double* ay,
                     double* az, cudaStream_t s) {
    if (nleaf <= 0) return 0;
    constexpr int W = 4;
    const unsigned g = (unsigned)((nleaf + W - 1) / W);
    if (prec == 0)
        k_p2p_leaf2<double, W><<<g, W * 32, 0, s>>>(depth, nleaf, start, xs, ys, zs, qs, perm, pot, ax, ay, az);
    else
        k_p2p_leaf2<float, W><<<g, W * 32, 0, s>>>(depth, nleaf, start, xs, ys, zs, qs, perm, pot, ax, ay, az);
    count_launch();
    return 0;
}

// ---------------------------------------------------------------------------
// FP32 P2P on positions relative to leaf centres: one warp per target leaf,
// its targets in blocks of up to 32 with 2, 3 or 4 targets per lane (each
// staged source is used that many times from registers), lane groups split
// the sources, one 16-byte shared load per source.  The
// target leaf itself comes first among the 27 neighbour leaves: only the
// chunks that hold its particles can contain the self pair or coincident
// pairs (r^2 == 0 exactly, dropped by a select as the direct sum skips
// them); particles of distinct leaves never coincide, so the other chunks
// run without the select.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void p2p32_pair(const float4 sv, const float4 p, float& f, float& x, float& y, float& z) {
    const float rx = sv.x - p.x, ry = sv.y - p.y, rz = sv.z - p.z;
    const float r2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
    const float ir = fmm_rsqrt(r2);
    const float qir = sv.w * ir, qir3 = qir * ir * ir;
    f += qir; x = fmaf(qir3, rx, x); y = fmaf(qir3, ry, y); z = fmaf(qir3, rz, z);
}
__device__ __forceinline__ void p2p32_pair_guarded(const float4 sv, const float4 p, float& f, float& x, float& y,
                                                   float& z) {
    const float rx = sv.x - p.x, ry = sv.y - p.y, rz = sv.z - p.z;
    const float r2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
    const float ir = r2 > 0.f ? fmm_rsqrt(r2) : 0.f;
    const float qir = sv.w * ir, qir3 = qir * ir * ir;
    f += qir; x = fmaf(qir3, rx, x); y = fmaf(qir3, ry, y); z = fmaf(qir3, rz, z);
}
// The near field of one block of up to 32 targets [t0, t0 + tn) of a leaf:
// NT targets per lane on lane groups of tp lanes (tp * NT >= tn), the
// 32 / tp groups splitting each staged chunk of 32 sources, the groups'
// sums added by shuffles.  The 27 neighbour leaves' sources are addressed
// through the warp's prefix sums (incl, excl, sbS, offsets ox..oz per lane);
// the chunks holding the target leaf's own particles ([0, nself)) take the
// r^2 == 0 select.  FUSED: each output written once as the far field sF
// (scaled by exact powers of two) plus the near field; otherwise the near
// field added to the outputs.
template <int NT, bool FUSED>
__device__ __forceinline__ void p2p32_block(int t0, int tn, int tp, int lane, float4* __restrict__ sP,
                                            const float4* __restrict__ sF, int total, int incl, int excl, int sbS,
                                            float ox, float oy, float oz, int nself, const float4* __restrict__ pos,
                                            const int* __restrict__ perm, float inv_hf, double* __restrict__ pot,
                                            double* __restrict__ ax, double* __restrict__ ay,
                                            double* __restrict__ az) {
    const int G = 32 / tp, grp = lane / tp, tl = lane % tp;
    float4 pt[NT];
    float f[NT], gx[NT], gy[NT], gz[NT];
#pragma unroll
    for (int j = 0; j < NT; ++j) {
        const int k = tl + tp * j;
        pt[j] = k < tn ? pos[t0 + k] : make_float4(0.f, 0.f, 0.f, 0.f);
        f[j] = gx[j] = gy[j] = gz[j] = 0.f;
    }
    for (int c0 = 0; c0 < total; c0 += 32) {
        {
            const int g = min(c0 + lane, total - 1);
            int i = 0;
#pragma unroll
            for (int step = 16; step >= 1; step >>= 1) {
                const int v = __shfl_sync(0xffffffffu, incl, i + step - 1);
                if (v <= g) i += step;
            }
            const int sbi = __shfl_sync(0xffffffffu, sbS, i), exi = __shfl_sync(0xffffffffu, excl, i);
            const float oxi = __shfl_sync(0xffffffffu, ox, i), oyi = __shfl_sync(0xffffffffu, oy, i),
                        ozi = __shfl_sync(0xffffffffu, oz, i);
            __syncwarp();
            if (c0 + lane < total) {
                const float4 v = pos[sbi + (g - exi)];
                sP[lane] = make_float4(v.x + oxi, v.y + oyi, v.z + ozi, v.w);
            }
            __syncwarp();
        }
        const int cnt = min(32, total - c0);
        if (c0 < nself) {
            for (int k = grp; k < cnt; k += G) {
                const float4 sv = sP[k];
#pragma unroll
                for (int j = 0; j < NT; ++j) p2p32_pair_guarded(sv, pt[j], f[j], gx[j], gy[j], gz[j]);
            }
        } else {
#pragma unroll 2
            for (int k = grp; k < cnt; k += G) {
                const float4 sv = sP[k];
#pragma unroll
                for (int j = 0; j < NT; ++j) p2p32_pair(sv, pt[j], f[j], gx[j], gy[j], gz[j]);
            }
        }
    }
#pragma unroll
    for (int j = 0; j < NT; ++j)
        for (int o = tp; o < 32; o <<= 1) {
            f[j] += __shfl_xor_sync(0xffffffffu, f[j], o); gx[j] += __shfl_xor_sync(0xffffffffu, gx[j], o);
            gy[j] += __shfl_xor_sync(0xffffffffu, gy[j], o); gz[j] += __shfl_xor_sync(0xffffffffu, gz[j], o);
        }
    if (grp == 0) {
#pragma unroll
        for (int j = 0; j < NT; ++j) {
            const int k = tl + tp * j;
            if (k >= tn) continue;
            const int o = perm[t0 + k];
            if constexpr (FUSED) {
                // the far field scaled as k_l2p_leaf2 scales it, plus the near
                // field in FP64 as the two-step form adds it
                const float4 F = sF[k];
                pot[o] = __dsub_rn((double)(-F.x * inv_hf), (double)f[j]);
                ax[o] = __dadd_rn((double)(F.y * inv_hf * inv_hf), (double)gx[j]);
                ay[o] = __dadd_rn((double)(F.z * inv_hf * inv_hf), (double)gy[j]);
                az[o] = __dadd_rn((double)(F.w * inv_hf * inv_hf), (double)gz[j]);
            } else {
                pot[o] -= (double)f[j]; ax[o] += (double)gx[j]; ay[o] += (double)gy[j]; az[o] += (double)gz[j];
            }
        }
    }
}

// the block schedule for tn targets: 2 per lane on 4 lanes up to 8 targets,
// on 8 lanes up to 16; 3 and 4 per lane on 8 lanes up to 24 and 32
template <bool FUSED>
__device__ __forceinline__ void p2p32_block_any(int t0, int tn, int lane, float4* sP, const float4* sF, int total,
                                                int incl, int excl, int sbS, float ox, float oy, float oz, int nself,
                                                const float4* pos, const int* perm, float inv_hf, double* pot,
                                                double* ax, double* ay, double* az) {
    if (tn <= 8)
        p2p32_block<2, FUSED>(t0, tn, 4, lane, sP, sF, total, incl, excl, sbS, ox, oy, oz, nself, pos, perm, inv_hf,
                              pot, ax, ay, az);
    else if (tn <= 16)
        p2p32_block<2, FUSED>(t0, tn, 8, lane, sP, sF, total, incl, excl, sbS, ox, oy, oz, nself, pos, perm, inv_hf,
                              pot, ax, ay, az);
    else if (tn <= 24)
        p2p32_block<3, FUSED>(t0, tn, 8, lane, sP, sF, total, incl, excl, sbS, ox, oy, oz, nself, pos, perm, inv_hf,
                              pot, ax, ay, az);
    else
        p2p32_block<4, FUSED>(t0, tn, 8, lane, sP, sF, total, incl, excl, sbS, ox, oy, oz, nself, pos, perm, inv_hf,
                              pot, ax, ay, az);
}

// sources of the 27 neighbour leaves of leaf c, one leaf per lane (lane 0:
// the leaf itself, so its particles come first): start, count and the
// offset of the leaf's centre; incl/excl: the warp's prefix sums of the counts
__device__ __forceinline__ void p2p32_neighbours(int depth, int64_t c, int lane, const int* __restrict__ start,
                                                 int& sbS, int& cntS, float& ox, float& oy, float& oz, int& incl,
                                                 int& excl, int& total, int& nself) {
    const int side = 1 << depth;
    const float h = 1.0f / (float)side;
    int ix, iy, iz;
    cell_coords(depth, c, ix, iy, iz);
    cntS = 0; sbS = 0; ox = oy = oz = 0.f;
    if (lane < 27) {
        const int d = lane == 0 ? 13 : lane <= 13 ? lane - 1 : lane;
        const int dx = d % 3 - 1, dy = (d / 3) % 3 - 1, dz = d / 9 - 1;
        const int jx = ix + dx, jy = iy + dy, jz = iz + dz;
        if (jx >= 0 && jy >= 0 && jz >= 0 && jx < side && jy < side && jz < side) {
            const int64_t S = cell_index(depth, jx, jy, jz);
            sbS = start[S];
            cntS = start[S + 1] - sbS;
            ox = dx * h; oy = dy * h; oz = dz * h;
        }
    }
    incl = cntS;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    total = __shfl_sync(0xffffffffu, incl, 31);
    excl = incl - cntS;
    nself = __shfl_sync(0xffffffffu, cntS, 0);
}

template <int WARPS>
__global__ void __launch_bounds__(WARPS * 32)
k_p2p32(int depth, int64_t nleaf, const int* __restrict__ start, const float4* __restrict__ pos,
        const int* __restrict__ perm, double* __restrict__ pot, double* __restrict__ ax, double* __restrict__ ay,
        double* __restrict__ az) {
    __shared__ float4 sP[WARPS][32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t c = (int64_t)blockIdx.x * WARPS + w;
    if (c >= nleaf) return;
    const int b = start[c], e = start[c + 1];
    if (b == e) return;
    int sbS, cntS, incl, excl, total, nself;
    float ox, oy, oz;
    p2p32_neighbours(depth, c, lane, start, sbS, cntS, ox, oy, oz, incl, excl, total, nself);
    for (int t0 = b; t0 < e; t0 += 32)
        p2p32_block_any<false>(t0, min(32, e - t0), lane, sP[w], nullptr, total, incl, excl, sbS, ox, oy, oz, nself,
                               pos, perm, 0.f, pot, ax, ay, az);
}

// ---------------------------------------------------------------------------
// Far and near field in one pass (FP32 form, uniform octree): one warp per
// target leaf evaluates the leaf's local expansion at its particles (the
// arithmetic of k_l2p_leaf2, one target per lane), then the near field of
// k_p2p32 (the same block schedule, p2p32_block), and writes each particle's
// potential and acceleration once, in
// the operation order of k_l2p_leaf2 followed by k_p2p32 (explicitly
// rounded, so the result is that sequence's), without the separate write
// and read-modify-write of the caller-order outputs.
// ---------------------------------------------------------------------------
// far field at one point (scaled offset r from the leaf centre): the
// arithmetic of k_l2p_leaf2; not inlined, so that the expansion is read
// from shared memory per point instead of being held in registers
template <int P>
__device__ __noinline__ float4 l2p_point32(const float* Ln, float rx, float ry, float rz) {
    float fx[P + 1], fy[P + 1], fz[P + 1];
    fx[0] = fy[0] = fz[0] = 1.f;
#pragma unroll
    for (int q = 1; q <= P; ++q) {
        fx[q] = fx[q - 1] * rx * float(1.0 / q);
        fy[q] = fy[q - 1] * ry * float(1.0 / q);
        fz[q] = fz[q - 1] * rz * float(1.0 / q);
    }
    float ph = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
    l2p_all<P, float, 0>(Ln, fx, fy, fz, ph, gx, gy, gz);
    return make_float4(ph, gx, gy, gz);
}

// at most 64 registers (8 blocks of 4 warps per SM): with more, the 3- and
// 4-target blocks cost the pass more in occupancy than they save
template <int P, int WARPS, typename LT>   // LT: the type of the stored locals
__global__ void __launch_bounds__(WARPS * 32, 32 / WARPS)
k_l2p_p2p32(int basis, int depth, int64_t nleaf, const int* __restrict__ start, const float4* __restrict__ pos,
            const int* __restrict__ perm, const LT* __restrict__ Lt, const float* __restrict__ expand,
            DevOffsets off, double* __restrict__ pot, double* __restrict__ ax, double* __restrict__ ay,
            double* __restrict__ az) {
    constexpr int NS = (P + 1) * (P + 2) * (P + 3) / 6;
    constexpr int NN = nested_col_off<P, float>(P + 1, 0);
    __shared__ float sA[WARPS][NS];
    __shared__ __align__(16) float sN[WARPS][NN];
    __shared__ float4 sF[WARPS][32];   // far field of a block of targets (potential, gradient; scaled units)
    __shared__ float4 sP[WARPS][32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t c = (int64_t)blockIdx.x * WARPS + w;
    if (c >= nleaf) return;
    const int b = start[c], e = start[c + 1];
    if (b == e) return;
    // the leaf's local expansion in the nested FP32 layout of k_l2p_leaf2
    if (basis) {
        constexpr int NT = (P + 1) * (P + 1);
        for (int t = lane; t < NT; t += 32) sA[w][t] = float(Lt[(int64_t)t * nleaf + c]);
        __syncwarp();
        for (int s = lane; s < NS; s += 32) {
            const int nx = c_sym_idx[s][0], ny = c_sym_idx[s][1], nz = c_sym_idx[s][2];
            const int j = nx + ny + nz;
            const int row = (j - nx) * (j - nx + 1) / 2 + nz;
            const float* E = expand + off.expand[j] + row * (2 * j + 1);
            float v = 0.f;
            for (int t = 0; t < 2 * j + 1; ++t) v += E[t] * sA[w][j * j + t];
            sN[w][nested_col_off<P, float>(nx, ny) + nz] = v;
        }
    } else {
        for (int s = lane; s < NS; s += 32)
            sN[w][nested_col_off<P, float>(c_sym_idx[s][0], c_sym_idx[s][1]) + c_sym_idx[s][2]] =
                float(Lt[(int64_t)s * nleaf + c]);
    }
    __syncwarp();
    const float inv_hf = (float)(1 << depth);   // exact
    const float* Ln = sN[w];
    int sbS, cntS, incl, excl, total, nself;
    float ox, oy, oz;
    p2p32_neighbours(depth, c, lane, start, sbS, cntS, ox, oy, oz, incl, excl, total, nself);
    for (int t0 = b; t0 < e; t0 += 32) {
        const int tn = min(32, e - t0);
        // far field of the block's targets, one per lane
        if (lane < tn) {
            const float4 v = pos[t0 + lane];
            sF[w][lane] = l2p_point32<P>(Ln, v.x * inv_hf, v.y * inv_hf, v.z * inv_hf);
        }
        __syncwarp();
        p2p32_block_any<true>(t0, tn, lane, sP[w], sF[w], total, incl, excl, sbS, ox, oy, oz, nself, pos, perm,
                              inv_hf, pot, ax, ay, az);
        __syncwarp();
    }
}

template <int P>
static void l2p_p2p32_p(int basis, int depth, int64_t nleaf, const int* start, const float4* pos, const int* perm,
                        const double* Lt, const DevTables& Tb, double* pot, double* ax, double* ay, double* az,
                        cudaStream_t s, const float* Lt32) {
    constexpr int W = 4;
    const unsigned g = (unsigned)((nleaf + W - 1) / W);
    if (Lt32)
        k_l2p_p2p32<P, W, float><<<g, W * 32, 0, s>>>(basis, depth, nleaf, start, pos, perm, Lt32, Tb.expand32,
                                                       Tb.offsets(), pot, ax, ay, az);
    else
        k_l2p_p2p32<P, W, double><<<g, W * 32, 0, s>>>(basis, depth, nleaf, start, pos, perm, Lt, Tb.expand32,
                                                        Tb.offsets(), pot, ax, ay, az);
}

int launch_l2p_p2p32(int p, int basis, int depth, int64_t nleaf, const int* start, const float4* pos, const int* perm,
                     const double* Lt, const DevTables& Tb, double* pot, double* ax, double* ay, double* az,
                     cudaStream_t s, const float* Lt32) {
    if (nleaf <= 0) return 0;
#define CF(P) l2p_p2p32_p<P>(basis, depth, nleaf, start, pos, perm, Lt, Tb, pot, ax, ay, az, s, Lt32)
    FMM_P_SWITCH(p, CF)
#undef CF
    count_launch();
    return 0;
}

int launch_p2p32(int depth, int64_t nleaf, const int* start, const float4* pos, const int* perm, double* pot,
                 double* ax, double* ay, double* az, cudaStream_t s) {
    if (nleaf <= 0) return 0;
    constexpr int W = 4;
    k_p2p32<W><<<(unsigned)((nleaf + W - 1) / W), W * 32, 0, s>>>(depth, nleaf, start, pos, perm, pot, ax, ay, az);
    count_launch();
    return 0;
}

}  // namespace fmm
