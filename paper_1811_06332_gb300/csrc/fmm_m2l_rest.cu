// The part of Eq. M2L that the swapped tensor-core kernel leaves to the CUDA
// cores when it runs the first K-part only (kernel shape 3; BF16 form,
// traceless basis, p = 6..8): the tables it reads.
//
// In the regrouped form L_n += sum_m Kt_o(n, m) M_m over the 189 offsets o of
// a target's interaction list, with Kt_o(n, m) = D_{n+m}(-o)/m! nonzero only
// for |n| + |m| <= p.  The tensor cores contract the multipole columns
// m = 0..47 (the first K-part of 48).  The columns m >= 48 (ranks >= 6) reach
// only the local rows of rank a <= p - 6, (p - 5)^2 of them, and a row of
// rank a only its (p - a + 1)^2 - 48 columns above 47: 86 products per pair
// at p = 8 out of 1365.  As 128-row tensor-core tiles they would cost as much
// as the first K-part; k_m2l_rest does them as FP32 FMAs after the
// tensor-core kernel and adds them to L, reading
//   Mrest  the columns >= 48 of a level's multipoles, cell-major FP32, one
//          16-byte aligned record of rest_cstride(p) floats per cell
//          (k_rest_pack, once per level and step, from the plan's FP32 copy
//          of the multipoles when it has one), and
//   Krest  per offset, the rows of rank <= p - 6 one after the other, each
//          with its entries of columns >= 48 padded to a multiple of 4
//          (k_build_krest, once per plan).
#include "fmm_internal.h"
#include "fmm_device.cuh"
#include "fmm_m2l_rest.cuh"

namespace fmm {

// One block of 64 threads per 8 x 16 target cells of one parity class and
// plane, two targets per thread (x, y) and (x, y + 8); for each source class
// and plane shift the block copies (cp.async) the 10 x 18 source cells'
// records and the nine (dx, dy) offsets' entries to shared memory, then every
// thread accumulates its targets' rows over the offsets that are not near
// neighbours (packed FP32x2 FMAs over column pairs, each entry load serving
// both targets), and finally adds them to the locals the tensor-core kernel
// wrote.  With nsplit > 1 (small levels, where one block per tile leaves
// most schedulers idle) the eight source classes are split into nsplit
// consecutive groups, one block per tile and group; each block writes its
// sums to part[group] and k_rest_sum adds the groups in order.
template <int P>
__global__ void __launch_bounds__(64)
k_m2l_rest(int l, int nsplit, const float4* __restrict__ Mrest, const float4* __restrict__ Krest,
           double* __restrict__ Lt, int64_t ncell, float* __restrict__ Lt32, float* __restrict__ part) {
    constexpr int NR = rs_rows(P);
    constexpr int CS = rs_cstride(P);
    constexpr int KS = rs_kstride(P);
    constexpr int CS4 = CS / 4, KS4 = KS / 4;
    constexpr int ROW4 = RS_RX * CS4;   // 16-byte chunks of one region row (contiguous in Mrest)
    __shared__ __align__(16) float sM[RS_RX * RS_RY * CS];
    __shared__ __align__(16) float sK[9 * KS];
    const int hs = 1 << (l - 1);
    const int64_t h3 = (int64_t)hs * hs * hs;
    const int ntx = hs / RS_TX, nty = hs / RS_TY;
    const int64_t tpc = (int64_t)ntx * nty * hs;
    const int grp = (int)(blockIdx.x / (8 * tpc));   // source-class group
    const int64_t bt = blockIdx.x % (8 * tpc);
    const int cls = (int)(bt / tpc);
    const int64_t t = bt % tpc;
    const int sc0 = grp * (8 / nsplit), sc1 = sc0 + 8 / nsplit;
    const int ti = (int)(t % ntx), tj = (int)((t / ntx) % nty), tk = (int)(t / ((int64_t)ntx * nty));
    const int cx = cls & 1, cy = (cls >> 1) & 1, cz = cls >> 2;
    const int x = threadIdx.x & 7, y = threadIdx.x >> 3;   // targets (x, y) and (x, y + 8)
    uint64_t aa[NR], ab[NR];   // per row: the sums of its even and odd columns (two floats)
#pragma unroll
    for (int r = 0; r < NR; ++r) aa[r] = ab[r] = 0ull;
#pragma unroll 1
    for (int sc = sc0; sc < sc1; ++sc) {
        const int sx = sc & 1, sy = (sc >> 1) & 1, sz = sc >> 2;
#pragma unroll 1
        for (int dz = -1; dz <= 1; ++dz) {
            const int gk = tk + dz;
            if (gk < 0 || gk >= hs) continue;   // no sources in that plane
            const int oz = 2 * dz + sz - cz;
            __syncthreads();   // the previous stage is read
            // source rows gj = 16 tj - 1 .. 16 tj + 16 of cells gi = 8 ti - 1 .. 8 ti + 8, plane gk, class sc
#pragma unroll 2
            for (int row = 0; row < RS_RY; ++row) {
                const int gj = RS_TY * tj + row - 1;
                const bool rok = gj >= 0 && gj < hs;
                const int64_t rbase = (sc * h3 + ((int64_t)gk * hs + gj) * hs + RS_TX * ti - 1) * CS4;
                for (int e = threadIdx.x; e < ROW4; e += 64) {
                    const int gi = RS_TX * ti - 1 + e / CS4;
                    const bool ok = rok && gi >= 0 && gi < hs;
                    rs_cp16(sM + 4 * (row * ROW4 + e), ok ? Mrest + rbase + e : Mrest, ok);
                }
            }
            for (int e = threadIdx.x; e < 9 * KS4; e += 64) {
                const int o = e / KS4, k4 = e % KS4;
                const int ox = 2 * (o % 3 - 1) + sx - cx, oy = 2 * (o / 3 - 1) + sy - cy;
                const int ridx = (3 - oz) * 49 + (3 - oy) * 7 + (3 - ox);   // the matrix of -o
                rs_cp16(sK + 4 * e, Krest + (int64_t)ridx * KS4 + k4, true);
            }
            asm volatile("cp.async.wait_all;" ::: "memory");
            __syncthreads();
#pragma unroll 1
            for (int o = 0; o < 9; ++o) {
                const int dx = o % 3 - 1, dy = o / 3 - 1;
                const int ox = 2 * dx + sx - cx, oy = 2 * dy + sy - cy;
                if (ox >= -1 && ox <= 1 && oy >= -1 && oy <= 1 && oz >= -1 && oz <= 1) continue;   // near field
                const float* sa = sM + ((y + dy + 1) * RS_RX + (x + dx + 1)) * CS;
                const float* sb = sa + 8 * RS_RX * CS;
                uint64_t ma[CS / 2], mb[CS / 2];
#pragma unroll
                for (int c = 0; c < CS; c += 4) {
                    const ulonglong2 va = *(const ulonglong2*)(sa + c), vb = *(const ulonglong2*)(sb + c);
                    ma[c / 2] = va.x; ma[c / 2 + 1] = va.y;
                    mb[c / 2] = vb.x; mb[c / 2 + 1] = vb.y;
                }
                rs_rank_rows2<P, 0, 0, 0>(sK + o * KS, ma, mb, aa, ab);
            }
        }
    }
    const int64_t tg = cls * h3 + ((int64_t)tk * hs + RS_TY * tj + y) * hs + RS_TX * ti + x;
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        const float va = __uint_as_float((uint32_t)aa[r]) + __uint_as_float((uint32_t)(aa[r] >> 32));
        const float vb = __uint_as_float((uint32_t)ab[r]) + __uint_as_float((uint32_t)(ab[r] >> 32));
        if (nsplit > 1) {
            float* pr = part + ((int64_t)grp * NR + r) * ncell;
            pr[tg] = va;
            pr[tg + 8 * hs] = vb;
        } else if (Lt32) {
            Lt32[(int64_t)r * ncell + tg] += va;
            Lt32[(int64_t)r * ncell + tg + 8 * hs] += vb;
        } else {
            Lt[(int64_t)r * ncell + tg] += (double)va;
            Lt[(int64_t)r * ncell + tg + 8 * hs] += (double)vb;
        }
    }
}

// L[r][cell] += the nsplit groups' sums part[g][r][cell], added in group
// order (rows r < nr of a level's coefficient-major locals)
__global__ void __launch_bounds__(256) k_rest_sum(int64_t nel, int nsplit, const float* __restrict__ part,
                                                  double* __restrict__ Lt, float* __restrict__ Lt32) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nel) return;
    float v = part[e];
    for (int g = 1; g < nsplit; ++g) v += part[(int64_t)g * nel + e];
    if (Lt32)
        Lt32[e] += v;
    else
        Lt[e] += (double)v;
}

// Mrest of level l from the FP64 coefficient-major multipoles M: a block
// transposes 64 cells through shared memory
template <int P>
__global__ void __launch_bounds__(256) k_rest_pack(int64_t ncell, const double* __restrict__ M, float* __restrict__ Mrest,
                                                   const float* __restrict__ M32) {
    constexpr int NCOL = (P + 1) * (P + 1) - RS_K0;
    constexpr int CS = rs_cstride(P);
    __shared__ float tile[64][CS + 1];
    const int64_t c0 = (int64_t)blockIdx.x * 64;
    const int cl = threadIdx.x & 63;
    for (int c = threadIdx.x >> 6; c < NCOL; c += 4)
        tile[cl][c] = c0 + cl >= ncell ? 0.f
                      : M32 ? M32[(int64_t)(RS_K0 + c) * ncell + c0 + cl]
                            : (float)M[(int64_t)(RS_K0 + c) * ncell + c0 + cl];
    __syncthreads();
    for (int e = threadIdx.x; e < 64 * CS; e += 256) {
        const int cell = e / CS, c = e % CS;
        if (c0 + cell < ncell) Mrest[c0 * CS + e] = c < NCOL ? tile[cell][c] : 0.f;
    }
}

// Krest[r][...]: per offset r (343), the rows of rank <= p - 6 one after the
// other, each with its columns m >= 48 (|n| + |m| <= p) padded to a multiple
// of 4: Kt_r(n, m) = D_{n+m}(r)/m! in FP32
template <int P>
__global__ void k_build_krest(const double* __restrict__ Dtab, float* __restrict__ Krest) {
    constexpr int NR = rs_rows(P), KS = rs_kstride(P);
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 343 * KS) return;
    const int ridx = t / KS, k = t % KS;
    int r = 0;
    while (r + 1 < NR && k >= rs_roff(P, r + 1)) ++r;
    const int c = k - rs_roff(P, r);
    float v = 0.f;
    if (c < rs_cols(P, r)) {
        const int m = RS_K0 + c;
        const int nx = c_tl_idx[r][0], ny = c_tl_idx[r][1], nz = c_tl_idx[r][2];
        const int mx = c_tl_idx[m][0], my = c_tl_idx[m][1], mz = c_tl_idx[m][2];
        v = (float)(Dtab[(int64_t)ridx * ns_of(P) + pos_sym(nx + mx, ny + my, nz + mz)] * c_invfact[mx] *
                    c_invfact[my] * c_invfact[mz]);
    }
    Krest[t] = v;
}

int rest_rows(int p) { return p >= 6 && p <= 8 ? rs_rows(p) : 0; }
int rest_kstride(int p) { return rest_rows(p) ? rs_kstride(p) : 0; }
int rest_cstride(int p) { return rest_rows(p) ? rs_cstride(p) : 0; }

#define RS_P_SWITCH(p, F) (p == 6 ? F(6) : p == 7 ? F(7) : F(8))

int rest_nsplit(int l) {
    const int64_t hs = (int64_t)1 << (l - 1);
    return 8 * (hs / RS_TX) * (hs / RS_TY) * hs < 1024 ? 4 : 1;
}

int launch_m2l_rest(int p, int l, const float* Mrest, const float* Krest, double* Lt, cudaStream_t s, float* Lt32,
                    float* part, int64_t part_cap) {
    const int hs = 1 << (l - 1);
    if (hs < RS_TY || rest_rows(p) == 0) return -1;
    const int64_t ncell = (int64_t)8 * hs * hs * hs;
    const int nr = rest_rows(p);
    int nsplit = rest_nsplit(l);
    if (!part || part_cap < (int64_t)nsplit * nr * ncell) nsplit = 1;
    const unsigned g = (unsigned)(8 * (int64_t)(hs / RS_TX) * (hs / RS_TY) * hs * nsplit);
    const float4* m4 = (const float4*)Mrest;
    const float4* k4 = (const float4*)Krest;
#define RS_L(P) (k_m2l_rest<P><<<g, 64, 0, s>>>(l, nsplit, m4, k4, Lt, ncell, Lt32, part), 0)
    RS_P_SWITCH(p, RS_L);
#undef RS_L
    count_launch();
    if (nsplit > 1) {
        const int64_t nel = (int64_t)nr * ncell;
        k_rest_sum<<<(unsigned)((nel + 255) / 256), 256, 0, s>>>(nel, nsplit, part, Lt, Lt32);
        count_launch();
    }
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

int build_krest(int p, const double* Dtab, float* Krest, cudaStream_t s) {
    if (!rest_rows(p)) return -1;
    const int n = 343 * rs_kstride(p);
#define RS_B(P) (k_build_krest<P><<<(n + 255) / 256, 256, 0, s>>>(Dtab, Krest), 0)
    RS_P_SWITCH(p, RS_B);
#undef RS_B
    count_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

int launch_rest_pack(int p, int l, const double* M, float* Mrest, cudaStream_t s, const float* M32) {
    if (!rest_rows(p)) return -1;
    const int64_t ncell = (int64_t)8 << (3 * (l - 1));
    const unsigned g = (unsigned)((ncell + 63) / 64);
#define RS_K(P) (k_rest_pack<P><<<g, 256, 0, s>>>(ncell, M, Mrest, M32), 0)
    RS_P_SWITCH(p, RS_K);
#undef RS_K
    count_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

}  // namespace fmm
