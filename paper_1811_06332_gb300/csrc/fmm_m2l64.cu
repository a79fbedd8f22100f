// M2L over uniform interaction lists, plain FP64 form.
#include "fmm_internal.h"

namespace fmm {

// ---------------------------------------------------------------------------
// M2L, plain FP64 form, over the uniform interaction lists of one level:
//   Lt_n(target) = sum_sources sum_m Mt_m/m! D_{n+m}(target - source)
// with D from a per-level-independent table over the 7^3 integer offsets
// (cell units), computed once in FP64 by the D-tensor recurrence.
// One warp per target cell; the source multipole is staged in shared memory
// pre-divided by m!, lanes stride the output components.
// ---------------------------------------------------------------------------
template <int WARPS>
__global__ void __launch_bounds__(WARPS * 32)
k_m2l_fp64_level(int p, int basis, int l, const double* __restrict__ Dtab, const double* __restrict__ Mt,
                 double* __restrict__ Lt, int64_t ncell) {
    __shared__ double sX[WARPS][FMM_NS_MAX];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t T = (int64_t)blockIdx.x * WARPS + w;
    if (T >= ncell) return;
    const int nc = ncoef_of(p, basis), ns = ns_of(p);
    const int side = 1 << l;
    int ix, iy, iz;
    cell_coords(l, T, ix, iy, iz);
    constexpr int PER = (FMM_NS_MAX + 31) / 32;
    double acc[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) acc[k] = 0.0;
    const int px = ix >> 1, py = iy >> 1, pz = iz >> 1;
#pragma unroll 1
    for (int o = 0; o < 216; ++o) {
                const int jx = 2 * px - 2 + o % 6, jy = 2 * py - 2 + (o / 6) % 6, jz = 2 * pz - 2 + o / 36;
                if (jx < 0 || jy < 0 || jz < 0 || jx >= side || jy >= side || jz >= side) continue;
                const int rx = ix - jx, ry = iy - jy, rz = iz - jz;
                if (rx >= -1 && rx <= 1 && ry >= -1 && ry <= 1 && rz >= -1 && rz <= 1) continue;
                const int64_t S = cell_index(l, jx, jy, jz);
                const double* D = Dtab + (int64_t)((rz + 3) * 49 + (ry + 3) * 7 + (rx + 3)) * ns;
                __syncwarp();
                for (int m = lane; m < nc; m += 32) {
                    const int mx = basis ? c_tl_idx[m][0] : c_sym_idx[m][0];
                    const int my = basis ? c_tl_idx[m][1] : c_sym_idx[m][1];
                    const int mz = basis ? c_tl_idx[m][2] : c_sym_idx[m][2];
                    sX[w][m] = Mt[(int64_t)m * ncell + S] * c_invfact[mx] * c_invfact[my] * c_invfact[mz];
                }
                __syncwarp();
#pragma unroll
                for (int k = 0; k < PER; ++k) {
                    const int r = lane + 32 * k;
                    if (r < nc) {
                        const int nx = basis ? c_tl_idx[r][0] : c_sym_idx[r][0];
                        const int ny = basis ? c_tl_idx[r][1] : c_sym_idx[r][1];
                        const int nz = basis ? c_tl_idx[r][2] : c_sym_idx[r][2];
                        const int mend = basis ? nt_of(p - nx - ny - nz) : ns_of(p - nx - ny - nz);
                        double v = acc[k];
                        for (int m = 0; m < mend; ++m) {
                            const int mx = basis ? c_tl_idx[m][0] : c_sym_idx[m][0];
                            const int my = basis ? c_tl_idx[m][1] : c_sym_idx[m][1];
                            const int mz = basis ? c_tl_idx[m][2] : c_sym_idx[m][2];
                            v += sX[w][m] * __ldg(&D[pos_sym(nx + mx, ny + my, nz + mz)]);
                        }
                        acc[k] = v;
                    }
                }
    }
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int r = lane + 32 * k;
        if (r < nc) Lt[(int64_t)r * ncell + T] = acc[k];
    }
}

int launch_m2l_fp64_level(int p, int basis, int l, const double* Dtab, const double* Mt, double* Lt,
                          int64_t ncell, cudaStream_t s) {
    constexpr int WARPS = 4;
    k_m2l_fp64_level<WARPS><<<(unsigned)((ncell + WARPS - 1) / WARPS), WARPS * 32, 0, s>>>(p, basis, l, Dtab, Mt,
                                                                                         Lt, ncell);
    count_launch();
    return 0;
}

}  // namespace fmm
