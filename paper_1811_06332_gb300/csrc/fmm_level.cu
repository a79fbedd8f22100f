// Uniform-octree M2M / L2L level kernels (scaled units, fixed shifts).
#include "fmm_internal.h"

namespace fmm {

// ---------------------------------------------------------------------------
// Uniform-octree level kernels (scaled units, fixed shifts).
//
// M2M: Mt(parent) = sum_c W_c Mt(child c), rows of W_c use only columns of
//      rank <= rank(row) (the shift never lowers a rank).
// L2L: Lt(child c) += V_c Lt(parent), rows use columns of rank >= rank(row).
// One warp per parent; lanes stride the output rows.
// ---------------------------------------------------------------------------
template <int WARPS>
__global__ void __launch_bounds__(WARPS * 32)
k_m2m_level(int p, int basis, int l, const double* __restrict__ W, const double* __restrict__ Mch,
            int64_t nch, double* __restrict__ Mpa, int64_t npa) {
    __shared__ double sX[WARPS][FMM_NS_MAX];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t P = (int64_t)blockIdx.x * WARPS + w;
    if (P >= npa) return;
    const int nc = ncoef_of(p, basis);
    int ix, iy, iz;
    cell_coords(l, P, ix, iy, iz);
    const int64_t lin = lin_index(l, ix, iy, iz);
    const int64_t blk = (int64_t)1 << (3 * l);
    constexpr int PER = (FMM_NS_MAX + 31) / 32;
    double acc[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) acc[k] = 0.0;
    for (int c = 0; c < 8; ++c) {
        const int64_t ch = c * blk + lin;
        __syncwarp();
        for (int j = lane; j < nc; j += 32) sX[w][j] = Mch[(int64_t)j * nch + ch];
        __syncwarp();
        const double* Wc = W + (int64_t)c * nc * nc;
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int r = lane + 32 * k;
            if (r < nc) {
                const int rk = basis ? (c_tl_idx[r][0] + c_tl_idx[r][1] + c_tl_idx[r][2])
                                     : (c_sym_idx[r][0] + c_sym_idx[r][1] + c_sym_idx[r][2]);
                const int jend = basis ? nt_of(rk) : ns_of(rk);
                const double* Wr = Wc + (int64_t)r * nc;
                double v = acc[k];
                for (int j = 0; j < jend; ++j) v += Wr[j] * sX[w][j];
                acc[k] = v;
            }
        }
    }
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int r = lane + 32 * k;
        if (r < nc) Mpa[(int64_t)r * npa + P] = acc[k];
    }
}

template <int WARPS>
__global__ void __launch_bounds__(WARPS * 32)
k_l2l_level(int p, int basis, int l, const double* __restrict__ V, const double* __restrict__ Lpa, int64_t npa,
            double* __restrict__ Lch, int64_t nch) {
    __shared__ double sX[WARPS][FMM_NS_MAX];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t P = (int64_t)blockIdx.x * WARPS + w;
    if (P >= npa) return;
    const int nc = ncoef_of(p, basis);
    int ix, iy, iz;
    cell_coords(l, P, ix, iy, iz);
    const int64_t lin = lin_index(l, ix, iy, iz);
    const int64_t blk = (int64_t)1 << (3 * l);
    for (int j = lane; j < nc; j += 32) sX[w][j] = Lpa[(int64_t)j * npa + P];
    __syncwarp();
    for (int c = 0; c < 8; ++c) {
        const int64_t ch = c * blk + lin;
        const double* Vc = V + (int64_t)c * nc * nc;
        for (int r = lane; r < nc; r += 32) {
            const int rk = basis ? (c_tl_idx[r][0] + c_tl_idx[r][1] + c_tl_idx[r][2])
                                 : (c_sym_idx[r][0] + c_sym_idx[r][1] + c_sym_idx[r][2]);
            const int j0 = basis ? rk * rk : ns_of(rk - 1);
            const double* Vr = Vc + (int64_t)r * nc;
            double v = 0.0;
            for (int j = j0; j < nc; ++j) v += Vr[j] * sX[w][j];
            Lch[(int64_t)r * nch + ch] += v;
        }
    }
}

int launch_m2m_level(int p, int basis, int l, const double* W, const double* Mch, int64_t nch, double* Mpa,
                     int64_t npa, cudaStream_t s) {
    constexpr int WARPS = 4;
    k_m2m_level<WARPS><<<(unsigned)((npa + WARPS - 1) / WARPS), WARPS * 32, 0, s>>>(p, basis, l, W, Mch, nch,
                                                                                    Mpa, npa);
    count_launch();
    return 0;
}

int launch_l2l_level(int p, int basis, int l, const double* V, const double* Lpa, int64_t npa, double* Lch,
                     int64_t nch, cudaStream_t s) {
    constexpr int WARPS = 4;
    k_l2l_level<WARPS><<<(unsigned)((npa + WARPS - 1) / WARPS), WARPS * 32, 0, s>>>(p, basis, l, V, Lpa, npa,
                                                                                    Lch, nch);
    count_launch();
    return 0;
}

}  // namespace fmm
