// P2M kernel of the uniform-octree FMM and of fmm_op_p2m.
#include "fmm_internal.h"

namespace fmm {

// ---------------------------------------------------------------------------
// P2M (Eq. P2M, Sec. 2.1): A_m = sum_a q_a (-(x_a - z)/h)^m for all |m| <= p,
// then  mode 0: SYM -> A, TRACELESS -> Mbar = D[A] (independent comps),
//       mode 1: TRACELESS -> M^r (reduced representative).
// One warp per cell.  centre == nullptr: uniform-octree leaf centres of
// level `depth` (cell numbering of cell_index).
// ---------------------------------------------------------------------------
template <int WARPS>
__global__ void __launch_bounds__(WARPS * 32)
k_p2m(int p, int basis, int mode, int64_t ncell, const int64_t* __restrict__ start64,
      const int* __restrict__ start32, const double* __restrict__ x, const double* __restrict__ y,
      const double* __restrict__ z, const double* __restrict__ q, const double* __restrict__ centre,
      int depth, double inv_h, double* __restrict__ M, int64_t ldm, const double* __restrict__ detr,
      const double* __restrict__ reduce, DevOffsets off) {
    __shared__ double sA[WARPS][FMM_NS_MAX];
    __shared__ double sP[WARPS][3][FMM_PMAX + 1];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t c = (int64_t)blockIdx.x * WARPS + w;
    if (c >= ncell) return;
    const int ns = ns_of(p);
    double cx, cy, cz;
    if (centre) {
        cx = centre[c]; cy = centre[ncell + c]; cz = centre[2 * ncell + c];
    } else {
        int ix, iy, iz;
        cell_coords(depth, c, ix, iy, iz);
        const double h = 1.0 / inv_h;
        cx = (ix + 0.5) * h; cy = (iy + 0.5) * h; cz = (iz + 0.5) * h;
    }
    const int64_t b = start64 ? start64[c] : start32[c];
    const int64_t e = start64 ? start64[c + 1] : start32[c + 1];
    constexpr int PER = (FMM_NS_MAX + 31) / 32;
    double acc[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) acc[k] = 0.0;
    for (int64_t a = b; a < e; ++a) {
        if (lane < 3) {
            const double r = lane == 0 ? (cx - x[a]) : lane == 1 ? (cy - y[a]) : (cz - z[a]);
            const double rs = r * inv_h;  // (-r_a / h)
            double v = 1.0;
            sP[w][lane][0] = 1.0;
            for (int k = 1; k <= p; ++k) { v *= rs; sP[w][lane][k] = v; }
        }
        __syncwarp();
        const double qa = q[a];
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int s = lane + 32 * k;
            if (s < ns)
                acc[k] += qa * sP[w][0][c_sym_idx[s][0]] * sP[w][1][c_sym_idx[s][1]] * sP[w][2][c_sym_idx[s][2]];
        }
        __syncwarp();
    }
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int s = lane + 32 * k;
        if (s < ns) sA[w][s] = acc[k];
    }
    __syncwarp();
    if (!basis) {
        for (int s = lane; s < ns; s += 32) M[(int64_t)s * ldm + c] = sA[w][s];
        return;
    }
    const int nt = nt_of(p);
    for (int t = lane; t < nt; t += 32) {
        const int nx = c_tl_idx[t][0], ny = c_tl_idx[t][1], nz = c_tl_idx[t][2];
        const int j = nx + ny + nz;
        const double* As = &sA[w][ns_of(j - 1)];
        const int cols = (j + 1) * (j + 2) / 2;
        const double* R;
        if (mode == 0) {
            const int row = (j - nx) * (j - nx + 1) / 2 + nz;
            R = detr + off.detr[j] + row * cols;
        } else {
            R = reduce + off.reduce[j] + (t - j * j) * cols;
        }
        double v = 0.0;
        for (int s = 0; s < cols; ++s) v += R[s] * As[s];
        M[(int64_t)t * ldm + c] = v;
    }
}

int launch_p2m(int p, int basis, int mode, int64_t ncell, const int64_t* start64, const int* start32,
               const double* x, const double* y, const double* z, const double* q, const double* centre,
               int depth, double inv_h, double* M, int64_t ldm, const DevTables& T, cudaStream_t s) {
    if (ncell <= 0) return 0;
    constexpr int W = 4;
    k_p2m<W><<<(unsigned)((ncell + W - 1) / W), W * 32, 0, s>>>(p, basis, mode, ncell, start64, start32, x, y,
                                                                 z, q, centre, depth, inv_h, M, ldm, T.detr,
                                                                 T.reduce, T.offsets());
    count_launch();
    return 0;
}

}  // namespace fmm
