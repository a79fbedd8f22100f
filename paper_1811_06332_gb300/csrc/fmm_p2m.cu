// P2M kernel of the uniform-octree FMM and of fmm_op_p2m.
#include "fmm_internal.h"

namespace fmm {

// ---------------------------------------------------------------------------
// P2M (Eq. P2M, Sec. 2.1): A_m = sum_a q_a (-(x_a - z)/h)^m for all |m| <= p,
// plus, with point dipoles (px != nullptr; App. B, "Dipoles"), the pure
// dipole M_{e_i} = -p_i of each particle shifted by M2M from x_a to z:
//     A_m += -sum_i m_i (p_i/h) (-(x_a - z)/h)^(m - e_i),
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
      const double* __restrict__ reduce, DevOffsets off, const double* __restrict__ px,
      const double* __restrict__ py, const double* __restrict__ pz) {
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
        if (px) {
            const double dx = px[a] * inv_h, dy = py[a] * inv_h, dz = pz[a] * inv_h;
#pragma unroll
            for (int k = 0; k < PER; ++k) {
                const int s = lane + 32 * k;
                if (s < ns) {
                    const int mx = c_sym_idx[s][0], my = c_sym_idx[s][1], mz = c_sym_idx[s][2];
                    double v = 0.0;
                    if (mx) v += mx * dx * sP[w][0][mx - 1] * sP[w][1][my] * sP[w][2][mz];
                    if (my) v += my * dy * sP[w][0][mx] * sP[w][1][my - 1] * sP[w][2][mz];
                    if (mz) v += mz * dz * sP[w][0][mx] * sP[w][1][my] * sP[w][2][mz - 1];
                    acc[k] -= v;
                }
            }
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
               int depth, double inv_h, double* M, int64_t ldm, const DevTables& T, cudaStream_t s,
               const double* px, const double* py, const double* pz) {
    if (ncell <= 0) return 0;
    constexpr int W = 4;
    k_p2m<W><<<(unsigned)((ncell + W - 1) / W), W * 32, 0, s>>>(p, basis, mode, ncell, start64, start32, x, y,
                                                                 z, q, centre, depth, inv_h, M, ldm, T.detr,
                                                                 T.reduce, T.offsets(), px, py, pz);
    count_launch();
    return 0;
}

// ---------------------------------------------------------------------------
// Point dipoles in the near field: the field of the dipole sources of the
// adjacent leaves (self excluded), ADDED into caller order via perm:
//   Phi += p_j . d / |d|^3,  grad Phi += p_j / |d|^3 - 3 (p_j . d) d / |d|^5,
//   d = x_i - x_j;  pot -= Phi, acc += grad Phi  (the library's sign).
// One warp per target leaf, lanes over its particles; FP64.
// ---------------------------------------------------------------------------
template <int WARPS>
__global__ void __launch_bounds__(WARPS * 32)
k_p2p_dipole(int depth, int64_t nleaf, const int* __restrict__ start, const double* __restrict__ xs,
             const double* __restrict__ ys, const double* __restrict__ zs, const double* __restrict__ pxs,
             const double* __restrict__ pys, const double* __restrict__ pzs, const int* __restrict__ perm,
             double* __restrict__ pot, double* __restrict__ ax, double* __restrict__ ay, double* __restrict__ az) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t c = (int64_t)blockIdx.x * WARPS + w;
    if (c >= nleaf) return;
    const int side = 1 << depth;
    int ix, iy, iz;
    cell_coords(depth, c, ix, iy, iz);
    for (int t = start[c] + lane; t < start[c + 1]; t += 32) {
        const double x = xs[t], y = ys[t], z = zs[t];
        double ph = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
        for (int d = 0; d < 27; ++d) {
            const int jx = ix + d % 3 - 1, jy = iy + (d / 3) % 3 - 1, jz = iz + d / 9 - 1;
            if (jx < 0 || jy < 0 || jz < 0 || jx >= side || jy >= side || jz >= side) continue;
            const int64_t S = cell_index(depth, jx, jy, jz);
            for (int j = start[S]; j < start[S + 1]; ++j) {
                const double dx = x - xs[j], dy = y - ys[j], dz = z - zs[j];
                const double r2 = dx * dx + dy * dy + dz * dz;
                if (j == t || r2 == 0.0) continue;
                const double ir = 1.0 / sqrt(r2), ir3 = ir * ir * ir, ir5 = ir3 * ir * ir;
                const double pd = pxs[j] * dx + pys[j] * dy + pzs[j] * dz;
                ph += pd * ir3;
                gx += pxs[j] * ir3 - 3.0 * pd * dx * ir5;
                gy += pys[j] * ir3 - 3.0 * pd * dy * ir5;
                gz += pzs[j] * ir3 - 3.0 * pd * dz * ir5;
            }
        }
        const int o = perm[t];
        pot[o] -= ph; ax[o] += gx; ay[o] += gy; az[o] += gz;
    }
}

int launch_p2p_dipole(int depth, int64_t nleaf, const int* start, const double* xs, const double* ys,
                      const double* zs, const double* pxs, const double* pys, const double* pzs, const int* perm,
                      double* pot, double* ax, double* ay, double* az, cudaStream_t s) {
    if (nleaf <= 0) return 0;
    constexpr int W = 4;
    k_p2p_dipole<W><<<(unsigned)((nleaf + W - 1) / W), W * 32, 0, s>>>(depth, nleaf, start, xs, ys, zs, pxs, pys,
                                                                       pzs, perm, pot, ax, ay, az);
    count_launch();
    return 0;
}

// Dipole moments in the plan's sorted particle order: out[i] = in[perm[i]].
__global__ void k_gather3(int64_t n, const int* __restrict__ perm, const double* __restrict__ a,
                          const double* __restrict__ b, const double* __restrict__ c, double* __restrict__ oa,
                          double* __restrict__ ob, double* __restrict__ oc) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int j = perm[i];
    oa[i] = a[j]; ob[i] = b[j]; oc[i] = c[j];
}

int launch_gather3(int64_t n, const int* perm, const double* a, const double* b, const double* c, double* oa,
                   double* ob, double* oc, cudaStream_t s) {
    if (n <= 0) return 0;
    k_gather3<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, perm, a, b, c, oa, ob, oc);
    count_launch();
    return 0;
}

}  // namespace fmm
