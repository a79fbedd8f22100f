// Per-device upload of the exact combinatorial maps (detracer, trace
// expansion, reduced representative) used by the operator kernels.
//
// Scaled units (uniform octree, cell side h at a level): the library stores
//   Mt_m = M_m / h^|m|,   Lt_n = L_n h^(|n|+1),
// so that every translation operator is the same at every level (shifts are
// +-h/4 per axis, M2L offsets are integer vectors in cell units) and every
// stored coefficient is O(1).  Powers of two scale exactly in floating point.
//
// Traceless basis inside the FMM: multipoles are kept as the unique tensor
// M^r supported on the nz <= 1 components with D[M^r] = Mbar (Eq. Detracer,
// App. A).  grad^k r^{-1} is trace free, so contracting it with M^r or with
// Mbar gives the same local expansion (Eq. M2L), with 2j+1 instead of
// (j+1)(j+2)/2 terms per multipole rank.
#include <cstdlib>

#include "fmm_internal.h"

namespace fmm {


static int g_tables_ready[64];
DevTables g_tab[64];

int ensure_tables(int dev) {
    if (dev < 0 || dev >= 64) return -1;
    if (g_tables_ready[dev]) return 0;
    DevTables& T = g_tab[dev];
    size_t nd = sizeof(fmm_detr_val), ne = sizeof(fmm_expand_val), nr = sizeof(fmm_reduce_val);
    if (cudaMalloc(&T.detr, nd) != cudaSuccess) return -3;
    if (cudaMalloc(&T.expand, ne) != cudaSuccess) return -3;
    if (cudaMalloc(&T.reduce, nr) != cudaSuccess) return -3;
    if (cudaMemcpy(T.detr, fmm_detr_val, nd, cudaMemcpyHostToDevice) != cudaSuccess) return -2;
    if (cudaMemcpy(T.expand, fmm_expand_val, ne, cudaMemcpyHostToDevice) != cudaSuccess) return -2;
    if (cudaMemcpy(T.reduce, fmm_reduce_val, nr, cudaMemcpyHostToDevice) != cudaSuccess) return -2;
    // FP32 copies for the FP32 forms (each table value rounded once)
    {
        const size_t cnt[3] = {nd / sizeof(double), ne / sizeof(double), nr / sizeof(double)};
        const double* src[3] = {fmm_detr_val, fmm_expand_val, fmm_reduce_val};
        float** dst[3] = {&T.detr32, &T.expand32, &T.reduce32};
        for (int k = 0; k < 3; ++k) {
            float* h = (float*)malloc(cnt[k] * sizeof(float));
            if (!h) return -3;
            for (size_t i = 0; i < cnt[k]; ++i) h[i] = (float)src[k][i];
            const bool ok = cudaMalloc(dst[k], cnt[k] * sizeof(float)) == cudaSuccess &&
                            cudaMemcpy(*dst[k], h, cnt[k] * sizeof(float), cudaMemcpyHostToDevice) == cudaSuccess;
            free(h);
            if (!ok) return -3;
        }
    }
    for (int j = 0; j <= FMM_PMAX + 1; ++j) {
        T.detr_off[j] = fmm_detr_off[j];
        T.expand_off[j] = fmm_expand_off[j];
        T.reduce_off[j] = fmm_reduce_off[j];
    }
    g_tables_ready[dev] = 1;
    return 0;
}

}  // namespace fmm
