// Device-side helpers shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "_gen/fmm_tables.h"

namespace fmm {

// Lt[i] = sum over g < groups of part[g m + i], in group order (fmm_m2l32.cu)
int launch_sum_parts(const double* part, double* Lt, int64_t m, int groups, cudaStream_t s);
int launch_sum_parts(const float* part, float* Lt, int64_t m, int groups, cudaStream_t s);
// Mpa(r, P) = sum over c = 0..7 of part[(c nc + r) npa + P], also to the FP32
// copy Mpa32 (fmm_m2l32.cu)
int launch_m2m32_sum(int nc, int64_t npa, const float* part, double* Mpa, float* Mpa32, cudaStream_t s);

// 1/sqrt(v): CUDA's double-precision rsqrt (at most 1 ulp from the exact
// value; one call in place of a rounded square root and a rounded division,
// which on this part's FP64 units costs several times the rest of a pair)
__device__ __forceinline__ double fmm_rsqrt(double v) { return rsqrt(v); }
// FP32: the PTX approximate reciprocal square root with subnormal inputs
// flushed to zero (one special-function instruction).  Its arguments are
// squared distances of FP32 offsets within a few cells, which for distinct
// points lie far above the subnormal range; exact zeros are excluded by the
// callers.
__device__ __forceinline__ float fmm_rsqrt(float v) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}

// Storage positions (App. D multi-indices; App. A compressed order).
__host__ __device__ __forceinline__ int ns_of(int p) { return p < 0 ? 0 : (p + 1) * (p + 2) * (p + 3) / 6; }
__host__ __device__ __forceinline__ int nt_of(int p) { return p < 0 ? 0 : (p + 1) * (p + 1); }
__host__ __device__ __forceinline__ int ncoef_of(int p, int basis) { return basis ? nt_of(p) : ns_of(p); }
// symmetric order: rank j block starts at ns(j-1); inside, (j-nx)(j-nx+1)/2 + nz
__host__ __device__ __forceinline__ int pos_sym(int nx, int ny, int nz) {
    const int j = nx + ny + nz, a = j - nx;
    return ns_of(j - 1) + a * (a + 1) / 2 + nz;
}
// independent (nz <= 1) traceless order: rank j block starts at j^2
__host__ __device__ __forceinline__ int pos_tl(int nx, int ny, int nz) {
    const int j = nx + ny + nz;
    return j * j + (nz == 0 ? ny : j + 1 + ny);
}

// Uniform octree cell numbering used for every level l >= 1: cells are
// grouped by the parity of their integer coordinates ("class" = x&1 |
// (y&1)<<1 | (z&1)<<2), then linear in (x>>1, y>>1, z>>1).  The 8 children
// of a parent at linear position P of level l-1 are then c*8^(l-1) + P.
__host__ __device__ __forceinline__ int64_t cell_index(int l, int ix, int iy, int iz) {
    if (l == 0) return 0;
    const int64_t hs = (int64_t)1 << (l - 1);
    const int cls = (ix & 1) | ((iy & 1) << 1) | ((iz & 1) << 2);
    return (int64_t)cls * hs * hs * hs + (((int64_t)(iz >> 1) * hs + (iy >> 1)) * hs + (ix >> 1));
}
__host__ __device__ __forceinline__ void cell_coords(int l, int64_t idx, int& ix, int& iy, int& iz) {
    if (l == 0) { ix = iy = iz = 0; return; }
    const int64_t hs = (int64_t)1 << (l - 1);
    const int64_t h3 = hs * hs * hs;
    const int cls = (int)(idx / h3);
    const int64_t lin = idx - cls * h3;
    const int jx = (int)(lin % hs), jy = (int)((lin / hs) % hs), jz = (int)(lin / (hs * hs));
    ix = 2 * jx + (cls & 1);
    iy = 2 * jy + ((cls >> 1) & 1);
    iz = 2 * jz + ((cls >> 2) & 1);
}
// plain linear index of level l (used for the parent of a child)
__host__ __device__ __forceinline__ int64_t lin_index(int l, int ix, int iy, int iz) {
    const int64_t s = (int64_t)1 << l;
    return ((int64_t)iz * s + iy) * s + ix;
}

}  // namespace fmm
