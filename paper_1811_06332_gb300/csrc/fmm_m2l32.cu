// FP32 offset-grouped M2L support: the packed per-offset matrices
//   Kt_r(n, m) = D_{n+m}(r)/m!   (cell units, |n| + |m| <= p; Eq. M2L)
// built in FP64 from the D-tensor table and rounded once to FP32, and the
// FP64 -> FP32 copy of the multipoles they multiply.
#include "fmm_internal.h"

namespace fmm {

// ent[e] = (nx, ny, nz, mx, my, mz) of packed entry e (row n, column m).
__global__ void k_build_ktab(int ns, int ksz, int kst, const unsigned char* __restrict__ ent,
                             const double* __restrict__ Dtab, float* __restrict__ K) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)343 * kst) return;
    const int r = (int)(i / kst), e = (int)(i % kst);
    float v = 0.f;
    if (e < ksz) {
        const unsigned char* t = ent + 6 * e;
        const double d = Dtab[(int64_t)r * ns + pos_sym(t[0] + t[3], t[1] + t[4], t[2] + t[5])];
        v = (float)(d * c_invfact[t[3]] * c_invfact[t[4]] * c_invfact[t[5]]);
    }
    K[i] = v;
}

// The same packed matrices kept in FP64 (the plain FP64 form's grouped M2L).
__global__ void k_build_ktab64(int ns, int ksz, int kst, const unsigned char* __restrict__ ent,
                               const double* __restrict__ Dtab, double* __restrict__ K) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)343 * kst) return;
    const int r = (int)(i / kst), e = (int)(i % kst);
    double v = 0.0;
    if (e < ksz) {
        const unsigned char* t = ent + 6 * e;
        const double d = Dtab[(int64_t)r * ns + pos_sym(t[0] + t[3], t[1] + t[4], t[2] + t[5])];
        v = d * c_invfact[t[3]] * c_invfact[t[4]] * c_invfact[t[5]];
    }
    K[i] = v;
}

static int packed_size(int p, int basis) {
    int ksz = 0;
    const int nc = ncoef_of(p, basis == 2 ? 1 : basis);
    for (int r = 0; r < nc; ++r) {
        const unsigned char* n = basis ? fmm_tl_idx[r] : fmm_sym_idx[r];
        const int rem = p - n[0] - n[1] - n[2];
        ksz += basis == 1 ? nt_of(rem) : ns_of(rem);
    }
    return ksz;
}

int launch_build_ktab64(int p, int basis, int kst, const unsigned char* ent, const double* Dtab, double* K,
                        cudaStream_t s) {
    const int ksz = packed_size(p, basis);
    const int64_t tot = (int64_t)343 * kst;
    k_build_ktab64<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(ns_of(p), ksz, kst, ent, Dtab, K);
    count_launch();
    return ksz;
}

int launch_build_ktab(int p, int basis, int kst, const unsigned char* ent, const double* Dtab, float* K,
                      cudaStream_t s) {
    int ksz = 0;
    const int nc = ncoef_of(p, basis);
    for (int r = 0; r < nc; ++r) {
        const unsigned char* n = basis ? fmm_tl_idx[r] : fmm_sym_idx[r];
        const int rem = p - n[0] - n[1] - n[2];
        ksz += basis ? nt_of(rem) : ns_of(rem);
    }
    const int64_t tot = (int64_t)343 * kst;
    k_build_ktab<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(ns_of(p), ksz, kst, ent, Dtab, K);
    count_launch();
    return ksz;
}

// Host-side packed entry list in the generator's layout (rows in storage
// order, each followed by its prefix of columns).  basis 2 (the TG
// variant): traceless rows, full symmetric columns.
int grouped_entries(int p, int basis, unsigned char* out, int cap) {
    const int nc = ncoef_of(p, basis == 2 ? 1 : basis);
    int e = 0;
    for (int r = 0; r < nc; ++r) {
        const unsigned char* n = basis ? fmm_tl_idx[r] : fmm_sym_idx[r];
        const int rem = p - n[0] - n[1] - n[2];
        const int pre = basis == 1 ? nt_of(rem) : ns_of(rem);
        for (int c = 0; c < pre; ++c) {
            const unsigned char* m = basis == 1 ? fmm_tl_idx[c] : fmm_sym_idx[c];
            if (e >= cap) return -1;
            unsigned char* o = out + 6 * e;
            o[0] = n[0]; o[1] = n[1]; o[2] = n[2]; o[3] = m[0]; o[4] = m[1]; o[5] = m[2];
            ++e;
        }
    }
    return e;
}

__global__ void k_to_f32(int64_t n, const double* __restrict__ a, float* __restrict__ b) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (float)a[i];
}

int launch_to_f32(int64_t n, const double* a, float* b, cudaStream_t s) {
    if (n <= 0) return 0;
    k_to_f32<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, a, b);
    count_launch();
    return 0;
}

// M2M of one level from the per-child FP32 contributions (m2m32c):
// Mpa(r, P) = sum over the child classes c = 0..7, in that order, of
// part[(c nc + r) npa + P]; written in FP64 and to the FP32 copy Mpa32.
__global__ void k_m2m32_sum(int nc, int64_t npa, const float* __restrict__ part, double* __restrict__ Mpa,
                            float* __restrict__ Mpa32) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)nc * npa) return;
    const int64_t r = i / npa, P = i - r * npa;
    float v = part[r * npa + P];
#pragma unroll
    for (int c = 1; c < 8; ++c) v += part[((int64_t)c * nc + r) * npa + P];
    Mpa[i] = (double)v;
    Mpa32[i] = v;
}

int launch_m2m32_sum(int nc, int64_t npa, const float* part, double* Mpa, float* Mpa32, cudaStream_t s) {
    const int64_t n = (int64_t)nc * npa;
    if (n <= 0) return 0;
    k_m2m32_sum<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(nc, npa, part, Mpa, Mpa32);
    return 0;
}

// Partial sums of the split FP64 grouped M2L, added in group order.
__global__ void k_sum_parts(const double* __restrict__ part, double* __restrict__ Lt, int64_t m, int groups) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    double v = 0.0;
    for (int g = 0; g < groups; ++g) v += part[(int64_t)g * m + i];
    Lt[i] = v;
}

int launch_sum_parts(const double* part, double* Lt, int64_t m, int groups, cudaStream_t s) {
    if (m <= 0) return 0;
    k_sum_parts<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(part, Lt, m, groups);
    return 0;
}

// The same for FP32 locals: the groups' FP32 partial sums added in group order.
__global__ void k_sum_parts32(const float* __restrict__ part, float* __restrict__ Lt, int64_t m, int groups) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    float v = 0.f;
    for (int g = 0; g < groups; ++g) v += part[(int64_t)g * m + i];
    Lt[i] = v;
}

int launch_sum_parts(const float* part, float* Lt, int64_t m, int groups, cudaStream_t s) {
    if (m <= 0) return 0;
    k_sum_parts32<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(part, Lt, m, groups);
    return 0;
}

}  // namespace fmm
