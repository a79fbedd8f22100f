// Zero far field for trees too shallow for M2L, and a plain fill.
#include "fmm_internal.h"

namespace fmm {

// Zero far field (trees too shallow for M2L): overwrite outputs with 0.
__global__ void k_zero4(int64_t n, double* a, double* b, double* c, double* d) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) { a[i] = 0.0; b[i] = 0.0; c[i] = 0.0; d[i] = 0.0; }
}
int launch_zero4(int64_t n, double* a, double* b, double* c, double* d, cudaStream_t s) {
    if (n <= 0) return 0;
    k_zero4<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, a, b, c, d);
    count_launch();
    return 0;
}

// Fill n values with v.
__global__ void k_fill(int64_t n, double* a, double v) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = v;
}
int launch_fill(int64_t n, double* a, double v, cudaStream_t s) {
    if (n <= 0) return 0;
    k_fill<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, a, v);
    count_launch();
    return 0;
}

}  // namespace fmm
