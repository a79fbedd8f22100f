// Binary median-split tree of App. C on the device: a cell holding more
// than max_leaf particles is split across the longest axis of its
// particles' bounding box (the first of x, y, z on ties) into two children
// with equal numbers of particles (the lower floor(n/2) by that coordinate,
// ties kept in the particles' current order), the lower child first; cells
// are shrink-wrapped, centred on their particles' bounding box.  Built
// level by level; each level reorders the particles of the cells it splits
// with two stable radix sorts (by the split coordinate, then by the start
// of the particle's cell, which restores every cell at its position).
#include "fmm_adaptive.h"

namespace fmm {

// Bounding box, centre and split decision of the nodes [lb, le): one block
// per node (grid-stride), particles of [nb, ne) read through perm.
__global__ void k_bt_nodes(int lb, int le, int max_leaf, const int* __restrict__ nb, const int* __restrict__ ne,
                           const int* __restrict__ perm, const double* __restrict__ x, const double* __restrict__ y,
                           const double* __restrict__ z, double* __restrict__ zc, int* __restrict__ axis,
                           int* __restrict__ nsplit) {
    __shared__ double s[6][256];
    for (int c = lb + blockIdx.x; c < le; c += gridDim.x) {
        double lo[3] = {1e308, 1e308, 1e308}, hi[3] = {-1e308, -1e308, -1e308};
        for (int a = nb[c] + threadIdx.x; a < ne[c]; a += blockDim.x) {
            const int i = perm[a];
            const double v[3] = {x[i], y[i], z[i]};
            for (int d = 0; d < 3; ++d) { lo[d] = fmin(lo[d], v[d]); hi[d] = fmax(hi[d], v[d]); }
        }
        for (int d = 0; d < 3; ++d) { s[d][threadIdx.x] = lo[d]; s[3 + d][threadIdx.x] = hi[d]; }
        __syncthreads();
        for (int o = blockDim.x / 2; o; o >>= 1) {
            if (threadIdx.x < o)
                for (int d = 0; d < 3; ++d) {
                    s[d][threadIdx.x] = fmin(s[d][threadIdx.x], s[d][threadIdx.x + o]);
                    s[3 + d][threadIdx.x] = fmax(s[3 + d][threadIdx.x], s[3 + d][threadIdx.x + o]);
                }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            double e[3];
            for (int d = 0; d < 3; ++d) {
                zc[3 * c + d] = __dmul_rn(__dadd_rn(s[d][0], s[3 + d][0]), 0.5);
                e[d] = __dsub_rn(s[3 + d][0], s[d][0]);
            }
            int ax = 0;
            for (int d = 1; d < 3; ++d) if (e[d] > e[ax]) ax = d;
            axis[c] = ax;
            nsplit[c - lb] = ne[c] - nb[c] > max_leaf ? 2 : 0;
        }
        __syncthreads();
    }
}

// Children of the splitting nodes: lower half [nb, mid), upper [mid, ne).
__global__ void k_bt_children(int lb, int le, const int* __restrict__ nsplit, const int* __restrict__ off,
                              int* __restrict__ lev, int* __restrict__ nb, int* __restrict__ ne,
                              int* __restrict__ child0, int* __restrict__ nchild, int* __restrict__ parent) {
    const int c = lb + blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= le) return;
    const int k = nsplit[c - lb];
    nchild[c] = k;
    child0[c] = k ? le + off[c - lb] : -1;
    if (!k) return;
    const int b = nb[c], e = ne[c], mid = b + (e - b) / 2;
    for (int j = 0; j < 2; ++j) {
        const int ch = le + off[c - lb] + j;
        lev[ch] = lev[c] + 1;
        nb[ch] = j ? mid : b;
        ne[ch] = j ? e : mid;
        parent[ch] = c;
        child0[ch] = -1;
        nchild[ch] = 0;
    }
}

// axis_at[a] = split axis of the node holding position a (3: not split)
__global__ void k_bt_mark(int lb, int le, const int* __restrict__ nb, const int* __restrict__ ne,
                          const int* __restrict__ nchild, const int* __restrict__ axis,
                          unsigned char* __restrict__ axis_at) {
    for (int c = lb + blockIdx.x; c < le; c += gridDim.x) {
        if (!nchild[c]) continue;
        const unsigned char ax = (unsigned char)axis[c];
        for (int a = nb[c] + threadIdx.x; a < ne[c]; a += blockDim.x) axis_at[a] = ax;
    }
}

// monotone map of a double to an unsigned key (-0 taken as +0, so that the
// two zeros compare equal as they do in floating point)
__device__ __forceinline__ uint64_t order64(double v) {
    const uint64_t u = (uint64_t)__double_as_longlong(v == 0.0 ? 0.0 : v);
    return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}

// pass 1 keys: the split coordinate (0 for particles whose cell is not split);
// the start of each particle's cell remembered by particle
__global__ void k_bt_keys1(int64_t n, const int* __restrict__ perm, const unsigned char* __restrict__ axis_at,
                           const int* __restrict__ segstart, const double* __restrict__ x,
                           const double* __restrict__ y, const double* __restrict__ z, uint64_t* __restrict__ key,
                           int* __restrict__ val, int* __restrict__ segof) {
    const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n) return;
    const int i = perm[a];
    const int ax = axis_at[a];
    key[a] = ax == 3 ? 0ull : order64(ax == 0 ? x[i] : ax == 1 ? y[i] : z[i]);
    val[a] = i;
    segof[i] = segstart[a];
}

// pass 2 keys: the start of the particle's cell
__global__ void k_bt_keys2(int64_t n, const int* __restrict__ val, const int* __restrict__ segof,
                           uint64_t* __restrict__ key) {
    const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a < n) key[a] = (uint64_t)segof[val[a]];
}

// the upper children start new cells
__global__ void k_bt_segstart(int lb, int le, const int* __restrict__ nb, const int* __restrict__ ne,
                              const int* __restrict__ nchild, int* __restrict__ segstart) {
    for (int c = lb + blockIdx.x; c < le; c += gridDim.x) {
        if (!nchild[c]) continue;
        const int mid = nb[c] + (ne[c] - nb[c]) / 2;
        for (int a = mid + threadIdx.x; a < ne[c]; a += blockDim.x) segstart[a] = mid;
    }
}

static unsigned blocks_for(int m) { return (unsigned)(m < 65535 ? (m > 0 ? m : 1) : 65535); }

int bt_nodes(int lb, int le, int max_leaf, const int* nb, const int* ne, const int* perm, const double* x,
             const double* y, const double* z, double* zc, int* axis, int* nsplit, cudaStream_t s) {
    k_bt_nodes<<<blocks_for(le - lb), 256, 0, s>>>(lb, le, max_leaf, nb, ne, perm, x, y, z, zc, axis, nsplit);
    count_launch();
    return 0;
}
int bt_children(int lb, int le, const int* nsplit, const int* off, int* lev, int* nb, int* ne, int* child0,
                int* nchild, int* parent, cudaStream_t s) {
    k_bt_children<<<(le - lb + 255) / 256, 256, 0, s>>>(lb, le, nsplit, off, lev, nb, ne, child0, nchild, parent);
    count_launch();
    return 0;
}
int bt_reorder_keys(int64_t n, int lb, int le, const int* nb, const int* ne, const int* nchild, const int* axis,
                    unsigned char* axis_at, const int* perm, const int* segstart, const double* x, const double* y,
                    const double* z, uint64_t* key, int* val, int* segof, cudaStream_t s) {
    cudaMemsetAsync(axis_at, 3, (size_t)n, s);
    k_bt_mark<<<blocks_for(le - lb), 256, 0, s>>>(lb, le, nb, ne, nchild, axis, axis_at);
    k_bt_keys1<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, perm, axis_at, segstart, x, y, z, key, val, segof);
    count_launch(); count_launch();
    return 0;
}
int bt_keys2(int64_t n, const int* val, const int* segof, uint64_t* key, cudaStream_t s) {
    k_bt_keys2<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, val, segof, key);
    count_launch();
    return 0;
}
int bt_segstart(int lb, int le, const int* nb, const int* ne, const int* nchild, int* segstart, cudaStream_t s) {
    k_bt_segstart<<<blocks_for(le - lb), 256, 0, s>>>(lb, le, nb, ne, nchild, segstart);
    count_launch();
    return 0;
}

}  // namespace fmm
