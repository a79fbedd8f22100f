// Uniform octree construction (App. C, with the octree of the uniform
// workloads): leaf of a particle from its coordinates, a counting sort of the
// particles into leaves (stable by original index), and the leaf ranges.
#include "fmm_internal.h"
#include "fmm_fixpoint.h"

namespace fmm {

static inline int64_t align_up(int64_t v, int64_t a) { return (v + a - 1) / a * a; }

size_t tree_scratch_bytes(int64_t n, int64_t nleaf) {
    // keys[n], order[n], fill[nleaf], scan block sums (two levels + slack)
    int64_t b = 0;
    b += align_up(n * 4, 256);
    b += align_up(n * 4, 256);
    b += align_up(nleaf * 4, 256);
    const int64_t nb1 = (nleaf + 4095) / 4096 + 1;
    const int64_t nb2 = (nb1 + 4095) / 4096 + 1;
    b += 2 * align_up(nb1 * 4, 256) + 2 * align_up(nb2 * 4, 256) + 1024;
    return (size_t)b;
}

__global__ void k_leaf_key(int64_t n, int depth, const double* __restrict__ x, const double* __restrict__ y,
                           const double* __restrict__ z, int* __restrict__ key, int* __restrict__ count,
                           const double* __restrict__ q, float4* __restrict__ pc) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int side = 1 << depth;
    const double xi = x[i], yi = y[i], zi = z[i];
    // inside the unit cube: leaf and offset in integer fixed point
    // (fmm_fixpoint.h); else (a point on or outside the boundary) in FP64,
    // clamped to the boundary leaves
    int64_t X, Y, Z;
    const bool fix = fix62(xi, X) && fix62(yi, Y) && fix62(zi, Z);
    int ix, iy, iz;
    if (fix) {
        ix = fix62_leaf(X, depth); iy = fix62_leaf(Y, depth); iz = fix62_leaf(Z, depth);
    } else {
        const double fs = (double)side;
        ix = min(max((int)floor(xi * fs), 0), side - 1);
        iy = min(max((int)floor(yi * fs), 0), side - 1);
        iz = min(max((int)floor(zi * fs), 0), side - 1);
    }
    const int k = (int)cell_index(depth, ix, iy, iz);
    key[i] = k;
    atomicAdd(&count[k], 1);
    if (pc) {
        // FP32 forms: the position relative to the centre of its leaf, in
        // caller order (coalesced here; the gather then moves one 16-byte
        // record per particle)
        if (fix) {
            pc[i] = make_float4(fix62_offset(X, ix, depth), fix62_offset(Y, iy, depth), fix62_offset(Z, iz, depth),
                                (float)q[i]);
        } else {
            const double h = 1.0 / (double)side;
            pc[i] = make_float4((float)(xi - (ix + 0.5) * h), (float)(yi - (iy + 0.5) * h),
                                (float)(zi - (iz + 0.5) * h), (float)q[i]);
        }
    }
}

// Exclusive scan of int32, 4096 elements per block (1024 threads x 4).
__global__ void __launch_bounds__(1024) k_scan_block(const int* __restrict__ in, int* __restrict__ out, int64_t m,
                                                    int* __restrict__ bsum) {
    __shared__ int wsum[32];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int64_t base = (int64_t)blockIdx.x * 4096 + tid * 4;
    int v[4], tot = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) { v[k] = (base + k < m) ? in[base + k] : 0; tot += v[k]; }
    int inc = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) wsum[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        int s = wsum[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += t;
        }
        wsum[lane] = s;
    }
    __syncthreads();
    int ex = inc - tot + (wid ? wsum[wid - 1] : 0);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (base + k < m) out[base + k] = ex;
        ex += v[k];
    }
    if (tid == 1023) {
        if (bsum) bsum[blockIdx.x] = wsum[31];
        else out[m] = wsum[31];   // one block: its sum is the total
    }
}

// adds the scanned block sums; the last element's thread also writes the total
__global__ void k_scan_add(const int* __restrict__ in, int* __restrict__ out, int64_t m,
                           const int* __restrict__ bscan) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) {
        const int v = out[i] + bscan[i / 4096];
        out[i] = v;
        if (i == m - 1) out[m] = v + in[i];
    }
}

__global__ void k_scan_total(const int* __restrict__ in, int* __restrict__ out, int64_t m) {
    if (threadIdx.x == 0 && blockIdx.x == 0) out[m] = m > 0 ? out[m - 1] + in[m - 1] : 0;
}

// exclusive scan of in[0..m) into out[0..m], out[m] = total.  Scratch: two
// block-sum arrays per recursion level.
static void scan_excl(const int* in, int* out, int64_t m, int* scratch, cudaStream_t s) {
    const int64_t nb = (m + 4095) / 4096;
    if (m > 0) {
        int* bsum = scratch;
        int* bscan = scratch + align_up(nb + 1, 64);
        k_scan_block<<<(unsigned)nb, 1024, 0, s>>>(in, out, m, nb > 1 ? bsum : nullptr);
        count_launch();
        if (nb > 1) {
            scan_excl(bsum, bscan, nb, bscan + align_up(nb + 1, 64), s);
            k_scan_add<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(in, out, m, bscan);
            count_launch();
        }
        return;
    }
    k_scan_total<<<1, 32, 0, s>>>(in, out, m);   // m == 0: the total is 0
    count_launch();
}

void scan_excl_int(const int* in, int* out, int64_t m, int* scratch, cudaStream_t s) {
    scan_excl(in, out, m, scratch, s);
}

__global__ void k_scatter(int64_t n, const int* __restrict__ key, const int* __restrict__ start,
                          int* __restrict__ fill, int* __restrict__ order) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int k = key[i];
    order[start[k] + atomicAdd(&fill[k], 1)] = (int)i;
}

// Restores original order inside each leaf (the scatter's atomics are not
// ordered): insertion sort, one thread per leaf.
__global__ void k_leaf_sort(int64_t nleaf, const int* __restrict__ start, int* __restrict__ order) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nleaf) return;
    const int b = start[c], e = start[c + 1];
    for (int i = b + 1; i < e; ++i) {
        const int v = order[i];
        int j = i - 1;
        while (j >= b && order[j] > v) { order[j + 1] = order[j]; --j; }
        order[j + 1] = v;
    }
}

__global__ void k_gather(int64_t n, const int* __restrict__ order, const double* __restrict__ x,
                         const double* __restrict__ y, const double* __restrict__ z, const double* __restrict__ q,
                         double* __restrict__ xs, double* __restrict__ ys, double* __restrict__ zs,
                         double* __restrict__ qs, int* __restrict__ perm, const float4* __restrict__ pc,
                         float4* __restrict__ pos32) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int o = order[i];
    perm[i] = o;
    if (pos32) {
        // FP32 forms: only the FP32 leaf-relative positions (computed by
        // k_leaf_key); their operators read no sorted FP64 coordinates
        pos32[i] = pc[o];
        return;
    }
    xs[i] = x[o]; ys[i] = y[o]; zs[i] = z[o]; qs[i] = q[o];
}

int launch_uniform_tree(int64_t n, int depth, const double* x, const double* y, const double* z, const double* q,
                        double* xs, double* ys, double* zs, double* qs, int* perm, int* start, void* scratch,
                        cudaStream_t s, float4* pos32, float4* pos32c) {
    if (pos32 && !pos32c) return -1;
    const int64_t nleaf = (int64_t)1 << (3 * depth);
    char* p = (char*)scratch;
    int* key = (int*)p;   p += align_up(n * 4, 256);
    int* order = (int*)p; p += align_up(n * 4, 256);
    int* fill = (int*)p;  p += align_up(nleaf * 4, 256);
    int* sc = (int*)p;
    if (cudaMemsetAsync(fill, 0, nleaf * sizeof(int), s) != cudaSuccess) return -2;
    if (n > 0) {
        k_leaf_key<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, depth, x, y, z, key, fill, q, pos32 ? pos32c : nullptr);
        count_launch();
    }
    scan_excl(fill, start, nleaf, sc, s);
    if (cudaMemsetAsync(fill, 0, nleaf * sizeof(int), s) != cudaSuccess) return -2;
    if (n > 0) {
        k_scatter<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, key, start, fill, order);
        count_launch();
    }
    k_leaf_sort<<<(unsigned)((nleaf + 255) / 256), 256, 0, s>>>(nleaf, start, order);
    count_launch();
    if (n > 0) {
        k_gather<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, order, x, y, z, q, xs, ys, zs, qs, perm, pos32c, pos32);
        count_launch();
    }
    return 0;
}

}  // namespace fmm
