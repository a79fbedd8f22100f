// Binary median-split tree of App. C on the device: a cell holding more
// than max_leaf particles is split across the longest axis of its
// particles' bounding box (the first of x, y, z on ties) into two children
// with equal numbers of particles (the lower floor(n/2) by that coordinate,
// equal coordinates ordered by the particles' original index), the lower
// child first; cells are shrink-wrapped, centred on their particles'
// bounding box.
//
// Built level by level from three permutations P_x, P_y, P_z of the
// particles, each sorted once by (coordinate, index) and kept sorted inside
// every cell: the cells of a level occupy the same position ranges in all
// three.  A cell's bounding box is the first and last entry of its range in
// each P_a; its split along axis s sends the first half of its P_s range to
// the lower child; the other permutations follow by a stable partition of
// each cell range by that side (a scan of flags), which keeps them sorted
// inside the children.  Every pass is one thread per sorted position.
#include "fmm_adaptive.h"

namespace fmm {

// monotone map of a double to an unsigned key (-0 taken as +0, so that the
// two zeros compare equal as they do in floating point)
__device__ __forceinline__ uint64_t order64(double v) {
    const uint64_t u = (uint64_t)__double_as_longlong(v == 0.0 ? 0.0 : v);
    return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}

// sort keys of one axis (a stable radix sort of (key, index) from the
// identity orders equal coordinates by index)
__global__ void k_bt_axis_keys(int64_t n, const double* __restrict__ c, uint64_t* __restrict__ key,
                               int* __restrict__ val) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    key[i] = order64(c[i]);
    val[i] = (int)i;
}

// Centre (bounding-box centre), split axis and split decision of the nodes
// [lb, le): the bounding box along axis a is the first and last particle of
// the node's range in P_a.
__global__ void k_bt_nodes(int lb, int le, int max_leaf, const int* __restrict__ nb, const int* __restrict__ ne,
                           const int* __restrict__ P, int64_t n, const double* __restrict__ x,
                           const double* __restrict__ y, const double* __restrict__ z, double* __restrict__ zc,
                           int* __restrict__ axis, int* __restrict__ nsplit) {
    const int c = lb + blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= le) return;
    const int b = nb[c], e = ne[c];
    const double* co[3] = {x, y, z};
    double ext[3];
    for (int d = 0; d < 3; ++d) {
        const double lo = co[d][P[(int64_t)d * n + b]], hi = co[d][P[(int64_t)d * n + e - 1]];
        zc[3 * c + d] = __dmul_rn(__dadd_rn(lo, hi), 0.5);
        ext[d] = __dsub_rn(hi, lo);
    }
    int ax = 0;
    for (int d = 1; d < 3; ++d) if (ext[d] > ext[ax]) ax = d;
    axis[c] = ax;
    nsplit[c - lb] = e - b > max_leaf ? 2 : 0;
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

// side[i] = 1 for the particles of a splitting node that go to the upper
// child: those in the upper half of the node's range in P_s (s its axis).
__global__ void k_bt_side(int64_t n, int lb, int le, const int* __restrict__ node, const int* __restrict__ nb,
                          const int* __restrict__ ne, const int* __restrict__ nchild, const int* __restrict__ axis,
                          const int* __restrict__ P, unsigned char* __restrict__ side) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int c = node[k];
    if (c < lb || c >= le || !nchild[c]) return;
    const int b = nb[c], mid = b + (ne[c] - b) / 2;
    side[P[(int64_t)axis[c] * n + k]] = k >= mid ? 1 : 0;
}

// flag[k] = 1 where the particle at position k of P_a goes to the lower
// child (positions of nodes that do not split take any value: the
// partition leaves them in place)
__global__ void k_bt_flags(int64_t n, const int* __restrict__ Pa, const unsigned char* __restrict__ side,
                           int* __restrict__ flag) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) flag[k] = side[Pa[k]] ? 0 : 1;
}

// Stable partition of every splitting node's range of P_a by side: the
// lower child's particles first, each group in its order.  scan is the
// exclusive scan of flag over all positions, so scan[k] - scan[b] lower
// particles precede position k inside its node [b, e).
__global__ void k_bt_partition(int64_t n, int lb, int le, const int* __restrict__ node, const int* __restrict__ nb,
                               const int* __restrict__ ne, const int* __restrict__ nchild,
                               const int* __restrict__ Pa, const int* __restrict__ scan, int* __restrict__ Pn) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int c = node[k];
    if (c < lb || c >= le || !nchild[c]) {
        Pn[k] = Pa[k];
        return;
    }
    const int b = nb[c], mid = b + (ne[c] - b) / 2;
    const int low = scan[k] - scan[b];                  // lower particles before k in the node
    const bool is_low = scan[k + 1] - scan[k] != 0;
    const int64_t dst = is_low ? b + low : mid + (k - b - low);
    Pn[dst] = Pa[k];
}

// node[k]: the node of the next level holding position k (unchanged where
// the node does not split)
__global__ void k_bt_advance(int64_t n, int lb, int le, int* __restrict__ node, const int* __restrict__ nb,
                             const int* __restrict__ ne, const int* __restrict__ nchild,
                             const int* __restrict__ child0) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int c = node[k];
    if (c < lb || c >= le || !nchild[c]) return;
    const int b = nb[c], mid = b + (ne[c] - b) / 2;
    node[k] = child0[c] + (k >= mid ? 1 : 0);
}

#define BT_GRID(n) (unsigned)(((int64_t)(n) + 255) / 256), 256, 0, s
int bt_axis_keys(int64_t n, const double* c, uint64_t* key, int* val, cudaStream_t s) {
    if (n <= 0) return 0;
    k_bt_axis_keys<<<BT_GRID(n)>>>(n, c, key, val);
    count_launch();
    return 0;
}
int bt_nodes(int lb, int le, int max_leaf, const int* nb, const int* ne, const int* P, int64_t n, const double* x,
             const double* y, const double* z, double* zc, int* axis, int* nsplit, cudaStream_t s) {
    k_bt_nodes<<<BT_GRID(le - lb)>>>(lb, le, max_leaf, nb, ne, P, n, x, y, z, zc, axis, nsplit);
    count_launch();
    return 0;
}
int bt_children(int lb, int le, const int* nsplit, const int* off, int* lev, int* nb, int* ne, int* child0,
                int* nchild, int* parent, cudaStream_t s) {
    k_bt_children<<<BT_GRID(le - lb)>>>(lb, le, nsplit, off, lev, nb, ne, child0, nchild, parent);
    count_launch();
    return 0;
}
int bt_side(int64_t n, int lb, int le, const int* node, const int* nb, const int* ne, const int* nchild,
            const int* axis, const int* P, unsigned char* side, cudaStream_t s) {
    k_bt_side<<<BT_GRID(n)>>>(n, lb, le, node, nb, ne, nchild, axis, P, side);
    count_launch();
    return 0;
}
int bt_flags(int64_t n, const int* Pa, const unsigned char* side, int* flag, cudaStream_t s) {
    k_bt_flags<<<BT_GRID(n)>>>(n, Pa, side, flag);
    count_launch();
    return 0;
}
int bt_partition(int64_t n, int lb, int le, const int* node, const int* nb, const int* ne, const int* nchild,
                 const int* Pa, const int* scan, int* Pn, cudaStream_t s) {
    k_bt_partition<<<BT_GRID(n)>>>(n, lb, le, node, nb, ne, nchild, Pa, scan, Pn);
    count_launch();
    return 0;
}
int bt_advance(int64_t n, int lb, int le, int* node, const int* nb, const int* ne, const int* nchild,
               const int* child0, cudaStream_t s) {
    k_bt_advance<<<BT_GRID(n)>>>(n, lb, le, node, nb, ne, nchild, child0);
    count_launch();
    return 0;
}
#undef BT_GRID

}  // namespace fmm
