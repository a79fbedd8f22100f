// fmm_evaluate_noalloc: the FP64 uniform-octree FMM for callers that must
// not allocate device memory.  Every buffer the evaluation needs (sorted
// particles, leaf ranges, tree-build counters, expansions, translation
// matrices, D-tensor table, combinatorial tables) lives in one file-scope
// __device__ array of fixed size; nothing is allocated on any call.
#include <cstring>
#include <string>
#include <vector>

#include "fmm_gb300.h"
#include "fmm_internal.h"

namespace {

using namespace fmm;

constexpr int64_t NA_MAX_N = FMM_NOALLOC_MAX_N;
constexpr int NA_MAX_DEPTH = FMM_NOALLOC_MAX_DEPTH;
constexpr int NA_MAX_P = FMM_NOALLOC_MAX_P;
constexpr int64_t NA_NC = (NA_MAX_P + 1) * (NA_MAX_P + 2) * (NA_MAX_P + 3) / 6;  // largest ncoef
constexpr int64_t NA_NLEAF = (int64_t)1 << (3 * NA_MAX_DEPTH);
constexpr int64_t NA_NCELL = (((int64_t)1 << (3 * (NA_MAX_DEPTH + 1))) - 1) / 7;  // all levels

constexpr int64_t al(int64_t v) { return (v + 255) / 256 * 256; }
// layout (byte offsets)
constexpr int64_t O_DETR = 0;
constexpr int64_t O_EXPAND = O_DETR + al(sizeof(fmm_detr_val));
constexpr int64_t O_REDUCE = O_EXPAND + al(sizeof(fmm_expand_val));
constexpr int64_t O_OFFS = O_REDUCE + al(sizeof(fmm_reduce_val));
constexpr int64_t O_DTAB = O_OFFS + al(343 * 3 * 8);
constexpr int64_t NA_KST = 924;   // packed grouped-M2L entries, largest for p = 6: C(12, 6) (symmetric)
constexpr int64_t O_ENT = O_DTAB + al(343 * NA_NC * 8);
constexpr int64_t O_K64 = O_ENT + al(6 * NA_KST);
constexpr int64_t O_W = O_K64 + al(343 * NA_KST * 8);
constexpr int64_t O_V = O_W + al(8 * NA_NC * NA_NC * 8);
constexpr int64_t O_XS = O_V + al(8 * NA_NC * NA_NC * 8);
constexpr int64_t O_PERM = O_XS + al(4 * NA_MAX_N * 8);
constexpr int64_t O_START = O_PERM + al(NA_MAX_N * 4);
constexpr int64_t O_M = O_START + al((NA_NLEAF + 1) * 4);
constexpr int64_t O_L = O_M + al(NA_NC * NA_NCELL * 8);
constexpr int64_t O_TREE = O_L + al(NA_NC * NA_NCELL * 8);
// tree-build scratch: keys[n], order[n], fill[nleaf], scan block sums
constexpr int64_t NA_TREE_BYTES = al(NA_MAX_N * 4) + al(NA_MAX_N * 4) + al(NA_NLEAF * 4) + 4 * 256 + 1024;
constexpr int64_t NA_BYTES = O_TREE + NA_TREE_BYTES;
static_assert(NA_BYTES <= FMM_NOALLOC_BYTES_APPROX && NA_BYTES > FMM_NOALLOC_BYTES_APPROX - 100000,
              "FMM_NOALLOC_BYTES_APPROX states the array's size");

// The scratch array.  In host code its name is a host-side stand-in, not a
// device address: the device address is obtained with cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

struct NaState {
    unsigned char* base = nullptr;  // device address of g_noalloc_scratch whose tables are uploaded
    int p = -1, basis = -1;         // translation matrices currently held
};
NaState g_na[64];

}  // namespace

std::string& fmm_thread_error();  // read by fmm_last_error(NULL)
static int na_fail(int code, const char* msg, cudaError_t e = cudaSuccess) {
    std::string& t = fmm_thread_error();
    t = msg;
    if (e != cudaSuccess) { t += ": "; t += cudaGetErrorString(e); }
    return code;
}

static int na_dtable(int p, const double* o, double* D, cudaStream_t s) {
    switch (p) {
        case 0: return launch_dtable_p0(343, o, D, s);
        case 1: return launch_dtable_p1(343, o, D, s);
        case 2: return launch_dtable_p2(343, o, D, s);
        case 3: return launch_dtable_p3(343, o, D, s);
        case 4: return launch_dtable_p4(343, o, D, s);
        case 5: return launch_dtable_p5(343, o, D, s);
        default: return launch_dtable_p6(343, o, D, s);
    }
}

extern "C" int fmm_evaluate_noalloc(int p, int basis, int depth, int64_t n, const double* x, const double* y,
                                    const double* z, const double* q, double* pot, double* ax, double* ay,
                                    double* az, void* stream) {
    if (p < 0 || p > NA_MAX_P) return na_fail(FMM_ERR_ARG, "p outside 0..FMM_NOALLOC_MAX_P");
    if (basis != 0 && basis != 1) return na_fail(FMM_ERR_ARG, "unknown basis");
    if (depth < 0 || depth > NA_MAX_DEPTH) return na_fail(FMM_ERR_ARG, "depth outside 0..FMM_NOALLOC_MAX_DEPTH");
    if (n < 0 || n > NA_MAX_N) return na_fail(FMM_ERR_ARG, "n outside 0..FMM_NOALLOC_MAX_N");
    if (n > 0 && (!x || !y || !z || !q || !pot || !ax || !ay || !az)) return na_fail(FMM_ERR_ARG, "null array");
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return na_fail(FMM_ERR_CUDA, "cudaGetDevice failed", e);
    if (dev < 0 || dev >= 64) return na_fail(FMM_ERR_UNSUPPORTED, "device ordinal above 63");
    NaState& st = g_na[dev];
    // Set-up and rebuilds copy from host memory and wait for the stream;
    // neither may be recorded into a graph that the caller is capturing.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(s, &cap);
    if (e != cudaSuccess) return na_fail(FMM_ERR_CUDA, "cudaStreamIsCapturing failed", e);
    const bool capturing = cap != cudaStreamCaptureStatusNone;
    const char* cap_msg =
        "the first call on a device, and a call whose (p, basis) differs from the previous call's, "
        "must not be made while the stream is being captured";
    if (capturing && (!st.base || st.p != p || st.basis != basis)) return na_fail(FMM_ERR_STATE, cap_msg);
    // The array's device address is looked up on every call: a changed
    // address (the module was loaded again) repeats the set-up.
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return na_fail(FMM_ERR_CUDA, "cudaGetSymbolAddress failed", e);
    unsigned char* b = (unsigned char*)ptr;
    const bool setup = st.base != b;
    if (setup && capturing) return na_fail(FMM_ERR_STATE, cap_msg);
    if (setup) {
        // one-time set-up on this device: the constant combinatorial tables
        double offs[343 * 3];
        for (int o = 0; o < 343; ++o) {
            const int rx = o % 7 - 3, ry = (o / 7) % 7 - 3, rz = o / 49 - 3;
            const bool near = rx >= -1 && rx <= 1 && ry >= -1 && ry <= 1 && rz >= -1 && rz <= 1;
            offs[3 * o] = near ? 10.0 : rx;
            offs[3 * o + 1] = near ? 10.0 : ry;
            offs[3 * o + 2] = near ? 10.0 : rz;
        }
        st.base = nullptr;
        st.p = st.basis = -1;
        if ((e = cudaMemcpy(b + O_DETR, fmm_detr_val, sizeof(fmm_detr_val), cudaMemcpyHostToDevice)) ||
            (e = cudaMemcpy(b + O_EXPAND, fmm_expand_val, sizeof(fmm_expand_val), cudaMemcpyHostToDevice)) ||
            (e = cudaMemcpy(b + O_REDUCE, fmm_reduce_val, sizeof(fmm_reduce_val), cudaMemcpyHostToDevice)) ||
            (e = cudaMemcpy(b + O_OFFS, offs, sizeof(offs), cudaMemcpyHostToDevice)))
            return na_fail(FMM_ERR_CUDA, "uploading tables failed", e);
        st.base = b;
    }
    const int nc = ncoef_of(p, basis);
    if (st.p != p || st.basis != basis) {
        // translation matrices and D-tensor table for this order and basis
        std::vector<double> W, V;
        build_translation(p, basis, W, V);
        st.p = st.basis = -1;
        if ((e = cudaMemcpyAsync(b + O_W, W.data(), W.size() * 8, cudaMemcpyHostToDevice, s)) ||
            (e = cudaMemcpyAsync(b + O_V, V.data(), V.size() * 8, cudaMemcpyHostToDevice, s)))
            return na_fail(FMM_ERR_CUDA, "uploading translation matrices failed", e);
        static_assert(NA_MAX_P == 6, "na_dtable covers p = 0..6");
        if (na_dtable(p, (const double*)(b + O_OFFS), (double*)(b + O_DTAB), s) != 0)
            return na_fail(FMM_ERR_CUDA, "D-tensor table launch failed", cudaGetLastError());
        count_launch();
        // packed FP64 matrices of the grouped M2L, as the FP64 plan builds them
        const int kst = grouped_kstride(p, basis);
        if (kst < 0 || kst > NA_KST) return na_fail(FMM_ERR_ARG, "grouped M2L layout exceeds the fixed array");
        unsigned char ent[6 * NA_KST];
        if (grouped_entries(p, basis, ent, kst) < 0) return na_fail(FMM_ERR_ARG, "grouped M2L layout failed");
        if ((e = cudaMemcpyAsync(b + O_ENT, ent, (size_t)6 * kst, cudaMemcpyHostToDevice, s)))
            return na_fail(FMM_ERR_CUDA, "uploading the grouped M2L layout failed", e);
        launch_build_ktab64(p, basis, kst, b + O_ENT, (const double*)(b + O_DTAB), (double*)(b + O_K64), s);
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess)  // host arrays W, V, ent go out of scope
            return na_fail(FMM_ERR_CUDA, "set-up of matrices failed", e);
        st.p = p;
        st.basis = basis;
    }
    DevTables T;
    T.detr = (double*)(b + O_DETR);
    T.expand = (double*)(b + O_EXPAND);
    T.reduce = (double*)(b + O_REDUCE);
    for (int j = 0; j <= FMM_PMAX + 1; ++j) {
        T.detr_off[j] = fmm_detr_off[j];
        T.expand_off[j] = fmm_expand_off[j];
        T.reduce_off[j] = fmm_reduce_off[j];
    }
    const int64_t nleaf = (int64_t)1 << (3 * depth);
    double* xs = (double*)(b + O_XS);
    double *ys = xs + NA_MAX_N, *zs = xs + 2 * NA_MAX_N, *qs = xs + 3 * NA_MAX_N;
    int* perm = (int*)(b + O_PERM);
    int* start = (int*)(b + O_START);
    double* Mb = (double*)(b + O_M);
    double* Lb = (double*)(b + O_L);
    int64_t lo[NA_MAX_DEPTH + 1], tot = 0;
    for (int l = 0; l <= depth; ++l) { lo[l] = tot; tot += (int64_t)nc << (3 * l); }
    const double* W = (const double*)(b + O_W);
    const double* V = (const double*)(b + O_V);
    const double* K64 = (const double*)(b + O_K64);
    // the kernels fmm_evaluate runs for an FMM_FP64 uniform plan, in its order
    if (launch_uniform_tree(n, depth, x, y, z, q, xs, ys, zs, qs, perm, start, b + O_TREE, s) != 0)
        return na_fail(FMM_ERR_CUDA, "tree build failed", cudaGetLastError());
    launch_p2m_leaf(0, p, basis, depth, nleaf, start, xs, ys, zs, qs, Mb + lo[depth], T, s);
    for (int l = depth - 1; l >= 2; --l)
        launch_m2m_level(p, basis, l, W, Mb + lo[l + 1], (int64_t)1 << (3 * (l + 1)), Mb + lo[l],
                         (int64_t)1 << (3 * l), s);
    for (int l = 2; l <= depth; ++l) {
        const int parts = launch_m2l_grp64(p, basis, l, Mb + lo[l], Lb + lo[l], K64, (int64_t)1 << (3 * l), s,
                                           nullptr, 0);   // no room for partial sums: unsplit
        for (int k = 0; k < parts; ++k) count_launch();
    }
    for (int l = 2; l < depth; ++l)
        launch_l2l_level(p, basis, l, V, Lb + lo[l], (int64_t)1 << (3 * l), Lb + lo[l + 1],
                         (int64_t)1 << (3 * (l + 1)), s);
    if (depth >= 2)
        launch_l2p_leaf2(0, p, basis, depth, nleaf, start, xs, ys, zs, perm, Lb + lo[depth], T, pot, ax, ay, az, s);
    else
        launch_zero4(n, pot, ax, ay, az, s);
    launch_p2p_leaf2(0, depth, nleaf, start, xs, ys, zs, qs, perm, pot, ax, ay, az, s);
    if ((e = cudaGetLastError()) != cudaSuccess) return na_fail(FMM_ERR_CUDA, "kernel launch failed", e);
    return FMM_OK;
}
