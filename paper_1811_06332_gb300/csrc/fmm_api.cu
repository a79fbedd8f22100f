// C-ABI of the GB300 Cartesian FMM library (declared in include/fmm_gb300.h):
// argument validation, the plan (tree, expansions, operator matrices), the
// FMM pipeline of App. C, and the operator-level batched entry points.
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "fmm_gb300.h"
#include "fmm_adaptive.h"
#include "fmm_internal.h"
#include "fmm_learn.h"

namespace fmm {
static std::atomic<int64_t> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
}  // namespace fmm

using namespace fmm;

static thread_local std::string t_err;

struct fmm_plan {
    fmm_config cfg;
    int dev = 0;
    std::string err;
    int nc = 0, ns = 0;
    // tree
    int64_t n = -1;
    int depth = 0;
    int64_t nleaf = 0;
    bool built = false;
    double *xs = nullptr, *ys = nullptr, *zs = nullptr, *qs = nullptr;
    int* perm = nullptr;
    int* start = nullptr;
    void* scratch = nullptr;
    size_t scratch_bytes = 0;
    // expansions, levels 0..depth, each [nc][8^l]
    double* Mbuf = nullptr;
    double* Lbuf = nullptr;
    int64_t lvl_off[FMM_PMAX + 2];
    // operator matrices (scaled units)
    double* W = nullptr;     // 8 x nc x nc  (M2M)
    double* V = nullptr;     // 8 x nc x nc  (L2L)
    double* Dtab = nullptr;  // 343 x ns     (M2L, integer offsets in cell units)
    float* K32 = nullptr;    // 343 x kstride packed FP32 M2L matrices (FMM_FP32)
    double* K64 = nullptr;   // 343 x kstride packed FP64 M2L matrices (FMM_FP64)
    double* part64 = nullptr;   // partial sums of the split FP64 grouped M2L on small levels
    int64_t part64_cap = 0;
    float* M32 = nullptr;    // FP32 copy of the multipoles (FMM_FP32)
    float* msym32 = nullptr; // FP32 traceless forms: the leaves' symmetric moments, leaf-major (P2M)
    float* L32 = nullptr;    // uniform FP32 and tensor-core forms with FP32 shifts: the local expansions in FP32
    float* lpart = nullptr;  // their split small levels' M2L partial sums (FP32)
    int64_t lpart_cap = 0;
    int kst = 0;
    // tensor-core forms (FMM_GEMM_BF16X3, FMM_GEMM_TF32X3)
    void* Kbf = nullptr;                 // 343 x {hi, lo} preformatted matrices (streamed-matrix kernel)
    void* Kgen = nullptr;                // BF16: group table + FP32 D vectors (on-chip-matrix kernel)
    int tc_kern = 0, tc_cw = 48, tc_niss = 4;   // kernel shape in use
    // kernel 3: the multipole columns >= 48 on the CUDA cores
    float* Mrest = nullptr;              // 8^depth x rest_cstride(p): columns >= 48, cell-major FP32
    float* Krest = nullptr;              // 343 x rest_kstride(p) matrix entries of those columns
    float* Rpart = nullptr;              // level 5's source-class group sums of those products
    int64_t rpart_cap = 0;               // floats in Rpart
    int tc_source = 0;                   // 0 default, 1 autotuned, 2 from the cache, 3 set by the caller
    cudaGraphExec_t ugexec = nullptr;    // uniform plans with use_graph: the captured step
    const void* ugkey[11] = {nullptr};   // what the captured step depends on
    int tc_ncand = 0;
    int tc_cand[8][4];                   // autotuner candidates: kernel, cw, niss, microseconds
    void* Mbf = nullptr;                 // per level >= 4: hi then lo operand tiles
    int64_t mbf_off[FMM_PMAX + 2];       // element offset of level l's hi block
    std::vector<unsigned char> maps;     // tensor maps, one block per level
    int* derr = nullptr;                 // device error word (bounded waits)
    // FP32 forms: positions relative to leaf centres, packed FP32 shifts
    float4* pos32 = nullptr;
    float4* pos32c = nullptr;   // the same in caller order (tree build scratch)
    float* W32 = nullptr;
    float* V32 = nullptr;
    float* part32 = nullptr;   // per-child FP32 M2M contributions: 8 x nc x 8^(depth-1)
    // point dipoles in sorted order (fmm_evaluate_dipoles)
    double* dip = nullptr;
    // host-call staging
    double* stage = nullptr;
    int64_t stage_n = 0;
    // adaptive octree state (cfg.adaptive)
    AdState* ad = nullptr;
    int sms = 152;
    // learned per-pair order (cfg.learned_p)
    unsigned char* mlp_dev = nullptr;   // packed BF16 model (MLP_DEV_BYTES)
    bool mlp_set = false;
    float log10_kappa = 0.f;
};

static bool is_tc(int prec) { return prec == FMM_GEMM_BF16X3 || prec == FMM_GEMM_TF32X3; }

// Uniform FP32 and tensor-core plans on the per-child FP32 M2M: P2M and M2M
// keep M32 (the FP32 copy of the multipoles) current at every level, so the
// M2M and M2L kernels read it instead of converting the FP64 expansions again.
static bool m32_current(const fmm_plan* pl) { return !pl->ad && pl->M32 && pl->W32 && pl->part32; }

// Uniform FP32 and tensor-core plans with the FP32 level shifts keep their
// local expansions in FP32 only (L32): M2L writes them, L2L updates them and
// L2P reads them without a conversion to or from FP64 (an FP64 operation
// holds this part's narrow FP64 pipe for 16 cycles per warp).  L32 is
// allocated exactly when these conditions hold.
static float* L32lev(fmm_plan* pl, int l) { return pl->L32 ? pl->L32 + pl->lvl_off[l] : nullptr; }

// storage basis of the multipoles and of the local expansions (the TG
// basis: symmetric multipoles, traceless locals; Sec. 3)
static int bM(const fmm_plan* pl) { return pl->cfg.basis == FMM_BASIS_TG ? 0 : pl->cfg.basis; }
static int bL(const fmm_plan* pl) { return pl->cfg.basis == FMM_BASIS_TG ? 1 : pl->cfg.basis; }

static void* tc_maps_at(fmm_plan* pl, int l) {
    // 64-byte aligned block of the host-side tensor maps of level l
    uintptr_t b = ((uintptr_t)pl->maps.data() + 63) & ~(uintptr_t)63;
    return (void*)(b + (size_t)l * tc_maps_bytes());
}

// ---------------------------------------------------------------------------
// tensor-core kernel shape: kernel (0: streamed matrices, 1: matrices built
// on chip, BF16 only; 2: the matrix as the A operand and the cells of a tile
// as N, BF16 only, cw = 256 its N) and chunk width; the autotuner times the
// candidates on the plan's deepest level and keeps the fastest, cached on disk
// ---------------------------------------------------------------------------
static bool tc_shape_valid(int tf, int kern, int cw) {
    if (kern == 0) return cw == 16 || cw == 32 || cw == 48 || cw == 96;
    if (kern == 2 || kern == 3) return !tf && cw == 256;
    return kern == 1 && !tf && (cw == 16 || cw == 32 || cw == 48 || cw == 96);
}

static int tc_set_shape(fmm_plan* pl, int kern, int cw, cudaStream_t s) {
    const int tf = pl->cfg.prec == FMM_GEMM_TF32X3;
    if (kern == 0) {
        if (tc_build_mat(pl->cfg.p, tf, cw, pl->Dtab, pl->Kbf, s) != 0) return -2;
        pl->tc_niss = tc_mat_niss(pl->cfg.p, tf, cw);
    } else if (kern == 2 || kern == 3) {
        if (tct_bytes() > tc_mat_bytes(tf) || tct_build(pl->cfg.p, pl->Dtab, pl->Kbf, s) != 0) return -2;
        pl->tc_niss = 2;
        if (kern == 3 && rest_rows(pl->cfg.p) > 0 && !pl->Mrest) {
            const int p = pl->cfg.p;
            const size_t nmax = (size_t)1 << (3 * pl->depth);
            if (cudaMalloc(&pl->Mrest, (size_t)rest_cstride(p) * nmax * sizeof(float)) != cudaSuccess ||
                cudaMalloc(&pl->Krest, (size_t)343 * rest_kstride(p) * sizeof(float)) != cudaSuccess ||
                build_krest(p, pl->Dtab, pl->Krest, s) != 0)
                return -2;
            // level 5 (16^3 cells per class) splits its source classes
            if (pl->depth >= 5) {
                const int64_t cap = (int64_t)rest_nsplit(5) * rest_rows(p) * ((int64_t)1 << 15);
                if (cudaMalloc(&pl->Rpart, (size_t)cap * sizeof(float)) != cudaSuccess) return -2;
                pl->rpart_cap = cap;
            }
        }
    } else {
        if (tg_build(pl->cfg.p, cw, 1, pl->Dtab, pl->Kgen, s) != 0) return -2;
        pl->tc_niss = 1;
    }
    pl->tc_kern = kern;
    pl->tc_cw = cw;
    return 0;
}

static std::string tc_cache_path() {
    if (const char* e = getenv("FMM_TUNE_CACHE")) return e;
    if (const char* x = getenv("XDG_CACHE_HOME"))
        if (*x) return std::string(x) + "/fmm_gb300/tune.json";
    if (const char* h = getenv("HOME"))
        if (*h) return std::string(h) + "/.cache/fmm_gb300/tune.json";
    return "";
}

static std::string tc_cache_key(const fmm_plan* pl) {
    cudaDeviceProp prop;
    std::string gpu = cudaGetDeviceProperties(&prop, pl->dev) == cudaSuccess ? prop.name : "unknown GPU";
    char buf[160];
    snprintf(buf, sizeof buf, "|p=%d|basis=%d|prec=%d|depth=%d", pl->cfg.p, pl->cfg.basis, pl->cfg.prec, pl->depth);
    return gpu + buf;
}

// M2L of one tensor-core level in the plan's current kernel shape
static int tc_level_call(fmm_plan* pl, int l, cudaStream_t s) {
    const int tf = pl->cfg.prec == FMM_GEMM_TF32X3, es = tc_elem_bytes(tf);
    char* hp = (char*)pl->Mbf + pl->mbf_off[l] * es;
    char* lp = hp + tc_m_elems(l) * es;
    const int p = pl->cfg.p;
    const float* m32 = m32_current(pl) ? pl->M32 + pl->lvl_off[l] : nullptr;
    const int rc = tc_m2l_level(p, tf, pl->tc_kern, pl->tc_cw, pl->tc_niss, l, pl->Mbuf + pl->lvl_off[l], hp, lp,
                                tc_maps_at(pl, l), pl->tc_kern == 1 ? pl->Kgen : pl->Kbf, pl->Lbuf + pl->lvl_off[l],
                                pl->derr, s, m32, L32lev(pl, l));
    // kernel 3: the multipole columns >= 48 (a cell-major FP32 copy of
    // them, then their products) on the CUDA cores, added to L
    if (rc == 0 && pl->tc_kern == 3 && rest_rows(p) > 0 &&
        (launch_rest_pack(p, l, pl->Mbuf + pl->lvl_off[l], pl->Mrest, s, m32) != 0 ||
         launch_m2l_rest(p, l, pl->Mrest, pl->Krest, pl->Lbuf + pl->lvl_off[l], s, L32lev(pl, l), pl->Rpart,
                         pl->rpart_cap) != 0))
        return -2;
    return rc;
}

// Times every candidate shape on level `l` (one warm-up and one timed
// launch each; the level's locals are overwritten by the real call after)
// and keeps the fastest.
static int tc_autotune(fmm_plan* pl, int l, cudaStream_t s) {
    const int tf = pl->cfg.prec == FMM_GEMM_TF32X3;
    static const int cand_bf16[][2] = {{0, 32}, {0, 48}, {0, 96}, {1, 48}, {1, 96}, {2, 256}, {3, 256}};
    static const int cand_tf32[][2] = {{0, 16}, {0, 32}, {0, 48}};
    const int (*cand)[2] = tf ? cand_tf32 : cand_bf16;
    const int nc = tf ? 3 : 7;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return -2;
    int best = -1;
    float bt = 1e30f;
    pl->tc_ncand = 0;
    for (int c = 0; c < nc; ++c) {
        if (tc_set_shape(pl, cand[c][0], cand[c][1], s) != 0) { best = -2; break; }
        if (tc_level_call(pl, l, s) != 0) { best = -2; break; }
        cudaEventRecord(e0, s);
        if (tc_level_call(pl, l, s) != 0) { best = -2; break; }
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) { best = -2; break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        int* r = pl->tc_cand[pl->tc_ncand++];
        r[0] = cand[c][0]; r[1] = cand[c][1]; r[2] = pl->tc_niss; r[3] = (int)(ms * 1000.f);
        if (ms < bt) { bt = ms; best = c; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (best < 0) return -2;
    if (tc_set_shape(pl, cand[best][0], cand[best][1], s) != 0) return -2;
    pl->tc_source = 1;
    const std::string path = tc_cache_path();
    if (!path.empty())
        tune_cache_put(path.c_str(), tc_cache_key(pl).c_str(), pl->tc_kern, pl->tc_cw, pl->tc_niss, bt);
    return 0;
}


static int fail_plan(fmm_plan* pl, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (pl) pl->err = buf;
    t_err = buf;
    return code;
}
#define FAIL(code, ...) return fail_plan(pl, code, __VA_ARGS__)
#define CK(call)                                                                                 \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess) FAIL(FMM_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)
#define CKLAUNCH()                                                                                    \
    do {                                                                                              \
        cudaError_t e_ = cudaGetLastError();                                                          \
        if (e_ != cudaSuccess) FAIL(FMM_ERR_CUDA, "kernel launch failed: %s", cudaGetErrorString(e_)); \
    } while (0)

static int tables_for_current(fmm_plan* pl, int* dev_out) {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    const int rc = ensure_tables(dev);
    if (rc == -3) FAIL(FMM_ERR_OOM, "allocating constant tables failed");
    if (rc != 0) FAIL(FMM_ERR_CUDA, "uploading constant tables failed");
    *dev_out = dev;
    return FMM_OK;
}

typedef int (*pair_launch_t)(int, int, int64_t, const void*, const double*, void*, int, cudaStream_t);
typedef int (*dten_launch_t)(int, int, int64_t, const double*, void*, cudaStream_t);
typedef int (*dtab_launch_t)(int, const double*, double*, cudaStream_t);
static const pair_launch_t k_pair[FMM_PMAX + 1] = {
    launch_m2l_pair_p0, launch_m2l_pair_p1, launch_m2l_pair_p2, launch_m2l_pair_p3,
    launch_m2l_pair_p4, launch_m2l_pair_p5, launch_m2l_pair_p6, launch_m2l_pair_p7,
    launch_m2l_pair_p8, launch_m2l_pair_p9, launch_m2l_pair_p10};
static const dten_launch_t k_dten[FMM_PMAX + 1] = {
    launch_dtensor_p0, launch_dtensor_p1, launch_dtensor_p2, launch_dtensor_p3,
    launch_dtensor_p4, launch_dtensor_p5, launch_dtensor_p6, launch_dtensor_p7,
    launch_dtensor_p8, launch_dtensor_p9, launch_dtensor_p10};
static const dtab_launch_t k_dtab[FMM_PMAX + 1] = {
    launch_dtable_p0, launch_dtable_p1, launch_dtable_p2, launch_dtable_p3,
    launch_dtable_p4, launch_dtable_p5, launch_dtable_p6, launch_dtable_p7,
    launch_dtable_p8, launch_dtable_p9, launch_dtable_p10};

// Thread-local error text of plan-less calls, also set by fmm_noalloc.cu.
std::string& fmm_thread_error() { return t_err; }

static inline cudaStream_t S(void* s) { return (cudaStream_t)s; }

extern "C" {

int fmm_ncoef(int p, int basis) {
    if (p < 0 || p > FMM_PMAX || (basis != 0 && basis != 1)) return FMM_ERR_ARG;
    return ncoef_of(p, basis);
}

const char* fmm_last_error(const fmm_plan* plan) { return plan ? plan->err.c_str() : t_err.c_str(); }

int64_t fmm_kernel_launches(void) { return g_launches.load(); }

int fmm_tc_layout(int p, int prec, int* out, int nout) {
    if (prec != FMM_GEMM_TF32X3) return FMM_ERR_ARG;
    if (!tc_supported(p, FMM_BASIS_TRACELESS) || !out || nout < 0) return FMM_ERR_ARG;
    return tc_layout(p, prec == FMM_GEMM_TF32X3, out, nout);
}

int fmm_tc_gen_layout(int p, int cw, int niss, int* out, int nout, uint32_t* groups, int gcap) {
    if (!out || nout < 0 || gcap < 0 || (gcap > 0 && !groups)) return fail_plan(nullptr, FMM_ERR_ARG, "bad output");
    const int n = tg_layout_host(p, cw, niss, out, nout, groups, gcap);
    if (n < 0) return fail_plan(nullptr, FMM_ERR_ARG, "p=%d, cw=%d, niss=%d not supported", p, cw, niss);
    return n;
}

int fmm_set_tc_shape(fmm_plan* pl, int kernel, int cw) {
    if (!pl) return fail_plan(nullptr, FMM_ERR_ARG, "plan is NULL");
    if (!is_tc(pl->cfg.prec) || pl->ad) FAIL(FMM_ERR_ARG, "not a tensor-core plan");
    if (!tc_shape_valid(pl->cfg.prec == FMM_GEMM_TF32X3, kernel, cw))
        FAIL(FMM_ERR_ARG, "kernel %d with chunk width %d is not a shape of this form", kernel, cw);
    if (tc_set_shape(pl, kernel, cw, 0) != 0 || cudaDeviceSynchronize() != cudaSuccess)
        FAIL(FMM_ERR_CUDA, "building the offset matrices failed: %s", cudaGetErrorString(cudaGetLastError()));
    pl->tc_source = 3;
    return FMM_OK;
}

int fmm_plan_tuning(const fmm_plan* pl, int* out, int nout) {
    if (!pl || !out || nout < 0) return fail_plan(nullptr, FMM_ERR_ARG, "null plan or output");
    if (!is_tc(pl->cfg.prec) || pl->ad) return fail_plan(nullptr, FMM_ERR_ARG, "not a tensor-core plan");
    int v[5 + 4 * 8], n = 0;
    v[n++] = pl->tc_kern; v[n++] = pl->tc_cw; v[n++] = pl->tc_niss; v[n++] = pl->tc_source; v[n++] = pl->tc_ncand;
    for (int c = 0; c < pl->tc_ncand; ++c)
        for (int k = 0; k < 4; ++k) v[n++] = pl->tc_cand[c][k];
    const int m = nout < n ? nout : n;
    for (int i = 0; i < m; ++i) out[i] = v[i];
    return m;
}

int fmm_tune_cache_get(const char* path, const char* key, int* vals) {
    if (!path || !key || !vals) return fail_plan(nullptr, FMM_ERR_ARG, "null argument");
    return tune_cache_get(path, key, vals, vals + 1, vals + 2, nullptr);
}

int fmm_tune_cache_put(const char* path, const char* key, const int* vals, double ms) {
    if (!path || !key || !vals) return fail_plan(nullptr, FMM_ERR_ARG, "null argument");
    const int r = tune_cache_put(path, key, vals[0], vals[1], vals[2], ms);
    if (r == -2) return fail_plan(nullptr, FMM_ERR_STATE, "writing %s failed", path);
    return r == 0 ? FMM_OK : fail_plan(nullptr, FMM_ERR_ARG, "bad path or key");
}

int fmm_plan_stats(const fmm_plan* pl, int64_t* out, int nout) {
    if (!pl || !out || nout < 0) return fail_plan(nullptr, FMM_ERR_ARG, "null plan or output");
    int64_t v[19] = {0};
    if (pl->ad && pl->cfg.learned_p && nout > 8 && pl->built)
        ad_order_counts(pl->ad, pl->cfg.p, v + 8, 0);
    if (pl->ad) {
        const AdState* A = pl->ad;
        v[0] = A->nn; v[1] = A->nleaf; v[2] = A->nm2l; v[3] = A->np2p; v[4] = A->ntarg;
        v[5] = A->m2l_blocks_per_sm; v[6] = A->lvl.empty() ? 0 : (int64_t)A->lvl.size() - 1;
        v[7] = A->gexec ? 1 : 0;
    } else {
        int64_t cells = 0;
        for (int l = 0; l <= pl->depth; ++l) cells += (int64_t)1 << (3 * l);
        v[0] = cells; v[1] = pl->nleaf; v[6] = pl->depth + 1;
        v[7] = pl->ugexec ? 1 : 0;
    }
    for (int k = 0; k < nout && k < 19; ++k) out[k] = v[k];
    return FMM_OK;
}

// ---------------------------------------------------------------------------
// operator-level entry points
// ---------------------------------------------------------------------------
int fmm_op_dtensor(int p, int basis, int prec, int64_t n, const double* r, void* D, void* stream) {
    fmm_plan* pl = nullptr;
    if (p < 0 || p > FMM_PMAX) FAIL(FMM_ERR_ARG, "p=%d outside 0..%d", p, FMM_PMAX);
    if (basis != 0 && basis != 1) FAIL(FMM_ERR_ARG, "unknown basis %d", basis);
    if (prec != FMM_FP64 && prec != FMM_FP32) FAIL(FMM_ERR_ARG, "prec must be FMM_FP64 or FMM_FP32");
    if (n < 0) FAIL(FMM_ERR_ARG, "n < 0");
    if (n > 0 && (!r || !D)) FAIL(FMM_ERR_ARG, "null array");
    k_dten[p](basis, prec, n, r, D, S(stream));
    if (n > 0) count_launch();
    CKLAUNCH();
    return FMM_OK;
}

int fmm_op_m2l(int p, int basis, int prec, int64_t n, const void* M, const double* r, void* L, int accumulate,
               void* stream) {
    fmm_plan* pl = nullptr;
    if (p < 0 || p > FMM_PMAX) FAIL(FMM_ERR_ARG, "p=%d outside 0..%d", p, FMM_PMAX);
    if (basis != 0 && basis != 1) FAIL(FMM_ERR_ARG, "unknown basis %d", basis);
    if (prec != FMM_FP64 && prec != FMM_FP32) FAIL(FMM_ERR_ARG, "prec must be FMM_FP64 or FMM_FP32");
    if (n < 0) FAIL(FMM_ERR_ARG, "n < 0");
    if (n > 0 && (!M || !r || !L)) FAIL(FMM_ERR_ARG, "null array");
    if (k_pair[p](basis, prec, n, M, r, L, accumulate, S(stream)) != 0) FAIL(FMM_ERR_ARG, "bad combination");
    if (n > 0) count_launch();
    CKLAUNCH();
    return FMM_OK;
}

int fmm_op_p2m(int p, int basis, int64_t ncell, const int64_t* start, const double* x, const double* y,
               const double* z, const double* q, const double* centre, double* M, void* stream) {
    fmm_plan* pl = nullptr;
    if (p < 0 || p > FMM_PMAX) FAIL(FMM_ERR_ARG, "p=%d outside 0..%d", p, FMM_PMAX);
    if (basis != 0 && basis != 1) FAIL(FMM_ERR_ARG, "unknown basis %d", basis);
    if (ncell < 0) FAIL(FMM_ERR_ARG, "ncell < 0");
    if (ncell > 0 && (!start || !x || !y || !z || !q || !centre || !M)) FAIL(FMM_ERR_ARG, "null array");
    int dev;
    if (int rc = tables_for_current(pl, &dev)) return rc;
    launch_p2m(p, basis, 0, ncell, start, nullptr, x, y, z, q, centre, 0, 1.0, M, ncell, g_tab[dev], S(stream));
    CKLAUNCH();
    return FMM_OK;
}

int fmm_op_m2m(int p, int basis, int prec, int64_t n, const void* Mc, const double* delta, void* Mp,
               void* stream) {
    fmm_plan* pl = nullptr;
    if (p < 0 || p > FMM_PMAX) FAIL(FMM_ERR_ARG, "p=%d outside 0..%d", p, FMM_PMAX);
    if (basis != 0 && basis != 1) FAIL(FMM_ERR_ARG, "unknown basis %d", basis);
    if (prec != FMM_FP64 && prec != FMM_FP32) FAIL(FMM_ERR_ARG, "prec must be FMM_FP64 or FMM_FP32");
    if (n < 0) FAIL(FMM_ERR_ARG, "n < 0");
    if (n > 0 && (!Mc || !delta || !Mp)) FAIL(FMM_ERR_ARG, "null array");
    if (n > 0 && Mc == Mp) FAIL(FMM_ERR_ARG, "Mc and Mp must be distinct");
    int dev;
    if (int rc = tables_for_current(pl, &dev)) return rc;
    launch_m2m_general(prec, p, basis, n, Mc, delta, Mp, g_tab[dev], S(stream));
    CKLAUNCH();
    return FMM_OK;
}

int fmm_op_m2m_fused(int p, int64_t n, const double* Mc, const double* delta, double* Mp, void* stream) {
    fmm_plan* pl = nullptr;
    if (p < 0 || p > FMM_PMAX) FAIL(FMM_ERR_ARG, "p=%d outside 0..%d", p, FMM_PMAX);
    if (n < 0) FAIL(FMM_ERR_ARG, "n < 0");
    if (n > 0 && (!Mc || !delta || !Mp)) FAIL(FMM_ERR_ARG, "null array");
    if (n > 0 && Mc == Mp) FAIL(FMM_ERR_ARG, "Mc and Mp must be distinct");
    int dev;
    if (int rc = tables_for_current(pl, &dev)) return rc;
    const int r = launch_m2m_fused(p, n, Mc, delta, Mp, g_tab[dev], S(stream));
    if (r == -3) FAIL(FMM_ERR_OOM, "allocating the fused M2M table failed");
    if (r) FAIL(FMM_ERR_CUDA, "uploading the fused M2M table failed");
    CKLAUNCH();
    return FMM_OK;
}

int fmm_m2m_fused_terms(int p) {
    if (p < 0 || p > FMM_PMAX) return fail_plan(nullptr, FMM_ERR_ARG, "p=%d outside 0..%d", p, FMM_PMAX);
    return m2m_fused_terms(p);
}

int fmm_op_l2l(int p, int basis, int prec, int64_t n, const void* Lp, const double* delta, void* Lc,
               void* stream) {
    fmm_plan* pl = nullptr;
    if (p < 0 || p > FMM_PMAX) FAIL(FMM_ERR_ARG, "p=%d outside 0..%d", p, FMM_PMAX);
    if (basis != 0 && basis != 1) FAIL(FMM_ERR_ARG, "unknown basis %d", basis);
    if (prec != FMM_FP64 && prec != FMM_FP32) FAIL(FMM_ERR_ARG, "prec must be FMM_FP64 or FMM_FP32");
    if (n < 0) FAIL(FMM_ERR_ARG, "n < 0");
    if (n > 0 && (!Lp || !delta || !Lc)) FAIL(FMM_ERR_ARG, "null array");
    if (n > 0 && Lp == Lc) FAIL(FMM_ERR_ARG, "Lp and Lc must be distinct");
    int dev;
    if (int rc = tables_for_current(pl, &dev)) return rc;
    launch_l2l_general(prec, p, basis, n, Lp, delta, Lc, g_tab[dev], S(stream));
    CKLAUNCH();
    return FMM_OK;
}

int fmm_op_l2p(int p, int basis, int prec, int64_t n, const void* L, const double* rb, void* out, void* stream) {
    fmm_plan* pl = nullptr;
    if (p < 0 || p > FMM_PMAX) FAIL(FMM_ERR_ARG, "p=%d outside 0..%d", p, FMM_PMAX);
    if (basis != 0 && basis != 1) FAIL(FMM_ERR_ARG, "unknown basis %d", basis);
    if (prec != FMM_FP64 && prec != FMM_FP32) FAIL(FMM_ERR_ARG, "prec must be FMM_FP64 or FMM_FP32");
    if (n < 0) FAIL(FMM_ERR_ARG, "n < 0");
    if (n > 0 && (!L || !rb || !out)) FAIL(FMM_ERR_ARG, "null array");
    int dev;
    if (int rc = tables_for_current(pl, &dev)) return rc;
    launch_l2p_general(prec, p, basis, n, L, rb, out, g_tab[dev], S(stream));
    CKLAUNCH();
    return FMM_OK;
}

int fmm_direct(int64_t n, const double* x, const double* y, const double* z, const double* q, int64_t nt,
               const int64_t* targets, double* pot, double* ax, double* ay, double* az, void* stream) {
    fmm_plan* pl = nullptr;
    if (n < 0) FAIL(FMM_ERR_ARG, "n < 0");
    if (!targets) nt = n;
    if (nt < 0) FAIL(FMM_ERR_ARG, "nt < 0");
    if (n > 0 && (!x || !y || !z || !q)) FAIL(FMM_ERR_ARG, "null source array");
    if (nt > 0 && (!pot || !ax || !ay || !az)) FAIL(FMM_ERR_ARG, "null output array");
    launch_direct(n, x, y, z, q, nt, targets, pot, ax, ay, az, S(stream));
    CKLAUNCH();
    return FMM_OK;
}

// ---------------------------------------------------------------------------
// plan
// ---------------------------------------------------------------------------
static void free_tree(fmm_plan* pl) {
    cudaFree(pl->xs); cudaFree(pl->ys); cudaFree(pl->zs); cudaFree(pl->qs);
    cudaFree(pl->perm); cudaFree(pl->start); cudaFree(pl->scratch);
    cudaFree(pl->Mbuf); cudaFree(pl->Lbuf); cudaFree(pl->M32); cudaFree(pl->Mbf); cudaFree(pl->pos32);
    cudaFree(pl->dip); cudaFree(pl->msym32); cudaFree(pl->L32); cudaFree(pl->lpart); cudaFree(pl->pos32c);
    pl->pos32c = nullptr;
    pl->msym32 = nullptr;
    pl->L32 = nullptr;
    pl->lpart = nullptr;
    pl->lpart_cap = 0;
    pl->dip = nullptr;
    pl->pos32 = nullptr;
    pl->M32 = nullptr;
    pl->Mbf = nullptr;
    pl->xs = pl->ys = pl->zs = pl->qs = nullptr;
    pl->perm = pl->start = nullptr;
    pl->scratch = nullptr;
    pl->Mbuf = pl->Lbuf = nullptr;
    pl->n = -1;
    pl->built = false;
}

// Translation matrices in scaled units (level independent):
//   M2M  Mt_n(parent) = sum_k n!/(k!(n-k)!) (-d)^(n-k) 2^-|k| Mt_k(child)
//   L2L  Lt_n(child)  = sum_k d^k/k! 2^-(|n|+1) Lt_(n+k)(parent)
// d = (z_child - z_parent)/h_parent = (+-1/4, +-1/4, +-1/4) for child class c
// (bit 0: x, bit 1: y, bit 2: z).  Traceless: M2M acts on the reduced
// representative (embed nz<=1 comps, shift, reduce), L2L on independent
// components (expand by the trace condition, shift, keep independent rows).
void build_translation(int p, int basis, std::vector<double>& W, std::vector<double>& V) {
    const int ns = ns_of(p), nc = ncoef_of(p, basis);
    std::vector<double> Sm((size_t)ns * ns), Vs((size_t)ns * ns);
    W.assign((size_t)8 * nc * nc, 0.0);
    V.assign((size_t)8 * nc * nc, 0.0);
    auto fact = [](int k) { double f = 1; for (int i = 2; i <= k; ++i) f *= i; return f; };
    auto binom = [&](int a, int b) { return fact(a) / (fact(b) * fact(a - b)); };
    auto ipow = [](double v, int e) { double r = 1; for (int i = 0; i < e; ++i) r *= v; return r; };
    for (int c = 0; c < 8; ++c) {
        const double d[3] = {(c & 1) ? 0.25 : -0.25, (c & 2) ? 0.25 : -0.25, (c & 4) ? 0.25 : -0.25};
        for (int a = 0; a < ns; ++a) {
            const unsigned char* n = fmm_sym_idx[a];
            for (int b = 0; b < ns; ++b) {
                const unsigned char* k = fmm_sym_idx[b];
                double s = 0.0, v = 0.0;
                if (k[0] <= n[0] && k[1] <= n[1] && k[2] <= n[2]) {
                    s = std::ldexp(1.0, -(k[0] + k[1] + k[2]));
                    for (int e = 0; e < 3; ++e) s *= binom(n[e], k[e]) * ipow(-d[e], n[e] - k[e]);
                }
                // Vs[a][b]: row n, column j = b with j >= n
                const unsigned char* j = k;
                if (j[0] >= n[0] && j[1] >= n[1] && j[2] >= n[2]) {
                    v = std::ldexp(1.0, -(n[0] + n[1] + n[2] + 1));
                    for (int e = 0; e < 3; ++e) v *= ipow(d[e], j[e] - n[e]) / fact(j[e] - n[e]);
                }
                Sm[(size_t)a * ns + b] = s;
                Vs[(size_t)a * ns + b] = v;
            }
        }
        double* Wc = W.data() + (size_t)c * nc * nc;
        double* Vc = V.data() + (size_t)c * nc * nc;
        if (!basis) {
            std::memcpy(Wc, Sm.data(), sizeof(double) * ns * ns);
            std::memcpy(Vc, Vs.data(), sizeof(double) * ns * ns);
            continue;
        }
        for (int to = 0; to < nc; ++to) {
            const unsigned char* no = fmm_tl_idx[to];
            const int jo = no[0] + no[1] + no[2];
            const int cols = (jo + 1) * (jo + 2) / 2;
            const double* R = fmm_reduce_val + fmm_reduce_off[jo] + (size_t)(to - jo * jo) * cols;
            for (int ti = 0; ti < nc; ++ti) {
                const unsigned char* ni = fmm_tl_idx[ti];
                const int ci = pos_sym(ni[0], ni[1], ni[2]);
                // M2M: reduce o shift o embed
                double w = 0.0;
                for (int s = 0; s < cols; ++s) w += R[s] * Sm[(size_t)(ns_of(jo - 1) + s) * ns + ci];
                Wc[(size_t)to * nc + ti] = w;
                // L2L: keep row o shift o expand
                const int ji = ni[0] + ni[1] + ni[2];
                const int ro = pos_sym(no[0], no[1], no[2]);
                const int rcols = (ji + 1) * (ji + 2) / 2;
                double v = 0.0;
                for (int s = 0; s < rcols; ++s) {
                    const double* Ex = fmm_expand_val + fmm_expand_off[ji] + (size_t)s * (2 * ji + 1);
                    v += Vs[(size_t)ro * ns + ns_of(ji - 1) + s] * Ex[ti - ji * ji];
                }
                Vc[(size_t)to * nc + ti] = v;
            }
        }
    }
}

int fmm_create(const fmm_config* cfg, fmm_plan** out) {
    fmm_plan* pl = nullptr;
    if (!out) FAIL(FMM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!cfg) FAIL(FMM_ERR_ARG, "cfg is NULL");
    if (cfg->p < 0 || cfg->p > FMM_PMAX) FAIL(FMM_ERR_ARG, "p=%d outside 0..%d", cfg->p, FMM_PMAX);
    if (cfg->basis != 0 && cfg->basis != 1 && cfg->basis != FMM_BASIS_TG)
        FAIL(FMM_ERR_ARG, "unknown basis %d", cfg->basis);
    if (cfg->basis == FMM_BASIS_TG && (cfg->adaptive || cfg->prec != FMM_FP64))
        FAIL(FMM_ERR_UNSUPPORTED, "FMM_BASIS_TG needs a uniform octree and FMM_FP64");
    if (cfg->prec < FMM_FP64 || cfg->prec > FMM_GEMM_BF16X3) FAIL(FMM_ERR_ARG, "unknown precision %d", cfg->prec);
    if (cfg->adaptive) {
        if (cfg->max_leaf < 1) FAIL(FMM_ERR_ARG, "max_leaf=%d must be >= 1", cfg->max_leaf);
        if (!(cfg->theta >= 0.0 && cfg->theta <= 1.0)) FAIL(FMM_ERR_ARG, "theta outside [0, 1]");
        if (cfg->prec != FMM_FP64 && cfg->prec != FMM_FP32)
            FAIL(FMM_ERR_UNSUPPORTED, "adaptive trees support FMM_FP64 and FMM_FP32");
    }
    if (cfg->ap) {
        if (!cfg->adaptive || cfg->basis != FMM_BASIS_TRACELESS || cfg->prec != FMM_FP64 || cfg->learned_p)
            FAIL(FMM_ERR_UNSUPPORTED, "the AP variant needs an adaptive tree, FMM_BASIS_TRACELESS and FMM_FP64");
    }
    if (cfg->binary_tree) {
        if (!cfg->adaptive || cfg->prec != FMM_FP64 || cfg->ap || cfg->learned_p)
            FAIL(FMM_ERR_UNSUPPORTED, "the binary tree needs an adaptive plan in FMM_FP64, without ap or learned_p");
    }
    if (cfg->learned_p) {
        if (!cfg->adaptive) FAIL(FMM_ERR_UNSUPPORTED, "learned_p needs an adaptive tree");
        if (cfg->basis != FMM_BASIS_SYM) FAIL(FMM_ERR_UNSUPPORTED, "learned_p needs FMM_BASIS_SYM");
        if (cfg->p < 4) FAIL(FMM_ERR_ARG, "learned_p needs p >= 4 (the features read ranks 1..4)");
        if (!(cfg->target_rel_err > 0.0)) FAIL(FMM_ERR_ARG, "learned_p needs target_rel_err > 0");
    }
    if (cfg->depth < 0 || cfg->depth > 9) FAIL(FMM_ERR_ARG, "depth=%d outside 0..9", cfg->depth);
    if ((cfg->prec == FMM_GEMM_BF16X3 || cfg->prec == FMM_GEMM_TF32X3) && !tc_supported(cfg->p, cfg->basis))
        FAIL(FMM_ERR_UNSUPPORTED, "the tensor-core form needs the traceless basis and 1 <= p <= 8");
    pl = new fmm_plan();
    pl->cfg = *cfg;
    if (cfg->adaptive) {
        pl->ad = new AdState();
        pl->ad->ap = cfg->ap ? 1 : 0;
        pl->ad->binary = cfg->binary_tree ? 1 : 0;
        pl->depth = 0;
    }
    pl->depth = cfg->depth;
    pl->nleaf = (int64_t)1 << (3 * cfg->depth);
    // storage per coefficient row: the TG basis keeps symmetric multipoles and
    // traceless locals (a prefix of the rows of the same arrays)
    pl->nc = ncoef_of(cfg->p, cfg->basis == FMM_BASIS_TG ? 0 : cfg->basis);
    pl->ns = ns_of(cfg->p);
    int dev;
    if (int rc = tables_for_current(pl, &dev)) { fmm_destroy(pl); return rc; }
    pl->dev = dev;
    cudaDeviceGetAttribute(&pl->sms, cudaDevAttrMultiProcessorCount, dev);
    if (cfg->adaptive) {
        if (cfg->learned_p &&
            (cudaMalloc(&pl->derr, sizeof(int)) != cudaSuccess || cudaMemset(pl->derr, 0, sizeof(int)) != cudaSuccess)) {
            fmm_destroy(pl);
            return fail_plan(nullptr, FMM_ERR_OOM, "allocating the device error word failed");
        }
        *out = pl;
        return FMM_OK;
    }
    std::vector<double> W, V;
    build_translation(cfg->p, bM(pl), W, V);
    if (cfg->basis == FMM_BASIS_TG) {
        std::vector<double> W1;
        build_translation(cfg->p, 1, W1, V);   // L2L on traceless locals
    }
    const size_t mb = W.size() * sizeof(double), vb = V.size() * sizeof(double);
    if (cudaMalloc(&pl->W, mb) != cudaSuccess || cudaMalloc(&pl->V, vb) != cudaSuccess ||
        cudaMalloc(&pl->Dtab, (size_t)343 * pl->ns * sizeof(double)) != cudaSuccess) {
        fmm_destroy(pl);
        return fail_plan(nullptr, FMM_ERR_OOM, "allocating operator matrices failed");
    }
    std::vector<double> offs(3 * 343);
    for (int o = 0; o < 343; ++o) {
        const int rx = o % 7 - 3, ry = (o / 7) % 7 - 3, rz = o / 49 - 3;
        const bool near = rx >= -1 && rx <= 1 && ry >= -1 && ry <= 1 && rz >= -1 && rz <= 1;
        offs[3 * o] = near ? 10.0 : rx;  // adjacent offsets are never used; keep them finite
        offs[3 * o + 1] = near ? 10.0 : ry;
        offs[3 * o + 2] = near ? 10.0 : rz;
    }
    double* doffs = nullptr;
    bool ok = cudaMemcpy(pl->W, W.data(), mb, cudaMemcpyHostToDevice) == cudaSuccess &&
              cudaMemcpy(pl->V, V.data(), vb, cudaMemcpyHostToDevice) == cudaSuccess &&
              cudaMalloc(&doffs, offs.size() * sizeof(double)) == cudaSuccess &&
              cudaMemcpy(doffs, offs.data(), offs.size() * sizeof(double), cudaMemcpyHostToDevice) == cudaSuccess;
    if (ok) {
        k_dtab[cfg->p](343, doffs, pl->Dtab, 0);
        count_launch();
        ok = cudaDeviceSynchronize() == cudaSuccess;
    }
    cudaFree(doffs);
    if (ok && cfg->prec != FMM_FP64 && shift32_supported(cfg->p, cfg->basis)) {
        // FP32 shift matrices packed row by row: M2M row n keeps the columns of
        // rank <= |n| (a prefix), L2L row n those of rank >= |n| (a suffix)
        const int nc = pl->nc;
        auto pre = [&](int k) { return k < 0 ? 0 : (cfg->basis ? (k + 1) * (k + 1) : ns_of(k)); };
        std::vector<float> w32, v32;
        for (int c = 0; c < 8; ++c) {
            for (int r = 0; r < nc; ++r) {
                const unsigned char* n = cfg->basis ? fmm_tl_idx[r] : fmm_sym_idx[r];
                const int rk = n[0] + n[1] + n[2];
                for (int k = 0; k < pre(rk); ++k) w32.push_back((float)W[((size_t)c * nc + r) * nc + k]);
            }
            for (int r = 0; r < nc; ++r) {
                const unsigned char* n = cfg->basis ? fmm_tl_idx[r] : fmm_sym_idx[r];
                const int rk = n[0] + n[1] + n[2];
                for (int k = pre(rk - 1); k < nc; ++k) v32.push_back((float)V[((size_t)c * nc + r) * nc + k]);
            }
        }
        ok = cudaMalloc(&pl->W32, w32.size() * 4) == cudaSuccess && cudaMalloc(&pl->V32, v32.size() * 4) == cudaSuccess &&
             cudaMemcpy(pl->W32, w32.data(), w32.size() * 4, cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(pl->V32, v32.data(), v32.size() * 4, cudaMemcpyHostToDevice) == cudaSuccess &&
             (cfg->adaptive || cfg->depth < 3 ||
              cudaMalloc(&pl->part32, (size_t)8 * nc * ((size_t)1 << (3 * (cfg->depth - 1))) * 4) == cudaSuccess);
    }
    if (ok && is_tc(cfg->prec)) {
        const int tf = cfg->prec == FMM_GEMM_TF32X3;
        ok = cudaMalloc(&pl->Kbf, tc_mat_bytes(tf)) == cudaSuccess && cudaMalloc(&pl->derr, sizeof(int)) == cudaSuccess &&
             cudaMemset(pl->derr, 0, sizeof(int)) == cudaSuccess &&
             (tf || cudaMalloc(&pl->Kgen, tg_b_bytes()) == cudaSuccess) &&
             tc_set_shape(pl, 0, tc_default_cw(tf), 0) == 0 && cudaDeviceSynchronize() == cudaSuccess;
        if (ok && cfg->autotune) {
            // a shape measured earlier for this GPU, order, basis, form and depth
            int k = 0, cw = 0, ni = 0;
            const std::string path = tc_cache_path();
            if (!path.empty() && tune_cache_get(path.c_str(), tc_cache_key(pl).c_str(), &k, &cw, &ni, nullptr) == 1 &&
                tc_shape_valid(tf, k, cw)) {
                ok = tc_set_shape(pl, k, cw, 0) == 0 && cudaDeviceSynchronize() == cudaSuccess;
                pl->tc_source = 2;
            }
        }
    }
    if (ok) {
        // packed per-offset matrices of the grouped M2L: FP32 (FP32 form and
        // the small levels of the tensor-core forms) or FP64 (FP64 form)
        const bool f64 = cfg->prec == FMM_FP64;
        pl->kst = grouped_kstride(cfg->p, cfg->basis);
        const int cap = pl->kst;
        std::vector<unsigned char> ent((size_t)6 * cap);
        unsigned char* dent = nullptr;
        ok = grouped_entries(cfg->p, cfg->basis, ent.data(), cap) >= 0 &&
             cudaMalloc(&dent, ent.size()) == cudaSuccess &&
             cudaMemcpy(dent, ent.data(), ent.size(), cudaMemcpyHostToDevice) == cudaSuccess &&
             (f64 ? cudaMalloc(&pl->K64, (size_t)343 * pl->kst * sizeof(double))
                  : cudaMalloc(&pl->K32, (size_t)343 * pl->kst * sizeof(float))) == cudaSuccess;
        if (ok && f64) {
            for (int l = 2; l <= cfg->depth; ++l) {
                const int64_t e = m2l_grp64_part_elems(cfg->p, cfg->basis, l);
                if (e > pl->part64_cap) pl->part64_cap = e;
            }
            ok = pl->part64_cap == 0 || cudaMalloc(&pl->part64, (size_t)pl->part64_cap * sizeof(double)) == cudaSuccess;
        }
        if (ok) {
            if (f64)
                launch_build_ktab64(cfg->p, cfg->basis, pl->kst, dent, pl->Dtab, pl->K64, 0);
            else
                launch_build_ktab(cfg->p, cfg->basis, pl->kst, dent, pl->Dtab, pl->K32, 0);
            ok = cudaDeviceSynchronize() == cudaSuccess;
        }
        cudaFree(dent);
    }
    if (!ok) {
        fmm_destroy(pl);
        return fail_plan(nullptr, FMM_ERR_CUDA, "plan set-up failed: %s", cudaGetErrorString(cudaGetLastError()));
    }
    *out = pl;
    return FMM_OK;
}

void fmm_destroy(fmm_plan* pl) {
    if (!pl) return;
    ad_free(pl->ad);
    free_tree(pl);
    cudaFree(pl->W); cudaFree(pl->V); cudaFree(pl->Dtab); cudaFree(pl->stage); cudaFree(pl->K32); cudaFree(pl->K64);
    cudaFree(pl->part64);
    if (pl->ugexec) cudaGraphExecDestroy(pl->ugexec);
    cudaFree(pl->Kbf); cudaFree(pl->Kgen); cudaFree(pl->derr); cudaFree(pl->W32); cudaFree(pl->V32); cudaFree(pl->mlp_dev);
    cudaFree(pl->part32);
    cudaFree(pl->Mrest); cudaFree(pl->Krest); cudaFree(pl->Rpart);
    delete pl;
}

int fmm_build_tree(fmm_plan* pl, int64_t n, const double* x, const double* y, const double* z, const double* q,
                   void* stream) {
    if (!pl) return fail_plan(nullptr, FMM_ERR_ARG, "plan is NULL");
    if (n < 0 || n > (int64_t)0x7fffffff) FAIL(FMM_ERR_ARG, "n=%lld outside 0..2^31-1", (long long)n);
    if (n > 0 && (!x || !y || !z || !q)) FAIL(FMM_ERR_ARG, "null particle array");
    if (pl->ad) {
        const int rc = ad_build(pl->ad, n, x, y, z, q, pl->cfg.max_leaf, pl->cfg.theta, pl->nc,
                                pl->cfg.prec == FMM_FP64 ? 0 : 1, S(stream));
        if (rc == -3) FAIL(FMM_ERR_OOM, "allocating adaptive tree storage failed");
        if (rc) FAIL(FMM_ERR_CUDA, "adaptive tree build failed: %s", cudaGetErrorString(cudaGetLastError()));
        if (pl->cfg.learned_p) {
            const int r2 = ad_learn_prepare(pl->ad, S(stream));
            if (r2 == -3) FAIL(FMM_ERR_OOM, "allocating learned-order storage failed");
            if (r2) FAIL(FMM_ERR_CUDA, "learned-order set-up failed: %s", cudaGetErrorString(cudaGetLastError()));
            if (pl->ad->orders_fixed && pl->ad->n_orders != pl->ad->nm2l) pl->ad->orders_fixed = false;
            pl->ad->orders_chosen = false;
        }
        pl->n = n;
        pl->built = true;
        return FMM_OK;
    }
    if (n != pl->n) {
        free_tree(pl);
        const int64_t nn = n > 0 ? n : 1;
        const int nc = pl->nc;
        int64_t tot = 0;
        for (int l = 0; l <= pl->depth; ++l) { pl->lvl_off[l] = tot; tot += (int64_t)nc << (3 * l); }
        pl->scratch_bytes = tree_scratch_bytes(nn, pl->nleaf);
        if (cudaMalloc(&pl->xs, nn * 8) != cudaSuccess || cudaMalloc(&pl->ys, nn * 8) != cudaSuccess ||
            cudaMalloc(&pl->zs, nn * 8) != cudaSuccess || cudaMalloc(&pl->qs, nn * 8) != cudaSuccess ||
            cudaMalloc(&pl->perm, nn * 4) != cudaSuccess ||
            cudaMalloc(&pl->start, (pl->nleaf + 1) * 4) != cudaSuccess ||
            cudaMalloc(&pl->scratch, pl->scratch_bytes) != cudaSuccess ||
            cudaMalloc(&pl->Mbuf, tot * 8) != cudaSuccess || cudaMalloc(&pl->Lbuf, tot * 8) != cudaSuccess ||
            (pl->cfg.prec != FMM_FP64 && cudaMalloc(&pl->M32, tot * 4) != cudaSuccess) ||
            (pl->cfg.prec != FMM_FP64 && cudaMalloc(&pl->pos32, nn * 16) != cudaSuccess) ||
            (pl->cfg.prec != FMM_FP64 && cudaMalloc(&pl->pos32c, nn * 16) != cudaSuccess) ||
            (pl->cfg.prec != FMM_FP64 && bM(pl) == FMM_BASIS_TRACELESS &&
             cudaMalloc(&pl->msym32, (size_t)pl->nleaf * ((ns_of(pl->cfg.p) + 3) / 4 * 4) * 4) != cudaSuccess) ||
            (pl->cfg.prec != FMM_FP64 && pl->V32 && cudaMalloc(&pl->L32, tot * 4) != cudaSuccess)) {
            cudaGetLastError();
            free_tree(pl);
            FAIL(FMM_ERR_OOM, "allocating tree storage for n=%lld failed", (long long)n);
        }
        if (pl->L32) {
            pl->lpart_cap = 0;
            for (int l = 2; l <= pl->depth; ++l) {
                const int64_t e = m2l_grpf_part_elems(pl->cfg.p, pl->cfg.basis, l);
                if (e > pl->lpart_cap) pl->lpart_cap = e;
            }
        }
        if (pl->lpart_cap > 0 && cudaMalloc(&pl->lpart, (size_t)pl->lpart_cap * 4) != cudaSuccess) {
            cudaGetLastError();
            free_tree(pl);
            FAIL(FMM_ERR_OOM, "allocating tree storage for n=%lld failed", (long long)n);
        }
        if (is_tc(pl->cfg.prec)) {
            const int tf = pl->cfg.prec == FMM_GEMM_TF32X3, es = tc_elem_bytes(tf);
            int64_t tb = 0;
            for (int l = 0; l <= pl->depth; ++l) {
                pl->mbf_off[l] = tb;
                if (l >= tc_first_level()) tb += 2 * (int64_t)tc_m_elems(l);
            }
            pl->maps.assign((size_t)(pl->depth + 1) * tc_maps_bytes() + 64, 0);
            if (tb > 0 && cudaMalloc(&pl->Mbf, tb * es) != cudaSuccess) {
                cudaGetLastError();
                free_tree(pl);
                FAIL(FMM_ERR_OOM, "allocating tensor-core operands failed");
            }
            for (int l = tc_first_level(); l <= pl->depth; ++l) {
                char* hi = (char*)pl->Mbf + pl->mbf_off[l] * es;
                char* lo = hi + tc_m_elems(l) * es;
                if (tc_encode_maps(l, tf, hi, lo, tc_maps_at(pl, l)) != 0) {
                    free_tree(pl);
                    FAIL(FMM_ERR_CUDA, "encoding TMA tensor maps failed");
                }
            }
        }
        pl->n = n;
    }
    if (launch_uniform_tree(n, pl->depth, x, y, z, q, pl->xs, pl->ys, pl->zs, pl->qs, pl->perm, pl->start,
                            pl->scratch, S(stream), pl->pos32, pl->pos32c) != 0)
        FAIL(FMM_ERR_CUDA, "tree build failed: %s", cudaGetErrorString(cudaGetLastError()));
    CKLAUNCH();
    pl->built = true;
    return FMM_OK;
}

static double* Mlev(fmm_plan* pl, int l) { return pl->Mbuf + pl->lvl_off[l]; }
static double* Llev(fmm_plan* pl, int l) { return pl->Lbuf + pl->lvl_off[l]; }

#define NEED_TREE() \
    if (!pl) return fail_plan(nullptr, FMM_ERR_ARG, "plan is NULL"); \
    if (!pl->built) FAIL(FMM_ERR_STATE, "fmm_build_tree has not been called")

int fmm_p2m(fmm_plan* pl, void* stream) {
    NEED_TREE();
    if (pl->ad) { ad_run_p2m(pl->ad, pl->cfg.prec == FMM_FP64 ? 0 : 1, pl->cfg.p, pl->cfg.basis, g_tab[pl->dev], S(stream)); CKLAUNCH(); return FMM_OK; }
    const int d = pl->depth;
    launch_p2m_leaf(pl->cfg.prec == FMM_FP64 ? 0 : 1, pl->cfg.p, bM(pl), d, pl->nleaf, pl->start, pl->xs,
                    pl->ys, pl->zs, pl->qs, Mlev(pl, d), g_tab[pl->dev], S(stream), pl->pos32, pl->msym32,
                    m32_current(pl) ? pl->M32 + pl->lvl_off[d] : nullptr);
    CKLAUNCH();
    return FMM_OK;
}

int fmm_m2m(fmm_plan* pl, void* stream) {
    NEED_TREE();
    if (pl->ad) {
        ad_run_m2m(pl->ad, pl->cfg.prec == FMM_FP64 ? 0 : 1, pl->cfg.p, pl->cfg.basis, g_tab[pl->dev], S(stream));
        // AP: about the centre of mass the dipole vanishes; it is set to exactly 0
        if (pl->ad->ap && pl->cfg.p >= 1) ad_zero_dipole(pl->ad->nn, pl->nc, pl->ad->M, S(stream));
        CKLAUNCH();
        return FMM_OK;
    }
    if (pl->W32) {
        for (int l = pl->depth - 1; l >= 2; --l) {
            const bool c32 = m32_current(pl);
            const int nl = launch_shift32(pl->cfg.p, pl->cfg.basis, 1, l, pl->W32, Mlev(pl, l + 1),
                                          (int64_t)1 << (3 * (l + 1)), Mlev(pl, l), (int64_t)1 << (3 * l), S(stream),
                                          pl->part32, c32 ? pl->M32 + pl->lvl_off[l + 1] : nullptr,
                                          c32 ? pl->M32 + pl->lvl_off[l] : nullptr);
            for (int k = 0; k < nl; ++k) count_launch();
        }
        CKLAUNCH();
        return FMM_OK;
    }
    for (int l = pl->depth - 1; l >= 2; --l)
        launch_m2m_level(pl->cfg.p, bM(pl), l, pl->W, Mlev(pl, l + 1), (int64_t)1 << (3 * (l + 1)),
                         Mlev(pl, l), (int64_t)1 << (3 * l), S(stream));
    CKLAUNCH();
    return FMM_OK;
}

static int m2l_uniform(fmm_plan* pl, int lo, int hi, void* stream);

int fmm_m2l(fmm_plan* pl, void* stream) {
    NEED_TREE();
    if (pl->ad) {
        if (pl->cfg.learned_p) {
            if (!pl->ad->orders_fixed && !pl->mlp_set)
                FAIL(FMM_ERR_STATE, "learned_p plan without a model (fmm_set_mlp) or pair orders (fmm_set_pair_orders)");
            const float thr = (float)log10(pl->cfg.target_rel_err) + pl->log10_kappa;
            if (ad_run_m2l_orders(pl->ad, pl->cfg.p, pl->cfg.basis, pl->cfg.prec == FMM_FP64 ? 0 : 1, pl->sms,
                                  pl->mlp_dev, thr, pl->derr, S(stream)))
                FAIL(FMM_ERR_CUDA, "per-order M2L failed: %s", cudaGetErrorString(cudaGetLastError()));
            CKLAUNCH();
            return FMM_OK;
        }
        if (ad_run_m2l(pl->ad, pl->cfg.p, pl->cfg.basis, pl->cfg.prec == FMM_FP64 ? 0 : 1, pl->sms, S(stream)))
            FAIL(FMM_ERR_UNSUPPORTED, "no list M2L kernel for this order and basis");
        CKLAUNCH();
        return FMM_OK;
    }
    return m2l_uniform(pl, 2, pl->depth, stream);
}

// M2L of the uniform levels lo..hi (clamped to 2..depth) of any form.
static int m2l_uniform(fmm_plan* pl, int lo, int hi, void* stream) {
    if (lo < 2) lo = 2;
    if (hi > pl->depth) hi = pl->depth;
    if (lo > hi) return FMM_OK;
    if (is_tc(pl->cfg.prec)) {
        const int tf = pl->cfg.prec == FMM_GEMM_TF32X3, es = tc_elem_bytes(tf);
        // levels below the first tensor-core level (class grids smaller than one
        // 8 x 16 x 1 column) on the FP32 grouped kernel
        const int lt = hi < tc_first_level() - 1 ? hi : tc_first_level() - 1;
        if (lo <= lt) {
            const int64_t b = pl->lvl_off[lo], e = pl->lvl_off[lt] + ((int64_t)pl->nc << (3 * lt));
            if (!m32_current(pl)) launch_to_f32(e - b, pl->Mbuf + b, pl->M32 + b, S(stream));
            for (int l = lo; l <= lt; ++l) {
                const int parts =
                    pl->L32 ? launch_m2l_grpf(pl->cfg.p, pl->cfg.basis, l, pl->M32 + pl->lvl_off[l], L32lev(pl, l),
                                              pl->K32, (int64_t)1 << (3 * l), S(stream), pl->lpart, pl->lpart_cap)
                            : launch_m2l_grp(pl->cfg.p, pl->cfg.basis, l, pl->M32 + pl->lvl_off[l], Llev(pl, l),
                                             pl->K32, (int64_t)1 << (3 * l), S(stream));
                for (int k = 0; k < parts; ++k) count_launch();
            }
        }
        const int l0 = lo > tc_first_level() ? lo : tc_first_level();
        if (l0 <= hi && pl->cfg.autotune && pl->tc_source == 0 && tc_autotune(pl, pl->depth, S(stream)) != 0)
            FAIL(FMM_ERR_CUDA, "tensor-core autotuning failed: %s", cudaGetErrorString(cudaGetLastError()));
        (void)es;
        for (int l = l0; l <= hi; ++l)
            if (tc_level_call(pl, l, S(stream)) != 0)
                FAIL(FMM_ERR_CUDA, "tensor-core M2L launch failed: %s", cudaGetErrorString(cudaGetLastError()));
        CKLAUNCH();
        return FMM_OK;
    }
    if (pl->cfg.prec == FMM_FP32) {
        const int64_t b = pl->lvl_off[lo], e = pl->lvl_off[hi] + ((int64_t)pl->nc << (3 * hi));
        if (!m32_current(pl)) launch_to_f32(e - b, pl->Mbuf + b, pl->M32 + b, S(stream));
        for (int l = lo; l <= hi; ++l) {
            const int parts =
                pl->L32 ? launch_m2l_grpf(pl->cfg.p, pl->cfg.basis, l, pl->M32 + pl->lvl_off[l], L32lev(pl, l),
                                          pl->K32, (int64_t)1 << (3 * l), S(stream), pl->lpart, pl->lpart_cap)
                        : launch_m2l_grp(pl->cfg.p, pl->cfg.basis, l, pl->M32 + pl->lvl_off[l], Llev(pl, l),
                                         pl->K32, (int64_t)1 << (3 * l), S(stream));
            for (int k = 0; k < parts; ++k) count_launch();
        }
        CKLAUNCH();
        return FMM_OK;
    }
    for (int l = lo; l <= hi; ++l) {
        const int parts = launch_m2l_grp64(pl->cfg.p, pl->cfg.basis, l, Mlev(pl, l), Llev(pl, l), pl->K64,
                                           (int64_t)1 << (3 * l), S(stream), pl->part64, pl->part64_cap);
        for (int k = 0; k < parts; ++k) count_launch();
    }
    CKLAUNCH();
    return FMM_OK;
}

int fmm_m2l_levels(fmm_plan* pl, int lmin, int lmax, void* stream) {
    NEED_TREE();
    if (pl->ad) FAIL(FMM_ERR_UNSUPPORTED, "fmm_m2l_levels needs a uniform octree (adaptive plans use fmm_m2l)");
    if (lmin > lmax) FAIL(FMM_ERR_ARG, "lmin=%d > lmax=%d", lmin, lmax);
    return m2l_uniform(pl, lmin, lmax, stream);
}

int fmm_l2l(fmm_plan* pl, void* stream) {
    NEED_TREE();
    if (pl->ad) { ad_run_l2l(pl->ad, pl->cfg.prec == FMM_FP64 ? 0 : 1, pl->cfg.p, pl->cfg.basis, g_tab[pl->dev], S(stream)); CKLAUNCH(); return FMM_OK; }
    if (pl->V32) {
        for (int l = 2; l < pl->depth; ++l) {
            const int nl = pl->L32 ? launch_l2l32f(pl->cfg.p, pl->cfg.basis, l, pl->V32, L32lev(pl, l),
                                                   (int64_t)1 << (3 * l), L32lev(pl, l + 1),
                                                   (int64_t)1 << (3 * (l + 1)), S(stream))
                                   : launch_shift32(pl->cfg.p, pl->cfg.basis, 0, l, pl->V32, Llev(pl, l),
                                                    (int64_t)1 << (3 * l), Llev(pl, l + 1),
                                                    (int64_t)1 << (3 * (l + 1)), S(stream));
            for (int k = 0; k < nl; ++k) count_launch();
        }
        CKLAUNCH();
        return FMM_OK;
    }
    for (int l = 2; l < pl->depth; ++l)
        launch_l2l_level(pl->cfg.p, bL(pl), l, pl->V, Llev(pl, l), (int64_t)1 << (3 * l), Llev(pl, l + 1),
                         (int64_t)1 << (3 * (l + 1)), S(stream));
    CKLAUNCH();
    return FMM_OK;
}

int fmm_l2p(fmm_plan* pl, double* pot, double* ax, double* ay, double* az, void* stream) {
    NEED_TREE();
    if (pl->n > 0 && (!pot || !ax || !ay || !az)) FAIL(FMM_ERR_ARG, "null output array");
    if (pl->ad) {
        ad_run_l2p(pl->ad, pl->cfg.prec == FMM_FP64 ? 0 : 1, pl->cfg.p, pl->cfg.basis, g_tab[pl->dev], pot, ax, ay, az, S(stream));
        if (pl->ad->ap) launch_fill(pl->n, pot, 0.0, S(stream));   // AP: the gradient only
        CKLAUNCH();
        return FMM_OK;
    }
    if (pl->depth >= 2)
        launch_l2p_leaf2(pl->cfg.prec == FMM_FP64 ? 0 : 1, pl->cfg.p, bL(pl), pl->depth, pl->nleaf,
                         pl->start, pl->xs, pl->ys, pl->zs, pl->perm, Llev(pl, pl->depth), g_tab[pl->dev], pot, ax,
                         ay, az, S(stream), pl->pos32, L32lev(pl, pl->depth));
    else
        launch_zero4(pl->n, pot, ax, ay, az, S(stream));
    CKLAUNCH();
    return FMM_OK;
}

int fmm_p2p(fmm_plan* pl, double* pot, double* ax, double* ay, double* az, void* stream) {
    NEED_TREE();
    if (pl->n > 0 && (!pot || !ax || !ay || !az)) FAIL(FMM_ERR_ARG, "null output array");
    if (pl->ad) {
        ad_run_p2p(pl->ad, pl->cfg.prec == FMM_FP64 ? 0 : 1, pl->sms, pot, ax, ay, az, S(stream));
        if (pl->ad->ap) launch_fill(pl->n, pot, 0.0, S(stream));   // AP: the gradient only
        CKLAUNCH();
        return FMM_OK;
    }
    if (pl->pos32)
        launch_p2p32(pl->depth, pl->nleaf, pl->start, pl->pos32, pl->perm, pot, ax, ay, az, S(stream));
    else
        launch_p2p_leaf2(0, pl->depth, pl->nleaf, pl->start, pl->xs, pl->ys, pl->zs, pl->qs, pl->perm, pot, ax, ay,
                         az, S(stream));
    CKLAUNCH();
    return FMM_OK;
}

int fmm_l2p_p2p(fmm_plan* pl, double* pot, double* ax, double* ay, double* az, void* stream) {
    NEED_TREE();
    if (pl->n > 0 && (!pot || !ax || !ay || !az)) FAIL(FMM_ERR_ARG, "null output array");
    if (!pl->ad && pl->pos32 && pl->depth >= 2) {
        // the FP32 uniform form: far and near field in one kernel
        launch_l2p_p2p32(pl->cfg.p, bL(pl), pl->depth, pl->nleaf, pl->start, pl->pos32, pl->perm, Llev(pl, pl->depth),
                         g_tab[pl->dev], pot, ax, ay, az, S(stream), L32lev(pl, pl->depth));
        CKLAUNCH();
        return FMM_OK;
    }
    int rc;
    if ((rc = fmm_l2p(pl, pot, ax, ay, az, stream))) return rc;
    return fmm_p2p(pl, pot, ax, ay, az, stream);
}

int fmm_evaluate(fmm_plan* pl, int64_t n, const double* x, const double* y, const double* z, const double* q,
                 double* pot, double* ax, double* ay, double* az, void* stream) {
    if (!pl) return fail_plan(nullptr, FMM_ERR_ARG, "plan is NULL");
    if (n > 0 && (!pot || !ax || !ay || !az)) FAIL(FMM_ERR_ARG, "null output array");
    int rc;
    if (!pl->ad && pl->cfg.use_graph && stream && n > 0 && pl->built && n == pl->n &&
        !(is_tc(pl->cfg.prec) && pl->cfg.autotune && pl->tc_source == 0)) {
        // uniform plan: the whole step (tree and operators) is captured once
        // into a CUDA graph and replayed while the particle count, the
        // arrays and the tensor-core kernel shape stay the same (the first
        // evaluation, which allocates and autotunes, runs eagerly)
        const void* key[11] = {x, y, z, q, pot, ax, ay, az, (const void*)(intptr_t)n,
                               (const void*)(intptr_t)pl->tc_kern, (const void*)(intptr_t)pl->tc_cw};
        if (!pl->ugexec || memcmp(key, pl->ugkey, sizeof key) != 0) {
            if (pl->ugexec) { cudaGraphExecDestroy(pl->ugexec); pl->ugexec = nullptr; }
            cudaGraph_t g = nullptr;
            CK(cudaStreamBeginCapture(S(stream), cudaStreamCaptureModeThreadLocal));
            const int r1 = fmm_build_tree(pl, n, x, y, z, q, stream) | fmm_p2m(pl, stream) | fmm_m2m(pl, stream) |
                           fmm_m2l(pl, stream) | fmm_l2l(pl, stream) | fmm_l2p_p2p(pl, pot, ax, ay, az, stream);
            const cudaError_t ce = cudaStreamEndCapture(S(stream), &g);
            if (r1 || ce != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                FAIL(FMM_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(ce));
            }
            const cudaError_t ie = cudaGraphInstantiate(&pl->ugexec, g, 0);
            cudaGraphDestroy(g);
            if (ie != cudaSuccess) FAIL(FMM_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(ie));
            memcpy(pl->ugkey, key, sizeof key);
        }
        CK(cudaGraphLaunch(pl->ugexec, S(stream)));
        return FMM_OK;
    }
    if ((rc = fmm_build_tree(pl, n, x, y, z, q, stream))) return rc;
    if (pl->ad && pl->cfg.use_graph && stream && n > 0 &&
        (pl->ad->m2l_blocks > 0 || (pl->cfg.learned_p && (pl->mlp_set || pl->ad->orders_fixed)))) {
        // replay the captured operator sequence while the tree keeps its
        // sizes and buffers; capture it again otherwise
        AdState* A = pl->ad;
        const void* key[8] = {A->M, pot, ax, (const void*)(intptr_t)A->gen, (const void*)(intptr_t)A->nn,
                              (const void*)(intptr_t)(((int64_t)A->ntarg << 32) ^ A->nleaf ^ (A->nm2l * 7919LL)),
                              (const void*)(intptr_t)((A->orders_fixed ? 1 : 0) | (pl->mlp_set ? 2 : 0)),
                              (const void*)(intptr_t)A->m2l_blocks};
        if (!A->gexec || memcmp(key, A->graph_key, sizeof key) != 0) {
            if (A->gexec) { cudaGraphExecDestroy(A->gexec); A->gexec = nullptr; }
            cudaGraph_t g = nullptr;
            CK(cudaStreamBeginCapture(S(stream), cudaStreamCaptureModeThreadLocal));
            const int r1 = fmm_p2m(pl, stream) | fmm_m2m(pl, stream) | fmm_m2l(pl, stream) | fmm_l2l(pl, stream) |
                           fmm_l2p(pl, pot, ax, ay, az, stream) | fmm_p2p(pl, pot, ax, ay, az, stream);
            const cudaError_t ce = cudaStreamEndCapture(S(stream), &g);
            if (r1 || ce != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                FAIL(FMM_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(ce));
            }
            const cudaError_t ie = cudaGraphInstantiate(&A->gexec, g, 0);
            cudaGraphDestroy(g);
            if (ie != cudaSuccess) FAIL(FMM_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(ie));
            memcpy(A->graph_key, key, sizeof key);
        }
        CK(cudaGraphLaunch(A->gexec, S(stream)));
        return FMM_OK;
    }
    if ((rc = fmm_p2m(pl, stream))) return rc;
    if ((rc = fmm_m2m(pl, stream))) return rc;
    if ((rc = fmm_m2l(pl, stream))) return rc;
    if ((rc = fmm_l2l(pl, stream))) return rc;
    return fmm_l2p_p2p(pl, pot, ax, ay, az, stream);
}

int fmm_evaluate_dipoles(fmm_plan* pl, int64_t n, const double* x, const double* y, const double* z, const double* q,
                         const double* px, const double* py, const double* pz, double* pot, double* ax, double* ay,
                         double* az, void* stream) {
    if (!pl) return fail_plan(nullptr, FMM_ERR_ARG, "plan is NULL");
    if (pl->ad || pl->cfg.prec != FMM_FP64)
        FAIL(FMM_ERR_UNSUPPORTED, "point dipoles need a uniform octree and FMM_FP64");
    if (n > 0 && (!px || !py || !pz || !pot || !ax || !ay || !az)) FAIL(FMM_ERR_ARG, "null array");
    int rc;
    if ((rc = fmm_build_tree(pl, n, x, y, z, q, stream))) return rc;
    cudaStream_t s = S(stream);
    if (!pl->dip && cudaMalloc(&pl->dip, (size_t)3 * (n > 0 ? n : 1) * sizeof(double)) != cudaSuccess) {
        pl->dip = nullptr;
        cudaGetLastError();
        FAIL(FMM_ERR_OOM, "allocating the sorted dipole moments failed");
    }
    double *pxs = pl->dip, *pys = pl->dip + n, *pzs = pl->dip + 2 * n;
    launch_gather3(n, pl->perm, px, py, pz, pxs, pys, pzs, s);
    const int d = pl->depth;
    // P2M of charges and dipoles (the general P2M kernel writes the plan's
    // scaled leaf multipoles; traceless: the reduced representative)
    launch_p2m(pl->cfg.p, bM(pl), 1, pl->nleaf, nullptr, pl->start, pl->xs, pl->ys, pl->zs, pl->qs, nullptr, d,
               (double)(1 << d), Mlev(pl, d), pl->nleaf, g_tab[pl->dev], s, pxs, pys, pzs);
    CKLAUNCH();
    if ((rc = fmm_m2m(pl, stream))) return rc;
    if ((rc = fmm_m2l(pl, stream))) return rc;
    if ((rc = fmm_l2l(pl, stream))) return rc;
    if ((rc = fmm_l2p(pl, pot, ax, ay, az, stream))) return rc;
    if ((rc = fmm_p2p(pl, pot, ax, ay, az, stream))) return rc;
    launch_p2p_dipole(d, pl->nleaf, pl->start, pl->xs, pl->ys, pl->zs, pxs, pys, pzs, pl->perm, pot, ax, ay, az, s);
    CKLAUNCH();
    return FMM_OK;
}

int fmm_evaluate_host(fmm_plan* pl, int64_t n, const double* x, const double* y, const double* z,
                      const double* q, double* pot, double* ax, double* ay, double* az, void* stream) {
    if (!pl) return fail_plan(nullptr, FMM_ERR_ARG, "plan is NULL");
    if (n < 0) FAIL(FMM_ERR_ARG, "n < 0");
    if (n > 0 && (!x || !y || !z || !q || !pot || !ax || !ay || !az)) FAIL(FMM_ERR_ARG, "null host array");
    if (n > pl->stage_n) {
        cudaFree(pl->stage);
        pl->stage = nullptr;
        pl->stage_n = 0;
        if (cudaMalloc(&pl->stage, (size_t)8 * n * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            FAIL(FMM_ERR_OOM, "allocating staging buffers failed");
        }
        pl->stage_n = n;
    }
    double* d = pl->stage;
    const size_t b = (size_t)n * sizeof(double);
    cudaStream_t s = S(stream);
    const double* in[4] = {x, y, z, q};
    double* outp[4] = {pot, ax, ay, az};
    for (int k = 0; k < 4; ++k) CK(cudaMemcpyAsync(d + (size_t)k * n, in[k], b, cudaMemcpyHostToDevice, s));
    int rc = fmm_evaluate(pl, n, d, d + n, d + 2 * n, d + 3 * n, d + 4 * n, d + 5 * n, d + 6 * n, d + 7 * n,
                          stream);
    if (rc) return rc;
    for (int k = 0; k < 4; ++k) CK(cudaMemcpyAsync(outp[k], d + (size_t)(4 + k) * n, b, cudaMemcpyDeviceToHost, s));
    return fmm_sync_status(pl, stream);
}

int fmm_sync_status(fmm_plan* pl, void* stream) {
    if (!pl) return fail_plan(nullptr, FMM_ERR_ARG, "plan is NULL");
    cudaStream_t s = S(stream);
    CK(cudaStreamSynchronize(s));
    if (!pl->derr) return FMM_OK;
    int herr = 0;
    CK(cudaMemcpy(&herr, pl->derr, sizeof(int), cudaMemcpyDeviceToHost));
    if (!herr) return FMM_OK;
    // reported once: the word is cleared for the work queued after this call
    CK(cudaMemset(pl->derr, 0, sizeof(int)));
    FAIL(FMM_ERR_TIMEOUT, "a bounded wait in a tensor-core kernel gave up (code %d); the outputs of the work "
                          "queued since the previous status check are undefined", herr);
}

int fmm_selftest_wait(int64_t spin, int arrive, void* stream) {
    fmm_plan* pl = nullptr;
    if (spin < 1) FAIL(FMM_ERR_ARG, "spin must be >= 1");
    cudaStream_t s = S(stream);
    int* derr = nullptr;
    if (cudaMalloc(&derr, sizeof(int)) != cudaSuccess) FAIL(FMM_ERR_OOM, "allocating the error word failed");
    int herr = 0;
    const bool ok = cudaMemsetAsync(derr, 0, sizeof(int), s) == cudaSuccess &&
                    wait_selftest((long)spin, arrive ? 1 : 0, derr, s) == 0 &&
                    cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, s) == cudaSuccess &&
                    cudaStreamSynchronize(s) == cudaSuccess;
    cudaFree(derr);
    if (!ok) FAIL(FMM_ERR_CUDA, "the wait self-test failed to run: %s", cudaGetErrorString(cudaGetLastError()));
    if (herr) FAIL(FMM_ERR_TIMEOUT, "the bounded wait gave up (code %d)", herr);
    return FMM_OK;
}

// ---------------------------------------------------------------------------
// learned per-pair order
// ---------------------------------------------------------------------------
static int check_blob(fmm_plan* pl, const float* blob) {
    if (!blob) FAIL(FMM_ERR_ARG, "blob is NULL");
    if (blob[0] != 6332.f || blob[1] != FMM_MLP_VERSION || blob[2] != (float)FMM_MLP_NF || blob[3] != 64.f ||
        blob[4] != (float)FMM_MLP_NOUT || blob[5] != 2.f)
        FAIL(FMM_ERR_ARG, "blob header is not {6332, 2, 12, 64, 9, 2, ...}");
    for (int f = 0; f < FMM_MLP_NF; ++f)
        if (!(blob[FMM_MLP_OFF_SD + f] > 0.f)) FAIL(FMM_ERR_ARG, "feature deviation %d is not positive", f);
    return FMM_OK;
}

static int need_pairs(fmm_plan* pl, cudaStream_t s) {
    if (!pl) return fail_plan(nullptr, FMM_ERR_ARG, "plan is NULL");
    if (!pl->ad) FAIL(FMM_ERR_ARG, "not an adaptive plan");
    if (!pl->built) FAIL(FMM_ERR_STATE, "fmm_build_tree has not been called");
    const int r = ad_learn_prepare(pl->ad, s);
    if (r == -3) FAIL(FMM_ERR_OOM, "allocating pair storage failed");
    if (r) FAIL(FMM_ERR_CUDA, "pair set-up failed: %s", cudaGetErrorString(cudaGetLastError()));
    return FMM_OK;
}

int fmm_plan_pairs(fmm_plan* pl, int32_t* tgt, int32_t* src, int64_t cap, int64_t* count) {
    if (int rc = need_pairs(pl, 0)) return rc;
    const int64_t np = pl->ad->nm2l;
    if (count) *count = np;
    if (cap < np || np == 0) return FMM_OK;
    if (!tgt || !src) FAIL(FMM_ERR_ARG, "null output array");
    CK(cudaMemcpy(tgt, pl->ad->ptgt, (size_t)np * 4, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(src, pl->ad->msrc, (size_t)np * 4, cudaMemcpyDeviceToHost));
    return FMM_OK;
}

int fmm_pair_data(fmm_plan* pl, float* feat, double* labels, void* stream) {
    if (int rc = need_pairs(pl, S(stream))) return rc;
    if (pl->cfg.basis != FMM_BASIS_SYM || pl->cfg.p < 4) FAIL(FMM_ERR_ARG, "pair data needs FMM_BASIS_SYM and p >= 4");
    if (labels && (pl->cfg.p != 10 || pl->cfg.prec != FMM_FP64))
        FAIL(FMM_ERR_ARG, "labels need p = 10 and FMM_FP64");
    if (pl->ad->nm2l > 0 && !feat && !labels) FAIL(FMM_ERR_ARG, "nothing to write");
    if (labels && pl->n > (1 << 18)) FAIL(FMM_ERR_ARG, "labels need n <= 2^18 (O(n^2) direct sum)");
    if (int rc = fmm_p2m(pl, stream)) return rc;
    if (int rc = fmm_m2m(pl, stream)) return rc;
    ad_node_features(pl->ad, S(stream));
    ad_far_estimate(pl->ad, S(stream));
    if (feat) ad_pair_features(pl->ad, feat, S(stream));
    if (labels && pl->n > 0) {
        // total forces at every particle (sorted order), FP64 direct sum
        AdState* A = pl->ad;
        double* tot = nullptr;
        if (cudaMalloc(&tot, (size_t)4 * pl->n * sizeof(double)) != cudaSuccess)
            FAIL(FMM_ERR_OOM, "allocating the label scratch failed");
        launch_direct(pl->n, A->xs, A->ys, A->zs, A->qs, pl->n, nullptr, tot, tot + pl->n, tot + 2 * pl->n,
                      tot + 3 * pl->n, S(stream));
        ad_pair_labels(A, labels, tot + pl->n, tot + 2 * pl->n, tot + 3 * pl->n, S(stream));
        const cudaError_t e = cudaStreamSynchronize(S(stream));
        cudaFree(tot);
        if (e != cudaSuccess) FAIL(FMM_ERR_CUDA, "label pass failed: %s", cudaGetErrorString(e));
    }
    CKLAUNCH();
    return FMM_OK;
}

int fmm_mlp_grad(const float* blob, int64_t n, const float* feat, const float* labels, float* loss, float* grad,
                 void* stream) {
    fmm_plan* pl = nullptr;
    if (int rc = check_blob(pl, blob)) return rc;
    if (n < 1 || n > (1 << 20)) FAIL(FMM_ERR_ARG, "n=%lld outside 1..2^20", (long long)n);
    if (!feat || !labels || !loss || !grad) FAIL(FMM_ERR_ARG, "null array");
    const int rc = mlp_grad_host(blob, n, feat, labels, loss, grad, S(stream));
    if (rc == -3) FAIL(FMM_ERR_OOM, "allocating trainer scratch failed");
    if (rc) FAIL(FMM_ERR_CUDA, "gradient pass failed: %s", cudaGetErrorString(cudaGetLastError()));
    return FMM_OK;
}

int fmm_mlp_train(float* blob, int64_t n, const float* feat, const float* labels, const int32_t* order, int epochs,
                  int batch, float lr, int fit_moments, float* loss_out, void* stream) {
    fmm_plan* pl = nullptr;
    if (!blob) FAIL(FMM_ERR_ARG, "blob is NULL");
    if (!fit_moments)
        if (int rc = check_blob(pl, blob)) return rc;
    if (n < 1 || n > (int64_t)0x7fffffff) FAIL(FMM_ERR_ARG, "n=%lld outside 1..2^31-1", (long long)n);
    if (!feat || !labels || !order) FAIL(FMM_ERR_ARG, "null array");
    if (epochs < 0 || batch < 1 || batch > (1 << 20) || !(lr > 0.f)) FAIL(FMM_ERR_ARG, "bad epochs, batch or lr");
    const int rc = mlp_train_host(blob, n, feat, labels, order, epochs, batch, lr, fit_moments, loss_out, S(stream));
    if (rc == -3) FAIL(FMM_ERR_OOM, "allocating trainer storage failed");
    if (rc) FAIL(FMM_ERR_CUDA, "training failed: %s", cudaGetErrorString(cudaGetLastError()));
    return FMM_OK;
}

int fmm_mlp_predict(const float* blob, int64_t n, const float* feat, float* pred, void* stream) {
    fmm_plan* pl = nullptr;
    if (int rc = check_blob(pl, blob)) return rc;
    if (n < 0) FAIL(FMM_ERR_ARG, "n < 0");
    if (n == 0) return FMM_OK;
    if (!feat || !pred) FAIL(FMM_ERR_ARG, "null array");
    std::vector<unsigned char> h(MLP_DEV_BYTES);
    mlp_pack_device(blob, h.data());
    unsigned char* d = nullptr;
    int* derr = nullptr;
    int dev = 0, sms = 152;
    CK(cudaGetDevice(&dev));
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaMalloc(&d, MLP_DEV_BYTES) != cudaSuccess || cudaMalloc(&derr, 4) != cudaSuccess) {
        cudaFree(d);
        FAIL(FMM_ERR_OOM, "allocating model storage failed");
    }
    cudaStream_t s = S(stream);
    int herr = 0;
    bool ok = cudaMemcpyAsync(d, h.data(), MLP_DEV_BYTES, cudaMemcpyHostToDevice, s) == cudaSuccess &&
              cudaMemsetAsync(derr, 0, 4, s) == cudaSuccess;
    if (ok) {
        mlp_predict_dev(d, n, feat, pred, sms, derr, s);
        ok = cudaMemcpyAsync(&herr, derr, 4, cudaMemcpyDeviceToHost, s) == cudaSuccess &&
             cudaStreamSynchronize(s) == cudaSuccess;
    }
    const cudaError_t e = cudaGetLastError();
    cudaFree(d);
    cudaFree(derr);
    if (!ok || e != cudaSuccess) FAIL(FMM_ERR_CUDA, "inference failed: %s", cudaGetErrorString(e));
    if (herr) FAIL(FMM_ERR_TIMEOUT, "a bounded wait in the tensor-core inference gave up (code %d)", herr);
    return FMM_OK;
}

int fmm_set_mlp(fmm_plan* pl, const float* blob, int64_t nblob) {
    if (!pl) return fail_plan(nullptr, FMM_ERR_ARG, "plan is NULL");
    if (!pl->cfg.learned_p) FAIL(FMM_ERR_ARG, "plan was not created with learned_p");
    if (nblob != FMM_MLP_NBLOB) FAIL(FMM_ERR_ARG, "nblob=%lld, expected %d", (long long)nblob, FMM_MLP_NBLOB);
    if (int rc = check_blob(pl, blob)) return rc;
    std::vector<unsigned char> h(MLP_DEV_BYTES);
    mlp_pack_device(blob, h.data());
    if (!pl->mlp_dev && cudaMalloc(&pl->mlp_dev, MLP_DEV_BYTES) != cudaSuccess) {
        pl->mlp_dev = nullptr;
        FAIL(FMM_ERR_OOM, "allocating model storage failed");
    }
    CK(cudaMemcpy(pl->mlp_dev, h.data(), MLP_DEV_BYTES, cudaMemcpyHostToDevice));
    pl->log10_kappa = blob[6];
    pl->mlp_set = true;
    return FMM_OK;
}

int fmm_plan_pair_orders(fmm_plan* pl, int8_t* orders, int64_t cap, int64_t* count) {
    if (!pl) return fail_plan(nullptr, FMM_ERR_ARG, "plan is NULL");
    if (!pl->cfg.learned_p || !pl->ad) FAIL(FMM_ERR_ARG, "plan was not created with learned_p");
    if (!pl->built) FAIL(FMM_ERR_STATE, "fmm_build_tree has not been called");
    const int64_t np = pl->ad->nm2l;
    if (count) *count = np;
    if (cap < np || np == 0) return FMM_OK;
    if (!orders) FAIL(FMM_ERR_ARG, "null output array");
    if (!pl->ad->porder || (!pl->ad->orders_fixed && !pl->ad->orders_chosen))
        FAIL(FMM_ERR_STATE, "no M2L has chosen the orders of this tree's pairs yet");
    CK(cudaDeviceSynchronize());
    CK(cudaMemcpy(orders, pl->ad->porder, (size_t)np, cudaMemcpyDeviceToHost));
    return FMM_OK;
}

int fmm_set_pair_orders(fmm_plan* pl, const int8_t* orders, int64_t n) {
    if (!pl) return fail_plan(nullptr, FMM_ERR_ARG, "plan is NULL");
    if (!pl->cfg.learned_p) FAIL(FMM_ERR_ARG, "plan was not created with learned_p");
    if (!orders) {
        if (pl->ad) pl->ad->orders_fixed = false;
        return FMM_OK;
    }
    if (int rc = need_pairs(pl, 0)) return rc;
    if (n != pl->ad->nm2l) FAIL(FMM_ERR_ARG, "n=%lld, the tree has %d M2L pairs", (long long)n, pl->ad->nm2l);
    for (int64_t k = 0; k < n; ++k)
        if (orders[k] < 0 || orders[k] > pl->cfg.p) FAIL(FMM_ERR_ARG, "order %d of pair %lld outside 0..p", orders[k], (long long)k);
    if (n > 0) CK(cudaMemcpy(pl->ad->porder, orders, (size_t)n, cudaMemcpyHostToDevice));
    pl->ad->orders_fixed = true;
    pl->ad->n_orders = n;
    return FMM_OK;
}

}  // extern "C"
