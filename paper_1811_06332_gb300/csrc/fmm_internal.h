// Internal declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "fmm_device.cuh"
#include "_gen/fmm_ctables.cuh"

namespace fmm {

struct DevOffsets {
    int detr[FMM_PMAX + 2];
    int expand[FMM_PMAX + 2];
    int reduce[FMM_PMAX + 2];
};

struct DevTables {
    double* detr = nullptr;
    double* expand = nullptr;
    double* reduce = nullptr;
    float* detr32 = nullptr;     // FP32 copies (FP32 forms)
    float* expand32 = nullptr;
    float* reduce32 = nullptr;
    int detr_off[FMM_PMAX + 2];
    int expand_off[FMM_PMAX + 2];
    int reduce_off[FMM_PMAX + 2];
    DevOffsets offsets() const {
        DevOffsets o;
        for (int j = 0; j < FMM_PMAX + 2; ++j) {
            o.detr[j] = detr_off[j];
            o.expand[j] = expand_off[j];
            o.reduce[j] = reduce_off[j];
        }
        return o;
    }
};

extern DevTables g_tab[64];
int ensure_tables(int dev);  // 0 ok, -2 CUDA error, -3 allocation failure
void count_launch();

// ---------------------------------------------------------------------------
// small warp helpers
// ---------------------------------------------------------------------------
static __device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Rebuilds the full symmetric polytensor X (ranks 0..p) from independent
// traceless components A (trace condition, App. B); lanes stride the output.
static __device__ __noinline__ void expand_tl_warp(int p, const double* A, double* X, const double* expand,
                               const DevOffsets& off, int lane) {
    const int ns = ns_of(p);
    for (int s = lane; s < ns; s += 32) {
        const int nx = c_sym_idx[s][0], ny = c_sym_idx[s][1], nz = c_sym_idx[s][2];
        const int j = nx + ny + nz;
        const int row = (j - nx) * (j - nx + 1) / 2 + nz;
        const double* E = expand + off.expand[j] + row * (2 * j + 1);
        double v = 0.0;
        for (int t = 0; t < 2 * j + 1; ++t) v += E[t] * A[j * j + t];
        X[s] = v;
    }
}

// generated per-order launchers (csrc/_gen/pair_P<p>.cu)
#define FMM_DECL_P(P)                                                                                   \
    int launch_dtensor_p##P(int basis, int prec, int64_t n, const double* r, void* D, cudaStream_t s); \
    int launch_m2l_pair_p##P(int basis, int prec, int64_t n, const void* M, const double* r, void* L, \
                             int accumulate, cudaStream_t s);                                           \
    int launch_dtable_p##P(int noff, const double* o, double* D, cudaStream_t s);
FMM_DECL_P(0) FMM_DECL_P(1) FMM_DECL_P(2) FMM_DECL_P(3) FMM_DECL_P(4) FMM_DECL_P(5)
FMM_DECL_P(6) FMM_DECL_P(7) FMM_DECL_P(8) FMM_DECL_P(9) FMM_DECL_P(10)
#undef FMM_DECL_P

// fmm_ops.cu
int launch_p2m(int p, int basis, int mode, int64_t ncell, const int64_t* start64, const int* start32,
               const double* x, const double* y, const double* z, const double* q, const double* centre,
               int depth, double inv_h, double* M, int64_t ldm, const DevTables& T, cudaStream_t s,
               const double* px = nullptr, const double* py = nullptr, const double* pz = nullptr);
int launch_p2p_dipole(int depth, int64_t nleaf, const int* start, const double* xs, const double* ys,
                      const double* zs, const double* pxs, const double* pys, const double* pzs, const int* perm,
                      double* pot, double* ax, double* ay, double* az, cudaStream_t s);
int launch_gather3(int64_t n, const int* perm, const double* a, const double* b, const double* c, double* oa,
                   double* ob, double* oc, cudaStream_t s);
// prec 0: double storage and arithmetic, 1: float
int launch_m2m_general(int prec, int p, int basis, int64_t n, const void* Mc, const double* delta, void* Mp,
                       const DevTables& T, cudaStream_t s);
int launch_l2l_general(int prec, int p, int basis, int64_t n, const void* Lp, const double* delta, void* Lc,
                       const DevTables& T, cudaStream_t s);
int launch_l2p_general(int prec, int p, int basis, int64_t n, const void* L, const double* rb, void* out,
                       const DevTables& T, cudaStream_t s);
// fused traceless M2M of Eq. Detracer2 (FP64); 0 ok, -2 CUDA error, -3 allocation failure
int launch_m2m_fused(int p, int64_t n, const double* Mc, const double* delta, double* Mp, const DevTables& T,
                     cudaStream_t s);
int m2m_fused_terms(int p);
int launch_direct(int64_t n, const double* x, const double* y, const double* z, const double* q, int64_t nt,
                  const int64_t* targets, double* pot, double* ax, double* ay, double* az, cudaStream_t s);
int launch_m2m_level(int p, int basis, int l, const double* W, const double* Mch, int64_t nch, double* Mpa,
                     int64_t npa, cudaStream_t s);
int launch_l2l_level(int p, int basis, int l, const double* V, const double* Lpa, int64_t npa, double* Lch,
                     int64_t nch, cudaStream_t s);
int launch_zero4(int64_t n, double* a, double* b, double* c, double* d, cudaStream_t s);
int launch_fill(int64_t n, double* a, double v, cudaStream_t s);

// fmm_leafops.cu (prec 0: double arithmetic, 1: float arithmetic)
int launch_p2m_leaf(int prec, int p, int basis, int depth, int64_t nleaf, const int* start, const double* xs,
                    const double* ys, const double* zs, const double* qs, double* M, const DevTables& Tb,
                    cudaStream_t s, const float4* pos32 = nullptr, float* msym = nullptr, float* M32 = nullptr);
int launch_l2p_leaf2(int prec, int p, int basis, int depth, int64_t nleaf, const int* start, const double* xs,
                     const double* ys, const double* zs, const int* perm, const double* Lt, const DevTables& Tb,
                     double* pot, double* ax, double* ay, double* az, cudaStream_t s,
                     const float4* pos32 = nullptr,
                     const float* Lt32 = nullptr);
int launch_p2p_leaf2(int prec, int depth, int64_t nleaf, const int* start, const double* xs, const double* ys,
                     const double* zs, const double* qs, const int* perm, double* pot, double* ax, double* ay,
                     double* az, cudaStream_t s);

// fmm_m2l32.cu and generated grp_*.cu
int launch_build_ktab(int p, int basis, int kst, const unsigned char* ent, const double* Dtab, float* K,
                      cudaStream_t s);
int grouped_entries(int p, int basis, unsigned char* out, int cap);
int launch_to_f32(int64_t n, const double* a, float* b, cudaStream_t s);
int launch_m2l_grp(int p, int basis, int l, const float* M, double* Lt, const float* K, int64_t ncell,
                   cudaStream_t s);
// the same with FP32 locals (uniform FP32 and tensor-core plans)
int launch_m2l_grpf(int p, int basis, int l, const float* M, float* Lt, const float* K, int64_t ncell,
                    cudaStream_t s, float* part, int64_t part_cap);
int64_t m2l_grpf_part_elems(int p, int basis, int l);   // floats of part for level l (0: unsplit)
// FP64 form of the grouped M2L (packed FP64 matrices)
int launch_build_ktab64(int p, int basis, int kst, const unsigned char* ent, const double* Dtab, double* K,
                        cudaStream_t s);
int launch_m2l_grp64(int p, int basis, int l, const double* M, double* Lt, const double* K, int64_t ncell,
                     cudaStream_t s, double* part, int64_t part_cap);
int64_t m2l_grp64_part_elems(int p, int basis, int l);
int grouped_kstride(int p, int basis);

// fmm_api.cu: translation matrices of the uniform octree in scaled units
}  // namespace fmm
#include <vector>
extern "C" __attribute__((visibility("hidden"))) void build_translation(int p, int basis, std::vector<double>& W, std::vector<double>& V);
namespace fmm {

// generated shift_*.cu: FP32 level shifts (m2m = 1: M2M, 0: L2L)
// part (M2M): 8 x nc x ny floats for the per-child form (with the FP32
// copies X32 of the children and Y32 of the parents), or nullptr.
// Returns the number of kernels launched, -1 without a kernel for (p, basis).
int launch_shift32(int p, int basis, int m2m, int l, const float* A, const double* X, int64_t nx, double* Y,
                   int64_t ny, cudaStream_t s, float* part = nullptr, const float* X32 = nullptr,
                   float* Y32 = nullptr);
int shift32_supported(int p, int basis);
// L2L on FP32 locals (generated l2l32f); the launches made, -1 without a kernel
int launch_l2l32f(int p, int basis, int l, const float* V, const float* X, int64_t nx, float* Y, int64_t ny,
                  cudaStream_t s);
int launch_l2p_p2p32(int p, int basis, int depth, int64_t nleaf, const int* start, const float4* pos, const int* perm,
                     const double* Lt, const DevTables& Tb, double* pot, double* ax, double* ay, double* az,
                     cudaStream_t s, const float* Lt32 = nullptr);
int launch_p2p32(int depth, int64_t nleaf, const int* start, const float4* pos, const int* perm, double* pot,
                 double* ax, double* ay, double* az, cudaStream_t s);

// fmm_m2l_tc.cu (tensor-core offset-grouped M2L, traceless basis)
// tf selects the operand type: 0 = BF16 hi/lo, 1 = TF32 hi/lo
int tc_supported(int p, int basis);
int tc_first_level();   // levels below run on the FP32 grouped kernel
int tc_layout(int p, int tf, int* out, int nout);
size_t tc_mat_bytes(int tf);
int tc_default_cw(int tf);
int tc_mat_niss(int p, int tf, int cw);
int tc_elem_bytes(int tf);
size_t tc_m_elems(int l);
int wait_selftest(long spin, int arrive, int* err, cudaStream_t s);
// tensor-core M2L with the matrix as the A operand (fmm_m2l_tct.cu)
int tct_np(int p);
size_t tct_bytes();
int tct_ty(int l);
void tct_box(int l, unsigned (&box)[5]);
int tct_build(int p, const double* Dtab, void* B, cudaStream_t s);
int tct_m2l_level(int p, int l, int first_part_only, const void* maps, const void* B, double* Lt, int* err,
                  cudaStream_t s, float* Lt32 = nullptr);
// tables of the multipole columns >= 48 that kernel shape 3 contracts on the
// CUDA cores (fmm_m2l_rest.cu): rows of rank <= p - 6
int rest_rows(int p);
int rest_kstride(int p);   // floats per offset of the matrix table
int rest_cstride(int p);   // floats per cell of the multipole copy
int build_krest(int p, const double* Dtab, float* Krest, cudaStream_t s);
int launch_rest_pack(int p, int l, const double* M, float* Mrest, cudaStream_t s, const float* M32 = nullptr);
// Lt (level l, after the tensor-core kernel) += those products.  Levels
// where rest_nsplit(l) > 1 split the source classes over that many blocks
// per tile when part holds rest_nsplit(l) * rest_rows(p) * 8^l floats
// (part_cap), summed in order by a second kernel; else one block per tile.
int rest_nsplit(int l);
int launch_m2l_rest(int p, int l, const float* Mrest, const float* Krest, double* Lt, cudaStream_t s,
                    float* Lt32 = nullptr, float* part = nullptr, int64_t part_cap = 0);
size_t tc_maps_bytes();
// kern 0: per-offset matrices streamed from global memory (tc_build_mat at
// chunk width cw; niss follows from the layout); kern 1 (BF16 only): the
// matrices built on chip (tg_build; niss 1 or 2)
int tc_build_mat(int p, int tf, int cw, const double* Dtab, void* B, cudaStream_t s);
int tc_encode_maps(int l, int tf, void* hi, void* lo, void* out_maps);
int tc_m2l_level(int p, int tf, int kern, int cw, int niss, int l, const double* M, void* hi, void* lo,
                 const void* maps, const void* B, double* Lt, int* err, cudaStream_t s,
                 const float* M32 = nullptr, float* Lt32 = nullptr);
// fmm_m2l_tcgen.cu (BF16 hi/lo form, offset matrices built on chip)
int tg_supported(int p);
size_t tg_b_bytes();
int tg_build(int p, int cw, int niss, const double* Dtab, void* B, cudaStream_t s);
int tg_m2l_level(int p, int cw, int niss, int l, const void* maps, const void* B, double* Lt, int* err,
                 cudaStream_t s, float* Lt32 = nullptr);
int tg_layout_host(int p, int cw, int niss, int* out, int nout, uint32_t* groups, int gcap);
int tg_default_cw();
int tg_default_niss();

// fmm_tune.cu: cache of autotuned tensor-core kernel shapes (JSON file)
int tune_cache_get(const char* path, const char* key, int* kernel, int* cw, int* niss, double* ms);
int tune_cache_put(const char* path, const char* key, int kernel, int cw, int niss, double ms);

// fmm_tree.cu
size_t tree_scratch_bytes(int64_t n, int64_t nleaf);
// exclusive scan of m ints into out[0..m] (out[m] = total)
void scan_excl_int(const int* in, int* out, int64_t m, int* scratch, cudaStream_t s);
int launch_uniform_tree(int64_t n, int depth, const double* x, const double* y, const double* z, const double* q,
                        double* xs, double* ys, double* zs, double* qs, int* perm, int* start, void* scratch,
                        cudaStream_t s, float4* pos32 = nullptr, float4* pos32c = nullptr);

}  // namespace fmm
