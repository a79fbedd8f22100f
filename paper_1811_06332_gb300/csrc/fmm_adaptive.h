// Adaptive-octree plan state and launchers (fmm_adaptive*.cu).
#pragma once
#include <vector>

#include "fmm_internal.h"

namespace fmm {

struct AdState {
    int64_t n = 0;
    int nc = 0;
    int nn = 0, nleaf = 0, nm2l = 0, np2p = 0, ntarg = 0;
    std::vector<int> lvl;   // level L: nodes [lvl[L], lvl[L+1])
    // particles (sorted) and sort buffers
    double *xs = nullptr, *ys = nullptr, *zs = nullptr, *qs = nullptr;
    int* perm = nullptr;
    uint64_t *k0 = nullptr, *k1 = nullptr;
    int *v0 = nullptr, *v1 = nullptr, *hist = nullptr, *hsum = nullptr, *scr = nullptr;
    double *box = nullptr, *part = nullptr;
    // nodes
    int *lev = nullptr, *ix = nullptr, *iy = nullptr, *iz = nullptr, *nb = nullptr, *ne = nullptr;
    int *child0 = nullptr, *nchild = nullptr, *parent = nullptr;
    double *zc = nullptr, *rad = nullptr;
    int ap = 0;             // AP variant: centre-of-mass centres (Q: total charge per node)
    int binary = 0;         // binary median-split tree (App. C) instead of the octree
    // binary tree: split axis per node; per axis a permutation of the
    // particles sorted by (coordinate, index) within every cell (and its
    // next-level copy), the side of the split per particle, the node holding
    // each sorted position, partition flags and their scan
    int *axis = nullptr, *btP = nullptr, *btnode = nullptr, *btflag = nullptr, *btscan = nullptr;
    unsigned char* btside = nullptr;
    size_t cap_axis = 0, cap_btP = 0, cap_btnode = 0, cap_btflag = 0, cap_btscan = 0, cap_btside = 0;
    double* Q = nullptr;
    size_t cap_Q = 0;
    float* radf = nullptr;   // radii / (side / 2^22) rounded to FP32 (MAC screen)
    int *bounds = nullptr, *nch = nullptr, *choff = nullptr;
    // traversal
    int2 *q0 = nullptr, *q1 = nullptr;
    int *cm = nullptr, *cp = nullptr, *cq = nullptr, *om = nullptr, *op = nullptr, *oq = nullptr;
    unsigned char* tmode = nullptr;   // traversal decision of each frontier pair
    int2 *m2l = nullptr, *p2p = nullptr;
    int *moff = nullptr, *msrc = nullptr, *poff = nullptr, *psrc = nullptr, *order = nullptr, *leaf = nullptr;
    int4* ic = nullptr;        // integer node centres (fmm_adaptive_leaf.cu)
    float4* pos32 = nullptr;   // FP32 form: particle offsets from their leaf centre, charge
    float scale32 = 0.f;       // side / 2^22: unit of the integer centres
    float mac_band = 1e-5f;    // relative band of the FP32 MAC screen
    double side = 0.0;         // side of the root cube (cell of level l: side / 2^l)
    // expansions (node-major)
    double *M = nullptr, *L = nullptr;
    float* M32 = nullptr;
    int* counter = nullptr;
    // capacities (bytes)
    size_t cap_xs = 0, cap_ys = 0, cap_zs = 0, cap_qs = 0, cap_perm = 0, cap_k0 = 0, cap_k1 = 0, cap_v0 = 0,
           cap_v1 = 0, cap_hist = 0, cap_hsum = 0, cap_scr = 0, cap_box = 0, cap_part = 0, cap_lev = 0, cap_ix = 0,
           cap_iy = 0, cap_iz = 0, cap_nb = 0, cap_ne = 0, cap_child0 = 0, cap_nchild = 0, cap_parent = 0,
           cap_zc = 0, cap_rad = 0, cap_radf = 0, cap_bounds = 0, cap_nch = 0, cap_choff = 0, cap_q0 = 0, cap_q1 = 0, cap_cm = 0,
           cap_cp = 0, cap_cq = 0, cap_om = 0, cap_op = 0, cap_oq = 0, cap_tmode = 0, cap_m2l = 0, cap_p2p = 0, cap_moff = 0,
           cap_msrc = 0, cap_poff = 0, cap_psrc = 0, cap_order = 0, cap_leaf = 0, cap_ic = 0, cap_pos32 = 0,
           cap_M = 0, cap_L = 0, cap_M32 = 0, cap_counter = 0;
    // learned per-pair M2L order (fmm_learn.cu, fmm_mlp_tc.cu)
    int* ptgt = nullptr;           // M2L pair -> target node
    float* nodeF = nullptr;        // per node: shape terms 1..4, ln count, radius, 0, 0
    signed char* porder = nullptr; // order of each M2L pair
    int* iota = nullptr;           // 0..nn-1: target order of the per-order M2L launches
    int *bcnt = nullptr, *boff = nullptr, *bsrc = nullptr;   // pairs grouped by (order, target)
    float* fsum = nullptr;         // per node: far-field magnitude sum and pair count of its own M2L list
    float* nodeK = nullptr;        // per node: log10 of the M2L pairs on its ancestor chain (itself included)
    size_t cap_ptgt = 0, cap_nodeF = 0, cap_porder = 0, cap_iota = 0, cap_bcnt = 0, cap_boff = 0, cap_bsrc = 0,
           cap_fsum = 0, cap_nodeK = 0;
    bool orders_fixed = false;     // orders given by the caller instead of the model
    bool orders_chosen = false;    // porder holds the model's orders for the current tree
    int64_t n_orders = 0;
    unsigned gen = 0;              // bumped whenever a buffer moves
    // autotuned persistent grid of the M2L kernel
    int m2l_blocks = 0, m2l_blocks_per_sm = 0;
    float m2l_tuned_ms = 0.f;
    // captured operator sequence
    cudaGraphExec_t gexec = nullptr;
    bool graph_ok = false;
    const void* graph_key[8] = {nullptr};
};

void ad_free(AdState* a);
int ad_build(AdState* a, int64_t n, const double* x, const double* y, const double* z, const double* q,
             int max_leaf, double theta, int nc, int prec, cudaStream_t s);
int ad_run_p2m(AdState* a, int prec, int p, int basis, const DevTables& T, cudaStream_t s);
int ad_run_m2m(AdState* a, int prec, int p, int basis, const DevTables& T, cudaStream_t s);
int ad_run_m2l(AdState* a, int p, int basis, int prec, int sms, cudaStream_t s);
int ad_run_l2l(AdState* a, int prec, int p, int basis, const DevTables& T, cudaStream_t s);
int ad_run_l2p(AdState* a, int prec, int p, int basis, const DevTables& T, double* pot, double* ax, double* ay, double* az,
               cudaStream_t s);
int ad_run_p2p(AdState* a, int prec, int sms, double* pot, double* ax, double* ay, double* az, cudaStream_t s);
int ad_learn_prepare(AdState* a, cudaStream_t s);
int ad_run_m2l_orders(AdState* a, int p, int basis, int prec, int sms, const unsigned char* mlp, float thr, int* err,
                      cudaStream_t s);
int ad_order_counts(AdState* a, int p, int64_t* out, cudaStream_t s);
int ad_order_keys(int n, const signed char* porder, uint64_t* key, int* val, cudaStream_t s);
int ad_bucket_csr(int n, int nn, const uint64_t* key, const int* val, const int* ptgt, const int* msrc, int* bsrc,
                  int* bcnt, cudaStream_t s);
int ad_iota(int n, int* a, cudaStream_t s);

// fmm_btree.cu (binary median-split tree)
int bt_axis_keys(int64_t n, const double* c, uint64_t* key, int* val, cudaStream_t s);
int bt_nodes(int lb, int le, int max_leaf, const int* nb, const int* ne, const int* P, int64_t n, const double* x,
             const double* y, const double* z, double* zc, int* axis, int* nsplit, cudaStream_t s);
int bt_children(int lb, int le, const int* nsplit, const int* off, int* lev, int* nb, int* ne, int* child0,
                int* nchild, int* parent, cudaStream_t s);
int bt_side(int64_t n, int lb, int le, const int* node, const int* nb, const int* ne, const int* nchild,
            const int* axis, const int* P, unsigned char* side, cudaStream_t s);
int bt_flags(int64_t n, const int* Pa, const unsigned char* side, int* flag, cudaStream_t s);
int bt_partition(int64_t n, int lb, int le, const int* node, const int* nb, const int* ne, const int* nchild,
                 const int* Pa, const int* scan, int* Pn, cudaStream_t s);
int bt_advance(int64_t n, int lb, int le, int* node, const int* nb, const int* ne, const int* nchild,
               const int* child0, cudaStream_t s);

// fmm_adaptive.cu
int radix_sort(int64_t n, uint64_t* k0, int* v0, uint64_t* k1, int* v1, int bits, int* hist, int* hsum,
                int* scratch, cudaStream_t s);
int ad_bbox(int64_t n, const double* x, const double* y, const double* z, double* part, double* box, cudaStream_t s);
int ad_morton(int64_t n, const double* x, const double* y, const double* z, const double* box, uint64_t* key,
              int* val, cudaStream_t s);
int ad_gather(int64_t n, const int* perm, const double* x, const double* y, const double* z, const double* q,
              double* xs, double* ys, double* zs, double* qs, cudaStream_t s);
int ad_split_count(int lb, int le, int max_leaf, const int* lev, const int* nb, const int* ne, const uint64_t* key,
                   int* bounds, int* nch, cudaStream_t s);
int ad_split_write(int lb, int le, const int* bounds, const int* nch, const int* choff, int* lev, int* ix, int* iy,
                   int* iz, int* nb, int* ne, int* child0, int* nchild, int* parent, cudaStream_t s);
int ad_centres(int nn, const int* lev, const int* ix, const int* iy, const int* iz, const double* box, double* zc,
               cudaStream_t s);
int ad_com(int lb, int le, const int* nb, const int* ne, const int* child0, const int* nchild, const double* xs,
           const double* ys, const double* zs, const double* qs, double* Q, double* zc, cudaStream_t s);
int ad_zero_dipole(int nn, int nc, double* M, cudaStream_t s);
int ad_radii(int lb, int le, const int* nb, const int* ne, const int* child0, const int* nchild, const double* zc,
             const double* xs, const double* ys, const double* zs, double* rad, cudaStream_t s);
int ad_trav_count(int nq, const int2* q, double theta, const int* nchild, const double* zc, const double* rad,
                  int* cm, int* cp, int* cq, unsigned char* mode, const int4* ic, const float* radf, float band,
                  cudaStream_t s);
int ad_radf(int nn, const double* rad, const double* box, float* radf, cudaStream_t s);
int ad_trav_write(int nq, const int2* q, const unsigned char* mode, const int* nchild, const int* child0,
                  const int* om, const int* op, const int* oq, int mbase, int pbase, int2* m2l, int2* p2p, int2* qn,
                  cudaStream_t s);
int ad_pair_keys(int n, const int2* pr, uint64_t* key, int* val, cudaStream_t s);
int ad_pair_csr(int n, const uint64_t* key, const int* val, const int2* pr, int* src, int* cnt, cudaStream_t s);
int ad_len_keys(int nn, const int* off, uint64_t* key, int* val, cudaStream_t s);
int ad_leaf_keys(int nn, const int* nchild, const int* nb, uint64_t* key, int* val, cudaStream_t s);
int ad_to_f32(int64_t n, const double* a, float* b, cudaStream_t s);
int ad_m2m(int prec, int p, int basis, int lb, int le, const int* child0, const int* nchild, const double* zc, double* Mn,
           const DevTables& T, const int* lev, double side, cudaStream_t s);
int ad_l2l(int prec, int p, int basis, int lb, int le, const int* parent, const double* zc, double* Ln, const DevTables& T,
           const int* lev, double side, cudaStream_t s);
int ad_p2p(int nwork, const int* work, const int* off, const int* src, const int* nb, const int* ne,
           const double* zc, const double* xs, const double* ys, const double* zs, const double* qs,
           const int* perm, double* pot, double* ax, double* ay, double* az, int* counter, int blocks,
           cudaStream_t s);
int launch_m2l_list(int p, int basis, int prec, int ntarg, const int* order, const int* off, const int* src,
                    const double* zc, const int4* ic, float scale, const void* M, int ldm, double* Ln, int ld,
                    int accum, int* counter, int blocks, cudaStream_t s);
// FP32 multipole rows are padded to a multiple of 4 floats (16-byte loads)
inline int ld32_of(int nc) { return (nc + 3) & ~3; }
int ad_to_f32_rows(int64_t rows, int nc, int ldm, const double* a, float* b, cudaStream_t s);

// fmm_adaptive_leaf.cu
int ad_pos32(int nleaf, const int* leaf, const int* nb, const int* ne, const double* zc, const double* xs,
             const double* ys, const double* zs, const double* qs, float4* pos32, cudaStream_t s);
int ad_icentre(int nn, const int* lev, const int* ix, const int* iy, const int* iz, int4* ic, cudaStream_t s);
int ad_p2m_leaf(int prec, int p, int basis, int nleaf, const int* leaf, const int* nb, const int* ne,
                const double* zc, const double* xs, const double* ys, const double* zs, const double* qs,
                const float4* pos32, double* Mn, const DevTables& Tb, const int* lev, double side, cudaStream_t s);
int ad_l2p_leaf(int prec, int p, int basis, int nleaf, const int* leaf, const int* nb, const int* ne,
                const double* zc, const double* xs, const double* ys, const double* zs, const float4* pos32,
                const int* perm, const double* Ln, const DevTables& Tb, double* pot, double* ax, double* ay,
                double* az, const int* lev, double side, cudaStream_t s);
int ad_p2p32(int nwork, const int* work, const int* off, const int* src, const int* nb, const int* ne, const int4* ic,
             float scale, const float4* pos32, const int* perm, double* pot, double* ax, double* ay, double* az,
             int* counter, int blocks, cudaStream_t s);

}  // namespace fmm
