// Adaptive-octree plan state: builds the tree and the interaction lists on
// the device (host loop over levels and traversal steps, sizes read back),
// and runs the operator sequence P2M, M2M, M2L, L2L, L2P, P2P over it.
//
// Batching: M2L and P2P run as persistent kernels that take work from an
// atomic counter (M2L targets ordered by list length, longest first); the
// persistent grid size of M2L is picked by timing candidates on the first
// evaluation of a plan (autotuner); the operator sequence can be captured
// into a CUDA graph and replayed while the tree and lists keep their sizes.
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "fmm_adaptive.h"
#include "fmm_learn.h"

namespace fmm {

static int grow_bytes(void** p, size_t* cap, size_t need, unsigned* gen) {
    if (need <= *cap) return 0;
    ++*gen;
    size_t nc = need + need / 2 + 4096;
    void* q = nullptr;
    if (cudaMalloc(&q, nc) != cudaSuccess) return -3;
    if (*p) {
        if (cudaMemcpy(q, *p, *cap, cudaMemcpyDeviceToDevice) != cudaSuccess) { cudaFree(q); return -2; }
        cudaFree(*p);
    }
    *p = q;
    *cap = nc;
    return 0;
}
#define GROW(ptr, capname, bytes)                                                            \
    do {                                                                                     \
        int r_ = grow_bytes((void**)&(ptr), &(capname), (size_t)(bytes), &a->gen);         \
        if (r_) return r_;                                                                   \
    } while (0)

void ad_free(AdState* a) {
    if (!a) return;
    void* ptrs[] = {a->Q, a->axis, a->btP, a->btnode, a->btflag, a->btscan, a->btside, a->xs, a->ys, a->zs, a->qs, a->perm, a->k0, a->k1, a->v0, a->v1, a->hist, a->hsum, a->scr,
                    a->box, a->part, a->lev, a->ix, a->iy, a->iz, a->nb, a->ne, a->child0, a->nchild, a->parent,
                    a->zc, a->rad, a->radf, a->bounds, a->nch, a->choff, a->q0, a->q1, a->cm, a->cp, a->cq, a->om, a->op,
                    a->oq, a->tmode, a->m2l, a->p2p, a->moff, a->msrc, a->poff, a->psrc, a->order, a->leaf, a->ic,
                    a->pos32, a->M, a->L, a->M32, a->counter, a->ptgt, a->nodeF, a->porder, a->iota,
                    a->bcnt, a->boff, a->bsrc, a->fsum, a->nodeK};
    for (void* p : ptrs) cudaFree(p);
    if (a->gexec) cudaGraphExecDestroy(a->gexec);
    delete a;
}

static int d2h_int(const int* d, int* h, cudaStream_t s) {
    if (cudaMemcpyAsync(h, d, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return -2;
    return cudaStreamSynchronize(s) == cudaSuccess ? 0 : -2;
}

// exclusive scan of n ints into out[0..n]; returns the total in *tot
static int scan_total(const int* in, int* out, int n, int* scr, int* tot, cudaStream_t s) {
    scan_excl_int(in, out, n, scr, s);
    return d2h_int(out + n, tot, s);
}

// sort (key, val) pairs by the low `bits` of key; the result is in (k0, v0)
// afterwards (after an odd number of passes the two buffer pairs swap roles)
static int sort_pairs(AdState* a, int64_t n, int bits, cudaStream_t s) {
    const int64_t nblk = (n + 2047) / 2048;
    GROW(a->hist, a->cap_hist, (256 * nblk + 1) * 4);
    GROW(a->hsum, a->cap_hsum, (256 * nblk + 1) * 4);
    if (radix_sort(n, a->k0, a->v0, a->k1, a->v1, bits, a->hist, a->hsum, a->scr, s)) {
        std::swap(a->k0, a->k1);
        std::swap(a->cap_k0, a->cap_k1);
        std::swap(a->v0, a->v1);
        std::swap(a->cap_v0, a->cap_v1);
    }
    return 0;
}

// Binary median-split tree (App. C; fmm_btree.cu): three permutations
// sorted by (coordinate, index), then level by level the nodes (bounding
// boxes from the permutations), their children and a stable partition of
// each permutation by the side of the split; finally the sorted particles,
// centres and radii.
static int build_binary(AdState* a, int64_t n, const double* x, const double* y, const double* z, const double* q,
                        int max_leaf, cudaStream_t s) {
    GROW(a->btP, a->cap_btP, (size_t)n * 24);          // P_x, P_y, P_z and their next-level copies
    GROW(a->btnode, a->cap_btnode, (size_t)n * 4);
    GROW(a->btflag, a->cap_btflag, (size_t)(n + 1) * 4);
    GROW(a->btscan, a->cap_btscan, (size_t)(n + 1) * 4);
    GROW(a->btside, a->cap_btside, (size_t)n);
    int* P = a->btP;
    int* Pn = a->btP + 3 * n;
    const double* co[3] = {x, y, z};
    for (int d = 0; d < 3; ++d) {
        bt_axis_keys(n, co[d], a->k0, a->v0, s);
        if (int r = sort_pairs(a, n, 64, s)) return r;
        cudaMemcpyAsync(P + d * n, a->v0, n * 4, cudaMemcpyDeviceToDevice, s);
    }
    cudaMemsetAsync(a->btnode, 0, n * 4, s);
    cudaMemsetAsync(a->btside, 0, n, s);
    int cap = 1024;
    auto node_cap = [&](int need) -> int {
        const size_t nd = (size_t)need;
        GROW(a->lev, a->cap_lev, nd * 4); GROW(a->nb, a->cap_nb, nd * 4); GROW(a->ne, a->cap_ne, nd * 4);
        GROW(a->child0, a->cap_child0, nd * 4); GROW(a->nchild, a->cap_nchild, nd * 4);
        GROW(a->parent, a->cap_parent, nd * 4); GROW(a->axis, a->cap_axis, nd * 4);
        GROW(a->zc, a->cap_zc, nd * 24);
        GROW(a->ix, a->cap_ix, nd * 4); GROW(a->iy, a->cap_iy, nd * 4); GROW(a->iz, a->cap_iz, nd * 4);
        return 0;
    };
    if (int r = node_cap(cap)) return r;
    {
        const int zero = 0, nn1 = (int)n, m1 = -1;
        cudaMemcpyAsync(a->lev, &zero, 4, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(a->nb, &zero, 4, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(a->ne, &nn1, 4, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(a->parent, &m1, 4, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(a->child0, &m1, 4, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(a->nchild, &zero, 4, cudaMemcpyHostToDevice, s);
        if (cudaStreamSynchronize(s) != cudaSuccess) return -2;   // host values must land first
    }
    a->lvl.assign(1, 0);
    int lb = 0, le = 1;
    while (le > lb) {
        a->lvl.push_back(le);
        const int m = le - lb;
        GROW(a->nch, a->cap_nch, (size_t)(m + 1) * 4);
        GROW(a->choff, a->cap_choff, (size_t)(m + 1) * 4);
        bt_nodes(lb, le, max_leaf, a->nb, a->ne, P, n, x, y, z, a->zc, a->axis, a->nch, s);
        int tot = 0;
        if (scan_total(a->nch, a->choff, m, a->scr, &tot, s)) return -2;
        if (le + tot > cap) {
            cap = 2 * (le + tot);
            if (int r = node_cap(cap)) return r;
        }
        bt_children(lb, le, a->nch, a->choff, a->lev, a->nb, a->ne, a->child0, a->nchild, a->parent, s);
        if (tot > 0) {
            bt_side(n, lb, le, a->btnode, a->nb, a->ne, a->nchild, a->axis, P, a->btside, s);
            for (int d = 0; d < 3; ++d) {
                bt_flags(n, P + d * n, a->btside, a->btflag, s);
                scan_excl_int(a->btflag, a->btscan, n, a->scr, s);
                bt_partition(n, lb, le, a->btnode, a->nb, a->ne, a->nchild, P + d * n, a->btscan, Pn + d * n, s);
            }
            std::swap(P, Pn);
            bt_advance(n, lb, le, a->btnode, a->nb, a->ne, a->nchild, a->child0, s);
        }
        lb = le;
        le = le + tot;
    }
    a->nn = le;
    // sorted order: P_x (every cell's particles contiguous, by x inside a leaf)
    GROW(a->perm, a->cap_perm, n * 4);
    cudaMemcpyAsync(a->perm, P, n * 4, cudaMemcpyDeviceToDevice, s);
    ad_gather(n, a->perm, x, y, z, q, a->xs, a->ys, a->zs, a->qs, s);
    GROW(a->rad, a->cap_rad, (size_t)a->nn * 8);
    for (int L = (int)a->lvl.size() - 2; L >= 0; --L)
        ad_radii(a->lvl[L], a->lvl[L + 1], a->nb, a->ne, a->child0, a->nchild, a->zc, a->xs, a->ys, a->zs, a->rad, s);
    cudaMemsetAsync(a->ix, 0, (size_t)a->nn * 4, s);
    cudaMemsetAsync(a->iy, 0, (size_t)a->nn * 4, s);
    cudaMemsetAsync(a->iz, 0, (size_t)a->nn * 4, s);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

int ad_build(AdState* a, int64_t n, const double* x, const double* y, const double* z, const double* q,
             int max_leaf, double theta, int nc, int prec, cudaStream_t s) {
    a->n = n;
    a->nc = nc;
    a->graph_ok = false;
    // per-particle storage
    GROW(a->xs, a->cap_xs, n * 8); GROW(a->ys, a->cap_ys, n * 8); GROW(a->zs, a->cap_zs, n * 8);
    GROW(a->qs, a->cap_qs, n * 8);
    const int64_t nk = n > 1 ? n : 2;
    GROW(a->k0, a->cap_k0, nk * 8); GROW(a->k1, a->cap_k1, nk * 8);
    GROW(a->v0, a->cap_v0, nk * 4); GROW(a->v1, a->cap_v1, nk * 4);
    GROW(a->scr, a->cap_scr, (size_t)1 << 22);
    GROW(a->box, a->cap_box, 64);
    GROW(a->part, a->cap_part, 256 * 6 * 8);
    GROW(a->counter, a->cap_counter, 64);
    if (n == 0) { a->nn = 0; a->nleaf = 0; a->nm2l = 0; a->np2p = 0; a->ntarg = 0; return 0; }
    ad_bbox(n, x, y, z, a->part, a->box, s);
    if (a->binary) {
        if (int r = build_binary(a, n, x, y, z, q, max_leaf, s)) return r;
    } else {
        ad_morton(n, x, y, z, a->box, a->k0, a->v0, s);
        if (int r = sort_pairs(a, n, 63, s)) return r;
        GROW(a->perm, a->cap_perm, n * 4);
        cudaMemcpyAsync(a->perm, a->v0, n * 4, cudaMemcpyDeviceToDevice, s);
        ad_gather(n, a->perm, x, y, z, q, a->xs, a->ys, a->zs, a->qs, s);
        // sorted keys stay in k0; keep a copy (k0/k1 are reused by later sorts)
        uint64_t* keys = a->k1;
        cudaMemcpyAsync(keys, a->k0, n * 8, cudaMemcpyDeviceToDevice, s);
        // ---------------- tree, level by level ----------------
        int cap = 1024;
        auto node_cap = [&](int need) -> int {
            const size_t nd = (size_t)need;
            GROW(a->lev, a->cap_lev, nd * 4); GROW(a->ix, a->cap_ix, nd * 4); GROW(a->iy, a->cap_iy, nd * 4);
            GROW(a->iz, a->cap_iz, nd * 4); GROW(a->nb, a->cap_nb, nd * 4); GROW(a->ne, a->cap_ne, nd * 4);
            GROW(a->child0, a->cap_child0, nd * 4); GROW(a->nchild, a->cap_nchild, nd * 4);
            GROW(a->parent, a->cap_parent, nd * 4);
            return 0;
        };
        if (int r = node_cap(cap)) return r;
        {
            const int zero = 0, nn1 = (int)n, m1 = -1;
            cudaMemcpyAsync(a->lev, &zero, 4, cudaMemcpyHostToDevice, s);
            cudaMemcpyAsync(a->ix, &zero, 4, cudaMemcpyHostToDevice, s);
            cudaMemcpyAsync(a->iy, &zero, 4, cudaMemcpyHostToDevice, s);
            cudaMemcpyAsync(a->iz, &zero, 4, cudaMemcpyHostToDevice, s);
            cudaMemcpyAsync(a->nb, &zero, 4, cudaMemcpyHostToDevice, s);
            cudaMemcpyAsync(a->ne, &nn1, 4, cudaMemcpyHostToDevice, s);
            cudaMemcpyAsync(a->parent, &m1, 4, cudaMemcpyHostToDevice, s);
            cudaMemcpyAsync(a->child0, &m1, 4, cudaMemcpyHostToDevice, s);
            cudaMemcpyAsync(a->nchild, &zero, 4, cudaMemcpyHostToDevice, s);
            if (cudaStreamSynchronize(s) != cudaSuccess) return -2;   // host values must land first
        }
        a->lvl.assign(1, 0);
        int lb = 0, le = 1;
        while (le > lb) {
            a->lvl.push_back(le);
            const int m = le - lb;
            GROW(a->bounds, a->cap_bounds, (size_t)m * 9 * 4);
            GROW(a->nch, a->cap_nch, (size_t)(m + 1) * 4);
            GROW(a->choff, a->cap_choff, (size_t)(m + 1) * 4);
            ad_split_count(lb, le, max_leaf, a->lev, a->nb, a->ne, keys, a->bounds, a->nch, s);
            int tot = 0;
            if (scan_total(a->nch, a->choff, m, a->scr, &tot, s)) return -2;
            if (le + tot > cap) {
                cap = 2 * (le + tot);
                if (int r = node_cap(cap)) return r;
            }
            ad_split_write(lb, le, a->bounds, a->nch, a->choff, a->lev, a->ix, a->iy, a->iz, a->nb, a->ne, a->child0,
                           a->nchild, a->parent, s);
            lb = le;
            le = le + tot;
        }
        a->nn = le;
        // lvl: level L holds nodes [lvl[L], lvl[L+1]); the last entry is nn
        GROW(a->zc, a->cap_zc, (size_t)a->nn * 24);
        GROW(a->rad, a->cap_rad, (size_t)a->nn * 8);
        ad_centres(a->nn, a->lev, a->ix, a->iy, a->iz, a->box, a->zc, s);
        if (a->ap) {
            // AP: centres of mass, bottom-up level by level
            GROW(a->Q, a->cap_Q, (size_t)a->nn * 8);
            for (int L = (int)a->lvl.size() - 2; L >= 0; --L)
                ad_com(a->lvl[L], a->lvl[L + 1], a->nb, a->ne, a->child0, a->nchild, a->xs, a->ys, a->zs, a->qs, a->Q,
                       a->zc, s);
        }
        for (int L = (int)a->lvl.size() - 2; L >= 0; --L)
            ad_radii(a->lvl[L], a->lvl[L + 1], a->nb, a->ne, a->child0, a->nchild, a->zc, a->xs, a->ys, a->zs, a->rad, s);
    }
    // integer centres (FP32 centre offsets), FP32 radii (MAC screen), cell side
    GROW(a->ic, a->cap_ic, (size_t)a->nn * 16);
    ad_icentre(a->nn, a->lev, a->ix, a->iy, a->iz, a->ic, s);
    GROW(a->radf, a->cap_radf, (size_t)a->nn * 4);
    ad_radf(a->nn, a->rad, a->box, a->radf, s);
    {
        double bx[4] = {0.0, 0.0, 0.0, 0.0};
        cudaMemcpyAsync(bx, a->box, 32, cudaMemcpyDeviceToHost, s);
        if (cudaStreamSynchronize(s) != cudaSuccess) return -2;
        const double side = bx[3];
        a->scale32 = (float)(side / 4194304.0);
        a->side = side;
        // relative band of the FP32 MAC screen: 1e-5 covers its own rounding
        // (~5e-7); the second term bounds the rounding of the FP64 centre
        // offsets, whose absolute error grows with the cube's distance from
        // the origin, relative to the smallest offset side / 2^22
        const double lo = fmax(fabs(bx[0]), fmax(fabs(bx[1]), fabs(bx[2])));
        const double band = 1e-5 + ldexp(lo / side + 2.0, -27);
        a->mac_band = band < 0.5 ? (float)band : 0.5f;
        // AP and the binary tree: the integer (octree) centres do not locate
        // the expansion centres, so the FP32 screen is bypassed and every pair
        // takes the FP64 rule
        if (a->ap || a->binary) a->mac_band = 1e30f;
    }
    // ---------------- directed dual traversal ----------------
    int nq = 1, nm = 0, np = 0;
    GROW(a->q0, a->cap_q0, 64);
    {
        const int2 root = make_int2(0, 0);
        cudaMemcpyAsync(a->q0, &root, 8, cudaMemcpyHostToDevice, s);
        if (cudaStreamSynchronize(s) != cudaSuccess) return -2;
    }
    while (nq > 0) {
        GROW(a->cm, a->cap_cm, (size_t)(nq + 1) * 4); GROW(a->cp, a->cap_cp, (size_t)(nq + 1) * 4);
        GROW(a->cq, a->cap_cq, (size_t)(nq + 1) * 4); GROW(a->om, a->cap_om, (size_t)(nq + 1) * 4);
        GROW(a->op, a->cap_op, (size_t)(nq + 1) * 4); GROW(a->oq, a->cap_oq, (size_t)(nq + 1) * 4);
        GROW(a->tmode, a->cap_tmode, (size_t)(nq + 1));
        ad_trav_count(nq, (const int2*)a->q0, theta, a->nchild, a->zc, a->rad, a->cm, a->cp, a->cq, a->tmode, a->ic,
                      a->radf, a->mac_band, s);
        int tot3[3] = {0, 0, 0};
        scan_excl_int(a->cm, a->om, nq, a->scr, s);
        scan_excl_int(a->cp, a->op, nq, a->scr, s);
        scan_excl_int(a->cq, a->oq, nq, a->scr, s);
        cudaMemcpyAsync(&tot3[0], a->om + nq, 4, cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(&tot3[1], a->op + nq, 4, cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(&tot3[2], a->oq + nq, 4, cudaMemcpyDeviceToHost, s);
        if (cudaStreamSynchronize(s) != cudaSuccess) return -2;
        const int tm = tot3[0], tp = tot3[1], tq = tot3[2];
        GROW(a->m2l, a->cap_m2l, (size_t)(nm + tm + 1) * 8);
        GROW(a->p2p, a->cap_p2p, (size_t)(np + tp + 1) * 8);
        GROW(a->q1, a->cap_q1, (size_t)(tq + 1) * 8);
        ad_trav_write(nq, (const int2*)a->q0, a->tmode, a->nchild, a->child0, a->om, a->op, a->oq, nm, np,
                      (int2*)a->m2l, (int2*)a->p2p, (int2*)a->q1, s);
        nm += tm;
        np += tp;
        std::swap(a->q0, a->q1);
        std::swap(a->cap_q0, a->cap_q1);
        nq = tq;
    }
    a->nm2l = nm;
    a->np2p = np;
    // ---------------- lists by target (stable) ----------------
    auto csr = [&](void* pairs, int npair, int** off, size_t* cap_off, int** srcp, size_t* cap_src) -> int {
        GROW(*off, *cap_off, (size_t)(a->nn + 1) * 4);
        GROW(*srcp, *cap_src, (size_t)(npair + 1) * 4);
        GROW(a->cm, a->cap_cm, (size_t)(a->nn + 1) * 4);
        cudaMemsetAsync(a->cm, 0, (size_t)(a->nn + 1) * 4, s);
        if (npair > 0) {
            GROW(a->k0, a->cap_k0, (size_t)npair * 8); GROW(a->k1, a->cap_k1, (size_t)npair * 8);
            GROW(a->v0, a->cap_v0, (size_t)npair * 4); GROW(a->v1, a->cap_v1, (size_t)npair * 4);
            ad_pair_keys(npair, (const int2*)pairs, a->k0, a->v0, s);
            int bits = 1;
            while ((1ll << bits) < a->nn) ++bits;
            if (int r = sort_pairs(a, npair, bits, s)) return r;
            ad_pair_csr(npair, a->k0, a->v0, (const int2*)pairs, *srcp, a->cm, s);
        }
        int tot = 0;
        return scan_total(a->cm, *off, a->nn, a->scr, &tot, s);
    };
    if (int r = csr(a->m2l, nm, &a->moff, &a->cap_moff, &a->msrc, &a->cap_msrc)) return r;
    if (int r = csr(a->p2p, np, &a->poff, &a->cap_poff, &a->psrc, &a->cap_psrc)) return r;
    // M2L work order (longest list first) and the number of targets with a list
    GROW(a->k0, a->cap_k0, (size_t)a->nn * 8); GROW(a->k1, a->cap_k1, (size_t)a->nn * 8);
    GROW(a->v0, a->cap_v0, (size_t)a->nn * 4); GROW(a->v1, a->cap_v1, (size_t)a->nn * 4);
    ad_len_keys(a->nn, a->moff, a->k0, a->v0, s);
    if (int r = sort_pairs(a, a->nn, 31, s)) return r;
    GROW(a->order, a->cap_order, (size_t)a->nn * 4);
    cudaMemcpyAsync(a->order, a->v0, (size_t)a->nn * 4, cudaMemcpyDeviceToDevice, s);
    // leaves in particle order
    ad_leaf_keys(a->nn, a->nchild, a->nb, a->k0, a->v0, s);
    if (int r = sort_pairs(a, a->nn, 33, s)) return r;
    GROW(a->leaf, a->cap_leaf, (size_t)a->nn * 4);
    cudaMemcpyAsync(a->leaf, a->v0, (size_t)a->nn * 4, cudaMemcpyDeviceToDevice, s);
    // counts back on the host: leaves, targets with M2L work
    {
        std::vector<int> nch(a->nn), off(a->nn + 1);
        cudaMemcpyAsync(nch.data(), a->nchild, (size_t)a->nn * 4, cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(off.data(), a->moff, (size_t)(a->nn + 1) * 4, cudaMemcpyDeviceToHost, s);
        if (cudaStreamSynchronize(s) != cudaSuccess) return -2;
        int nl = 0, nt = 0;
        for (int c = 0; c < a->nn; ++c) { nl += nch[c] == 0; nt += off[c + 1] > off[c]; }
        a->nleaf = nl;
        a->ntarg = nt;
    }
    // FP32 particle offsets from their leaf centre
    if (prec != 0) {
        GROW(a->pos32, a->cap_pos32, (size_t)n * 16);
        ad_pos32(a->nleaf, a->leaf, a->nb, a->ne, a->zc, a->xs, a->ys, a->zs, a->qs, a->pos32, s);
    }
    GROW(a->M, a->cap_M, (size_t)a->nn * nc * 8);
    GROW(a->L, a->cap_L, (size_t)a->nn * nc * 8);
    if (prec != 0) GROW(a->M32, a->cap_M32, (size_t)a->nn * ld32_of(nc) * 4);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

int ad_run_p2m(AdState* a, int prec, int p, int basis, const DevTables& T, cudaStream_t s) {
    if (a->n == 0) return 0;
    ad_p2m_leaf(prec, p, basis, a->nleaf, a->leaf, a->nb, a->ne, a->zc, a->xs, a->ys, a->zs, a->qs, a->pos32, a->M,
                T, a->lev, a->side, s);
    return 0;
}

int ad_run_m2m(AdState* a, int prec, int p, int basis, const DevTables& T, cudaStream_t s) {
    if (a->n == 0) return 0;
    for (int L = (int)a->lvl.size() - 2; L >= 0; --L)
        ad_m2m(prec, p, basis, a->lvl[L], a->lvl[L + 1], a->child0, a->nchild, a->zc, a->M, T, a->lev, a->side, s);
    return 0;
}

static int m2l_launch(AdState* a, int p, int basis, int prec, int blocks, cudaStream_t s) {
    cudaMemsetAsync(a->counter, 0, 4, s);
    const void* M = prec ? (const void*)a->M32 : (const void*)a->M;
    return launch_m2l_list(p, basis, prec ? 1 : 0, a->ntarg, a->order, a->moff, a->msrc, a->zc, a->ic, a->scale32, M,
                           prec ? ld32_of(a->nc) : a->nc, a->L, a->nc, 0, a->counter, blocks, s);
}

int ad_run_m2l(AdState* a, int p, int basis, int prec, int sms, cudaStream_t s) {
    if (a->n == 0) return 0;
    cudaMemsetAsync(a->L, 0, (size_t)a->nn * a->nc * 8, s);
    if (prec) ad_to_f32_rows(a->nn, a->nc, ld32_of(a->nc), a->M, a->M32, s);
    if (a->ntarg == 0) return 0;
    if (a->m2l_blocks == 0) {
        // autotune the persistent grid on the first evaluation: candidates of
        // 1..4 blocks of 128 threads per SM, each timed once after a warm-up
        // (the kernel overwrites its targets, so repeating it is harmless)
        int best = sms, bestb = 0;
        float bt = 1e30f;
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        for (int k = 1; k <= 4; ++k) {
            const int blocks = k * sms;
            m2l_launch(a, p, basis, prec, blocks, s);
            cudaEventRecord(e0, s);
            m2l_launch(a, p, basis, prec, blocks, s);
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < bt) { bt = ms; best = blocks; bestb = k; }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        a->m2l_blocks = best;
        a->m2l_blocks_per_sm = bestb;
        a->m2l_tuned_ms = bt;
    }
    if (m2l_launch(a, p, basis, prec, a->m2l_blocks, s) != 0) return -1;
    count_launch();
    return 0;
}

int ad_run_l2l(AdState* a, int prec, int p, int basis, const DevTables& T, cudaStream_t s) {
    if (a->n == 0) return 0;
    for (int L = 1; L + 1 < (int)a->lvl.size(); ++L)
        ad_l2l(prec, p, basis, a->lvl[L], a->lvl[L + 1], a->parent, a->zc, a->L, T, a->lev, a->side, s);
    return 0;
}

int ad_run_l2p(AdState* a, int prec, int p, int basis, const DevTables& T, double* pot, double* ax, double* ay, double* az,
               cudaStream_t s) {
    if (a->n == 0) return 0;
    ad_l2p_leaf(prec, p, basis, a->nleaf, a->leaf, a->nb, a->ne, a->zc, a->xs, a->ys, a->zs, a->pos32, a->perm, a->L,
                T, pot, ax, ay, az, a->lev, a->side, s);
    return 0;
}

int ad_run_p2p(AdState* a, int prec, int sms, double* pot, double* ax, double* ay, double* az, cudaStream_t s) {
    if (a->n == 0) return 0;
    cudaMemsetAsync(a->counter + 1, 0, 4, s);
    if (prec)
        ad_p2p32(a->nleaf, a->leaf, a->poff, a->psrc, a->nb, a->ne, a->ic, a->scale32, a->pos32, a->perm, pot, ax, ay,
                 az, a->counter + 1, 8 * sms, s);
    else
        ad_p2p(a->nleaf, a->leaf, a->poff, a->psrc, a->nb, a->ne, a->zc, a->xs, a->ys, a->zs, a->qs, a->perm, pot,
               ax, ay, az, a->counter + 1, 4 * sms, s);
    return 0;
}

// ---------------------------------------------------------------------------
// learned per-pair order
// ---------------------------------------------------------------------------
int ad_learn_prepare(AdState* a, cudaStream_t s) {
    const size_t nn = (size_t)(a->nn > 0 ? a->nn : 1), np = (size_t)(a->nm2l > 0 ? a->nm2l : 1);
    GROW(a->ptgt, a->cap_ptgt, np * 4);
    GROW(a->nodeF, a->cap_nodeF, nn * 32);
    GROW(a->porder, a->cap_porder, np);
    GROW(a->iota, a->cap_iota, nn * 4);
    GROW(a->bcnt, a->cap_bcnt, (FMM_PMAX + 1) * nn * 4 + 4);
    GROW(a->boff, a->cap_boff, (FMM_PMAX + 1) * nn * 4 + 4);
    GROW(a->bsrc, a->cap_bsrc, np * 4);
    GROW(a->fsum, a->cap_fsum, 2 * nn * 4);
    GROW(a->nodeK, a->cap_nodeK, nn * 4);
    if (a->nn > 0) {
        ad_pair_targets_launch(a->nn, a->nm2l, a->moff, a->ptgt, s);
        ad_iota(a->nn, a->iota, s);
    }
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

// M2L with one order per pair: the model (or the caller's orders) gives the
// order, the pairs are grouped by (order, target) with a stable sort, and
// one list M2L per order accumulates the rank prefix |n| + |m| <= q of Eq.
// M2L into the order-p local expansions.
int ad_run_m2l_orders(AdState* a, int p, int basis, int prec, int sms, const unsigned char* mlp, float thr, int* err,
                      cudaStream_t s) {
    if (a->n == 0) return 0;
    cudaMemsetAsync(a->L, 0, (size_t)a->nn * a->nc * 8, s);
    if (prec) ad_to_f32_rows(a->nn, a->nc, ld32_of(a->nc), a->M, a->M32, s);
    if (a->nm2l == 0) return 0;
    if (!a->orders_fixed) {
        ad_node_features(a, s);
        ad_far_estimate(a, s);
        mlp_orders_dev(mlp, a, thr, p, sms, err, s);
        a->orders_chosen = true;
    }
    ad_order_keys(a->nm2l, a->porder, a->k0, a->v0, s);
    if (int r = sort_pairs(a, a->nm2l, 4, s)) return r;
    const int nb = p + 1;
    cudaMemsetAsync(a->bcnt, 0, (size_t)nb * a->nn * 4 + 4, s);
    ad_bucket_csr(a->nm2l, a->nn, a->k0, a->v0, a->ptgt, a->msrc, a->bsrc, a->bcnt, s);
    scan_excl_int(a->bcnt, a->boff, (int64_t)nb * a->nn, a->scr, s);
    cudaMemsetAsync(a->counter + 2, 0, (size_t)nb * 4, s);
    const void* M = prec ? (const void*)a->M32 : (const void*)a->M;
    const int blocks = a->m2l_blocks > 0 ? a->m2l_blocks : 2 * sms;
    for (int q = 0; q < nb; ++q)
        launch_m2l_list(q, basis, prec ? 1 : 0, a->nn, a->iota, a->boff + (size_t)q * a->nn, a->bsrc, a->zc, a->ic,
                        a->scale32, M, prec ? ld32_of(a->nc) : a->nc, a->L, a->nc, 1, a->counter + 2 + q, blocks, s);
    return 0;
}

// pairs per order 0..p of the last grouping (host, synchronises)
int ad_order_counts(AdState* a, int p, int64_t* out, cudaStream_t s) {
    const int nb = p + 1;
    std::vector<int> h(nb + 1, 0);
    if (a->nm2l > 0 && a->boff) {
        for (int q = 0; q <= nb; ++q)
            cudaMemcpyAsync(&h[q], a->boff + (size_t)q * a->nn, 4, cudaMemcpyDeviceToHost, s);
        if (cudaStreamSynchronize(s) != cudaSuccess) return -2;
    }
    for (int q = 0; q < nb; ++q) out[q] = h[q + 1] - h[q];
    return 0;
}

}  // namespace fmm
