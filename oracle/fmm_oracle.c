/*
 * fmm_oracle.c -- plain FP64 CPU oracle for the Cartesian FMM operators of
 * Coles & Bieri, "An Optimizing Symbolic Algebra Approach for Generating Fast
 * Multipole Method Operators" (arXiv:1811.06332).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * restatement of the paper's equations against which the CUDA library is
 * checked.  Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline /
 * reference leg may load it.  The CUDA library never links, includes or calls
 * anything here, and nothing here is shared with it.
 *
 * Conventions (each one a reading of the paper where it leaves a choice open):
 *  - multi-index notation of App. D: n = (nx,ny,nz), |n| = nx+ny+nz,
 *    n! = nx! ny! nz!, r^n = x^nx y^ny z^nz; a negative component makes the
 *    whole term zero.
 *  - symmetric ("totally symmetric", compressed) storage, App. A: ranks 0..p
 *    concatenated; inside rank j the (j+1)(j+2)/2 components are ordered by
 *    descending nx, then descending ny.
 *  - traceless storage (Sec. 2.1 / App. B: only independent components are
 *    kept): inside rank j the 2j+1 components with nz <= 1, ordered
 *    (j,0,0),(j-1,1,0),...,(0,j,0),(j-1,0,1),...,(0,j-1,1).  Dependent
 *    components come from the trace condition A_{k+2ez} = -A_{k+2ex} - A_{k+2ey}.
 *  - normalisation of the main text (Sec. 2.1): M_n = sum_a q_a (-r_a)^n,
 *    M2L with 1/m!, L2L with delta^k/k!, L2P reads L_n at the particle.
 *  - the P2M sign printed as "-r_a^n" is read as (-r_a)^n (App. B, Eq.
 *    multipole v1 carries (-1)^n r_a^n).
 *  - output sign: pot = -Phi_paper (astrophysical sign, Sec. 2.1 last
 *    paragraph), acc = +grad Phi_paper = sum_j q_j (x_j - x_i)/|x_j - x_i|^3.
 *  - self-interaction excluded, no softening, coincident pairs skipped.
 *
 * Everything is double precision and straightforward loops; OpenMP is used
 * only to spread independent targets over host cores.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PMAX 12
#define NS_MAX 455 /* C(12+3,3) */
#define NT_MAX 169 /* (12+1)^2  */

/* ------------------------------------------------------------------------ */
/* Multi-index tables (App. D; storage sizes of the table in App. E)         */
/* ------------------------------------------------------------------------ */
static int g_init = 0;
static int g_sym[NS_MAX][3];                       /* sym index -> n     */
static int g_tl[NT_MAX][3];                        /* tl index  -> n     */
static int g_pos_sym[ORC_PMAX + 1][ORC_PMAX + 1][ORC_PMAX + 1];
static int g_pos_tl[ORC_PMAX + 1][ORC_PMAX + 1][ORC_PMAX + 1];
static double g_fact[4 * ORC_PMAX + 4];

__attribute__((constructor)) static void orc_init(void) {
    if (g_init) return;
    int c = 0;
    for (int j = 0; j <= ORC_PMAX; ++j)
        for (int nx = j; nx >= 0; --nx)
            for (int ny = j - nx; ny >= 0; --ny) {
                int nz = j - nx - ny;
                g_sym[c][0] = nx; g_sym[c][1] = ny; g_sym[c][2] = nz;
                g_pos_sym[nx][ny][nz] = c;
                ++c;
            }
    for (int a = 0; a <= ORC_PMAX; ++a)
        for (int b = 0; b <= ORC_PMAX; ++b)
            for (int d = 0; d <= ORC_PMAX; ++d) g_pos_tl[a][b][d] = -1;
    c = 0;
    for (int j = 0; j <= ORC_PMAX; ++j) {
        for (int ny = 0; ny <= j; ++ny) {           /* nz = 0 */
            g_tl[c][0] = j - ny; g_tl[c][1] = ny; g_tl[c][2] = 0;
            g_pos_tl[j - ny][ny][0] = c; ++c;
        }
        for (int ny = 0; ny <= j - 1; ++ny) {       /* nz = 1 */
            g_tl[c][0] = j - 1 - ny; g_tl[c][1] = ny; g_tl[c][2] = 1;
            g_pos_tl[j - 1 - ny][ny][1] = c; ++c;
        }
    }
    g_fact[0] = 1.0;
    for (int i = 1; i < 4 * ORC_PMAX + 4; ++i) g_fact[i] = g_fact[i - 1] * i;
    g_init = 1;
}

int orc_pmax(void) { return ORC_PMAX; }
int orc_ncoef_sym(int p) { return (p + 1) * (p + 2) * (p + 3) / 6; }
int orc_ncoef_tl(int p) { return (p + 1) * (p + 1); }
int orc_ncoef(int p, int basis) { return basis ? orc_ncoef_tl(p) : orc_ncoef_sym(p); }

/* Copies the multi-indices of the storage order into out[3*ncoef]. */
int orc_indices(int p, int basis, int* out) {
    orc_init();
    if (p < 0 || p > ORC_PMAX) return -1;
    int nc = orc_ncoef(p, basis);
    for (int i = 0; i < nc; ++i)
        for (int d = 0; d < 3; ++d) out[3 * i + d] = basis ? g_tl[i][d] : g_sym[i][d];
    return nc;
}

static double mfact(int nx, int ny, int nz) { return g_fact[nx] * g_fact[ny] * g_fact[nz]; }

/* (2k-1)!! for k >= 0, with (-1)!! = 1 */
static double dfact_odd(int k) {
    double v = 1.0;
    for (int i = 2 * k - 1; i > 1; i -= 2) v *= i;
    return v;
}

static double ipow(double x, int e) {
    double v = 1.0;
    for (int i = 0; i < e; ++i) v *= x;
    return v;
}

/* f_{n,m} of Eq. Detracer (App. A):
 * (-1)^|m| (2|n|-2|m|-1)!! n! / (2^|m| m! (n-2m)!)  for m <= floor(n/2). */
static double f_nm(const int n[3], const int m[3]) {
    int nn = n[0] + n[1] + n[2], mm = m[0] + m[1] + m[2];
    double v = dfact_odd(nn - mm) * mfact(n[0], n[1], n[2]) /
               (ldexp(1.0, mm) * mfact(m[0], m[1], m[2]) *
                mfact(n[0] - 2 * m[0], n[1] - 2 * m[1], n[2] - 2 * m[2]));
    return (mm & 1) ? -v : v;
}

/* Expands traceless storage into full symmetric storage, ranks 0..p, using
 * the trace condition (App. B: dependent elements are rebuilt from the trace,
 * e.g. A_zz = -A_xx - A_yy).  Symmetric order visits both right-hand sides
 * before the left-hand side. */
static void tl_to_sym(int p, const double* Atl, double* A) {
    int ns = orc_ncoef_sym(p);
    for (int i = 0; i < ns; ++i) {
        int nx = g_sym[i][0], ny = g_sym[i][1], nz = g_sym[i][2];
        if (nz <= 1)
            A[i] = Atl[g_pos_tl[nx][ny][nz]];
        else
            A[i] = -A[g_pos_sym[nx + 2][ny][nz - 2]] - A[g_pos_sym[nx][ny + 2][nz - 2]];
    }
}

/* Public version for tests. */
void orc_expand_traceless(int p, const double* Atl, double* A) {
    orc_init();
    tl_to_sym(p, Atl, A);
}

/* ------------------------------------------------------------------------ */
/* Detracer (Eq. Detracer, App. A)                                           */
/* ------------------------------------------------------------------------ */
/* T[A]_n = sum_{m <= floor(n/2)} f_{n,m} A^{(n:|m|)}_{n-2m},
 * A^{(n:mm)}_k = sum_{|k'|=mm} (mm!/k'!) A_{k+2k'} (m-fold trace).
 * A and out are full symmetric rank-nrank blocks (the rank-nrank slice of the
 * symmetric storage order). */
void orc_detracer_T(int nrank, const double* A, double* out) {
    orc_init();
    int off = orc_ncoef_sym(nrank - 1); /* 0 for nrank == 0 */
    int cnt = (nrank + 1) * (nrank + 2) / 2;
    for (int i = 0; i < cnt; ++i) {
        const int* n = g_sym[off + i];
        double s = 0.0;
        for (int mx = 0; mx <= n[0] / 2; ++mx)
            for (int my = 0; my <= n[1] / 2; ++my)
                for (int mz = 0; mz <= n[2] / 2; ++mz) {
                    int m[3] = {mx, my, mz};
                    int mm = mx + my + mz;
                    double tr = 0.0;
                    for (int kx = mm; kx >= 0; --kx)
                        for (int ky = mm - kx; ky >= 0; --ky) {
                            int kz = mm - kx - ky;
                            int ix = n[0] - 2 * mx + 2 * kx;
                            int iy = n[1] - 2 * my + 2 * ky;
                            int iz = n[2] - 2 * mz + 2 * kz;
                            tr += g_fact[mm] / mfact(kx, ky, kz) *
                                  A[g_pos_sym[ix][iy][iz] - off];
                        }
                    s += f_nm(n, m) * tr;
                }
        out[i] = s;
    }
}

/* D[A] = T[A] / (2n-1)!!  (App. A, the idempotent detracer). */
void orc_detracer_D(int nrank, const double* A, double* out) {
    orc_detracer_T(nrank, A, out);
    double s = 1.0 / dfact_odd(nrank);
    int cnt = (nrank + 1) * (nrank + 2) / 2;
    for (int i = 0; i < cnt; ++i) out[i] *= s;
}

/* Applies D[] rank by rank to a full symmetric polytensor (ranks 0..p). */
static void detrace_polytensor(int p, const double* A, double* out) {
    for (int j = 0; j <= p; ++j) {
        int off = orc_ncoef_sym(j - 1);
        orc_detracer_D(j, A + off, out + off);
    }
}

/* Writes (basis 1) the independent components of a full symmetric
 * polytensor, or (basis 0) all of them, adding into dst. */
static void add_out(int p, int basis, const double* Afull, double* dst) {
    if (!basis) {
        int ns = orc_ncoef_sym(p);
        for (int i = 0; i < ns; ++i) dst[i] += Afull[i];
    } else {
        int nt = orc_ncoef_tl(p);
        for (int i = 0; i < nt; ++i) dst[i] += Afull[g_pos_sym[g_tl[i][0]][g_tl[i][1]][g_tl[i][2]]];
    }
}

static void to_full(int p, int basis, const double* A, double* Afull) {
    if (basis)
        tl_to_sym(p, A, Afull);
    else
        memcpy(Afull, A, sizeof(double) * orc_ncoef_sym(p));
}

/* ------------------------------------------------------------------------ */
/* D-tensor: traceless gradient of 1/r (Eq. traceless grad and Eq.          */
/* Detracer3, App. A):                                                       */
/*   D_n(r) = grad^n r^{-1} = (-1)^|n| r^{-2|n|-1} T[r^n]_n,                 */
/*   T[r^n]_n = sum_{m <= floor(n/2)} f_{n,m} r^{2|m|} r^{n-2m}.             */
/* ------------------------------------------------------------------------ */
void orc_dtensor(int p, const double r[3], double* D) {
    orc_init();
    double x = r[0], y = r[1], z = r[2];
    double r2 = x * x + y * y + z * z;
    double rn = sqrt(r2);
    int ns = orc_ncoef_sym(p);
    for (int i = 0; i < ns; ++i) {
        const int* n = g_sym[i];
        int nn = n[0] + n[1] + n[2];
        double s = 0.0;
        for (int mx = 0; mx <= n[0] / 2; ++mx)
            for (int my = 0; my <= n[1] / 2; ++my)
                for (int mz = 0; mz <= n[2] / 2; ++mz) {
                    int m[3] = {mx, my, mz};
                    int mm = mx + my + mz;
                    s += f_nm(n, m) * ipow(r2, mm) * ipow(x, n[0] - 2 * mx) *
                         ipow(y, n[1] - 2 * my) * ipow(z, n[2] - 2 * mz);
                }
        double pre = pow(rn, -(2.0 * nn + 1.0));
        D[i] = ((nn & 1) ? -pre : pre) * s;
    }
}

void orc_dtensor_batch(int p, int64_t n, const double* rx, const double* ry,
                       const double* rz, double* D /* [ns][n] */) {
    orc_init();
    int ns = orc_ncoef_sym(p);
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < n; ++t) {
        double r[3] = {rx[t], ry[t], rz[t]}, d[NS_MAX];
        orc_dtensor(p, r, d);
        for (int i = 0; i < ns; ++i) D[(int64_t)i * n + t] = d[i];
    }
}

/* ------------------------------------------------------------------------ */
/* P2M (Eq. P2M, Sec. 2.1; App. B Eq. multipole v1 for the sign):            */
/*   M_n = sum_a q_a (-r_a)^n,  r_a = x_a - z_A;   traceless: Mbar = D[M].    */
/* M is added into (accumulate).                                             */
/* ------------------------------------------------------------------------ */
void orc_p2m(int p, int basis, int64_t na, const double* x, const double* y,
             const double* z, const double* q, const double zc[3], double* M) {
    orc_init();
    int ns = orc_ncoef_sym(p);
    double Ms[NS_MAX];
    for (int i = 0; i < ns; ++i) Ms[i] = 0.0;
    for (int64_t a = 0; a < na; ++a) {
        double ra[3] = {x[a] - zc[0], y[a] - zc[1], z[a] - zc[2]};
        for (int i = 0; i < ns; ++i) {
            const int* n = g_sym[i];
            Ms[i] += q[a] * ipow(-ra[0], n[0]) * ipow(-ra[1], n[1]) * ipow(-ra[2], n[2]);
        }
    }
    if (basis) {
        double Mt[NS_MAX];
        detrace_polytensor(p, Ms, Mt);
        add_out(p, basis, Mt, M);
    } else {
        add_out(p, basis, Ms, M);
    }
}

/* ------------------------------------------------------------------------ */
/* M2M (Eq. M2M and Eq. M2M part 2, Sec. 2.1):                               */
/*   M'_n(z' = z - delta) = sum_{k <= n} n!/(k!(n-k)!) (-delta)^{n-k} M_k(z)  */
/*   traceless: Mbar(z') = D[M'].   Result is added into Mp.                  */
/* ------------------------------------------------------------------------ */
void orc_m2m(int p, int basis, const double* Mc, const double delta[3], double* Mp) {
    orc_init();
    int ns = orc_ncoef_sym(p);
    double Ms[NS_MAX], Mn[NS_MAX];
    to_full(p, basis, Mc, Ms);
    double md[3] = {-delta[0], -delta[1], -delta[2]};
    for (int i = 0; i < ns; ++i) {
        const int* n = g_sym[i];
        double s = 0.0;
        for (int kx = 0; kx <= n[0]; ++kx)
            for (int ky = 0; ky <= n[1]; ++ky)
                for (int kz = 0; kz <= n[2]; ++kz) {
                    double binom = mfact(n[0], n[1], n[2]) /
                                   (mfact(kx, ky, kz) * mfact(n[0] - kx, n[1] - ky, n[2] - kz));
                    s += binom * ipow(md[0], n[0] - kx) * ipow(md[1], n[1] - ky) *
                         ipow(md[2], n[2] - kz) * Ms[g_pos_sym[kx][ky][kz]];
                }
        Mn[i] = s;
    }
    if (basis) {
        double Mt[NS_MAX];
        detrace_polytensor(p, Mn, Mt);
        add_out(p, basis, Mt, Mp);
    } else {
        add_out(p, basis, Mn, Mp);
    }
}

/* ------------------------------------------------------------------------ */
/* Fused traceless M2M (Eq. Detracer2, Sec. 2.1): the shift of Eq. M2M part  */
/* 2 inserted into the detracer of Eq. M2M and the terms regrouped by the    */
/* multipole component q.  Read (its printed symbols are partly garbled) as  */
/* the form that equals D[shift]: with j = n + 2k - 2m - q,                   */
/*   Mbar'_n = 1/(2n-1)!! sum_{|q| <= |n|} (Mbar_q / q!)                      */
/*             sum_{m <= floor(n/2)} f_{n,m} sum_{|k| = |m|} (|m|!/k!)        */
/*             ((j + q)!/j!) (-delta)^j          (terms with j >= 0)          */
/* whose q = 0 term is Mbar_0 D[(-delta)^n]_n.  Mbar_q runs over every        */
/* component (dependent ones from the trace condition).  Traceless storage  */
/* in and out; the independent outputs are added into Mp.                   */
/* ------------------------------------------------------------------------ */
void orc_m2m_fused(int p, const double* Mc, const double delta[3], double* Mp) {
    orc_init();
    int ns = orc_ncoef_sym(p), nt = orc_ncoef_tl(p);
    double Ms[NS_MAX];
    tl_to_sym(p, Mc, Ms);
    double md[3] = {-delta[0], -delta[1], -delta[2]};
    for (int t = 0; t < nt; ++t) {
        const int* n = g_tl[t];
        int nn = n[0] + n[1] + n[2];
        double s = 0.0;
        for (int iq = 0; iq < ns; ++iq) {
            const int* q = g_sym[iq];
            if (q[0] + q[1] + q[2] > nn) continue;
            double inner = 0.0;
            for (int mx = 0; mx <= n[0] / 2; ++mx)
                for (int my = 0; my <= n[1] / 2; ++my)
                    for (int mz = 0; mz <= n[2] / 2; ++mz) {
                        int m[3] = {mx, my, mz};
                        int mm = mx + my + mz;
                        double fm = f_nm(n, m);
                        for (int kx = mm; kx >= 0; --kx)
                            for (int ky = mm - kx; ky >= 0; --ky) {
                                int kz = mm - kx - ky;
                                int j[3] = {n[0] + 2 * kx - 2 * mx - q[0], n[1] + 2 * ky - 2 * my - q[1],
                                            n[2] + 2 * kz - 2 * mz - q[2]};
                                if (j[0] < 0 || j[1] < 0 || j[2] < 0) continue;
                                double w = fm * g_fact[mm] / mfact(kx, ky, kz) *
                                           mfact(j[0] + q[0], j[1] + q[1], j[2] + q[2]) / mfact(j[0], j[1], j[2]);
                                inner += w * ipow(md[0], j[0]) * ipow(md[1], j[1]) * ipow(md[2], j[2]);
                            }
                    }
            s += Ms[iq] / mfact(q[0], q[1], q[2]) * inner;
        }
        Mp[t] += s / dfact_odd(nn);
    }
}

/* ------------------------------------------------------------------------ */
/* M2L (Eq. M2L, Sec. 2.1):                                                  */
/*   L_n(z' = z + r) += sum_{|m| <= p-|n|} (1/m!) M_m(z) D_{n+m}(r)           */
/* D is the full symmetric D-tensor up to rank p (orc_dtensor).              */
/* ------------------------------------------------------------------------ */
void orc_m2l_D(int p, int basis, const double* M, const double* D, double* L) {
    orc_init();
    int ns = orc_ncoef_sym(p);
    double Ms[NS_MAX], Ls[NS_MAX];
    to_full(p, basis, M, Ms);
    for (int i = 0; i < ns; ++i) {
        const int* n = g_sym[i];
        int nn = n[0] + n[1] + n[2];
        double s = 0.0;
        if (basis && n[2] >= 2) { Ls[i] = 0.0; continue; } /* dependent output */
        int nm = orc_ncoef_sym(p - nn);
        for (int k = 0; k < nm; ++k) {
            const int* m = g_sym[k];
            s += Ms[k] / mfact(m[0], m[1], m[2]) *
                 D[g_pos_sym[n[0] + m[0]][n[1] + m[1]][n[2] + m[2]]];
        }
        Ls[i] = s;
    }
    add_out(p, basis, Ls, L);
}

void orc_m2l(int p, int basis, const double* M, const double r[3], double* L) {
    double D[NS_MAX];
    orc_dtensor(p, r, D);
    orc_m2l_D(p, basis, M, D, L);
}

/* Batched M2L over independent pairs: M [ncoef][n], offsets r [3][n] (SoA),
 * L [ncoef][n] accumulated (or overwritten when accumulate == 0). */
void orc_m2l_batch(int p, int basis, int64_t n, const double* M, const double* rx,
                   const double* ry, const double* rz, double* L, int accumulate) {
    orc_init();
    int nc = orc_ncoef(p, basis);
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < n; ++t) {
        double m[NS_MAX], l[NS_MAX], r[3] = {rx[t], ry[t], rz[t]};
        for (int i = 0; i < nc; ++i) {
            m[i] = M[(int64_t)i * n + t];
            l[i] = accumulate ? L[(int64_t)i * n + t] : 0.0;
        }
        orc_m2l(p, basis, m, r, l);
        for (int i = 0; i < nc; ++i) L[(int64_t)i * n + t] = l[i];
    }
}

/* ------------------------------------------------------------------------ */
/* L2L (Eq. L2L, Sec. 2.1):                                                  */
/*   L_n(z' = z + delta) += sum_{|k| <= p-|n|} delta^k/k! L_{n+k}(z)          */
/* ------------------------------------------------------------------------ */
void orc_l2l(int p, int basis, const double* Lp, const double delta[3], double* Lc) {
    orc_init();
    int ns = orc_ncoef_sym(p);
    double Ls[NS_MAX], Ln[NS_MAX];
    to_full(p, basis, Lp, Ls);
    for (int i = 0; i < ns; ++i) {
        const int* n = g_sym[i];
        int nn = n[0] + n[1] + n[2];
        int nk = orc_ncoef_sym(p - nn);
        double s = 0.0;
        for (int k = 0; k < nk; ++k) {
            const int* kk = g_sym[k];
            s += ipow(delta[0], kk[0]) * ipow(delta[1], kk[1]) * ipow(delta[2], kk[2]) /
                 mfact(kk[0], kk[1], kk[2]) *
                 Ls[g_pos_sym[n[0] + kk[0]][n[1] + kk[1]][n[2] + kk[2]]];
        }
        Ln[i] = s;
    }
    add_out(p, basis, Ln, Lc);
}

/* ------------------------------------------------------------------------ */
/* L2P (Eq. L2P, Sec. 2.1): shift L to the particle (delta = r_b) and read   */
/* the rank-0 and rank-1 components:                                         */
/*   Phi = sum_{|k|<=p} r_b^k/k! L_k,  dPhi/dx_i = sum_{|k|<=p-1} r_b^k/k! L_{k+e_i}. */
/* out[0] = Phi, out[1..3] = grad Phi (paper's positive-potential sign).     */
/* ------------------------------------------------------------------------ */
void orc_l2p(int p, int basis, const double* L, const double rb[3], double out[4]) {
    orc_init();
    double Ls[NS_MAX];
    to_full(p, basis, L, Ls);
    int ns = orc_ncoef_sym(p);
    double phi = 0.0, g[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < ns; ++k) {
        const int* kk = g_sym[k];
        int nk = kk[0] + kk[1] + kk[2];
        double w = ipow(rb[0], kk[0]) * ipow(rb[1], kk[1]) * ipow(rb[2], kk[2]) /
                   mfact(kk[0], kk[1], kk[2]);
        phi += w * Ls[k];
        if (nk <= p - 1) {
            g[0] += w * Ls[g_pos_sym[kk[0] + 1][kk[1]][kk[2]]];
            g[1] += w * Ls[g_pos_sym[kk[0]][kk[1] + 1][kk[2]]];
            g[2] += w * Ls[g_pos_sym[kk[0]][kk[1]][kk[2] + 1]];
        }
    }
    out[0] = phi; out[1] = g[0]; out[2] = g[1]; out[3] = g[2];
}

/* ------------------------------------------------------------------------ */
/* Direct sum (Eq. PhiAB, App. B) with the output sign convention above.     */
/* targets == NULL means every particle; otherwise nt indices.               */
/* ------------------------------------------------------------------------ */
void orc_direct(int64_t n, const double* x, const double* y, const double* z,
                const double* q, int64_t nt, const int64_t* targets, double* pot,
                double* ax, double* ay, double* az) {
    int64_t cnt = targets ? nt : n;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < cnt; ++t) {
        int64_t i = targets ? targets[t] : t;
        double ph = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double dx = x[j] - x[i], dy = y[j] - y[i], dz = z[j] - z[i];
            double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 == 0.0) continue;
            double ir = 1.0 / sqrt(r2);
            double ir3 = ir * ir * ir;
            ph += q[j] * ir;
            gx += q[j] * dx * ir3; gy += q[j] * dy * ir3; gz += q[j] * dz * ir3;
        }
        pot[t] = -ph; ax[t] = gx; ay[t] = gy; az[t] = gz;
    }
}

/* ------------------------------------------------------------------------ */
/* Point dipoles (App. B, "Dipoles and higher order multipoles").  A point   */
/* dipole p at x_a is read as the limit of charges +q at x_a + s and -q at    */
/* x_a - s with p = 2 q s.  About x_a its multipole (Eq. P2M, M_n =           */
/* sum q (-r_a)^n) is the pure dipole M_{e_i} = -p_i, every other component  */
/* zero; P2M of dipoles shifts that pure dipole to the expansion centre with */
/* M2M (Eq. M2M), delta = x_a - z_A (child: the dipole's own centre).  A      */
/* rank-1 tensor is traceless, so the traceless shift applies as it is.      */
/* Added into M.                                                             */
/* ------------------------------------------------------------------------ */
void orc_p2m_dipole(int p, int basis, int64_t na, const double* x, const double* y, const double* z,
                    const double* px, const double* py, const double* pz, const double zc[3], double* M) {
    orc_init();
    int nc = orc_ncoef(p, basis);
    double Md[NS_MAX];
    for (int64_t a = 0; a < na; ++a) {
        for (int i = 0; i < nc; ++i) Md[i] = 0.0;
        if (p >= 1) {
            const double pv[3] = {px[a], py[a], pz[a]};
            for (int d = 0; d < 3; ++d) {
                const int e[3] = {d == 0, d == 1, d == 2};
                const int pos = basis ? g_pos_tl[e[0]][e[1]][e[2]] : g_pos_sym[e[0]][e[1]][e[2]];
                Md[pos] = -pv[d];
            }
        }
        const double delta[3] = {x[a] - zc[0], y[a] - zc[1], z[a] - zc[2]};
        orc_m2m(p, basis, Md, delta, M);
    }
}

/* Potential and gradient of sources with charges q and dipoles (px, py, pz) */
/* at x_i (the paper's positive Phi): a charge adds q/|d|, a dipole          */
/* p.d/|d|^3, d = x_i - x_j; gradients -q d/|d|^3 and p/|d|^3 -             */
/* 3 (p.d) d/|d|^5.  Output sign convention as orc_direct: pot = -Phi,       */
/* acc = grad Phi.  targets == NULL: every particle.                         */
void orc_direct_dipole(int64_t n, const double* x, const double* y, const double* z, const double* q,
                       const double* px, const double* py, const double* pz, int64_t nt, const int64_t* targets,
                       double* pot, double* ax, double* ay, double* az) {
    int64_t cnt = targets ? nt : n;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < cnt; ++t) {
        int64_t i = targets ? targets[t] : t;
        double ph = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double d[3] = {x[i] - x[j], y[i] - y[j], z[i] - z[j]};
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (r2 == 0.0) continue;
            double ir = 1.0 / sqrt(r2), ir3 = ir * ir * ir, ir5 = ir3 * ir * ir;
            double pd = px[j] * d[0] + py[j] * d[1] + pz[j] * d[2];
            ph += q[j] * ir + pd * ir3;
            gx += -q[j] * d[0] * ir3 + px[j] * ir3 - 3.0 * pd * d[0] * ir5;
            gy += -q[j] * d[1] * ir3 + py[j] * ir3 - 3.0 * pd * d[1] * ir5;
            gz += -q[j] * d[2] * ir3 + pz[j] * ir3 - 3.0 * pd * d[2] * ir5;
        }
        pot[t] = -ph; ax[t] = gx; ay[t] = gy; az[t] = gz;
    }
}

/* ------------------------------------------------------------------------ */
/* Uniform-octree FMM (App. C, with the octree and "standard" separation     */
/* criterion of the uniform workloads): leaves at level `depth` of the unit   */
/* cube [0,1)^3, leaf of a particle i_d = min(floor(x_d 2^depth), 2^depth-1).  */
/* Same-level cells are well separated when their Chebyshev index distance   */
/* is >= 2; the interaction list of a cell is the children of its parent's  */
/* neighbours (parent included) that are not adjacent to it; M2L runs at     */
/* levels 2..depth; adjacent leaves (self included) are summed directly.     */
/* Expansion centres are geometric cell centres (App. C).                    */
/* If nsample >= 0 only the particles listed in sample[] are evaluated       */
/* (outputs have nsample entries, in that order); otherwise all n, in the    */
/* caller's order.                                                           */
/* ------------------------------------------------------------------------ */
typedef struct {
    int depth, p, basis, nc;
    int64_t n;
    const double *x, *y, *z, *q;
    int64_t* leaf_start; /* [nleaf+1] */
    int64_t* order;      /* particles sorted by leaf, stable */
    double** M;          /* per level, [ncell][nc] */
    double** L;
} uni_t;

static inline int64_t cell_id(int l, int ix, int iy, int iz) {
    int64_t s = (int64_t)1 << l;
    return ((int64_t)iz * s + iy) * s + ix;
}

static void cell_centre(int l, int ix, int iy, int iz, double c[3]) {
    double h = ldexp(1.0, -l);
    c[0] = (ix + 0.5) * h; c[1] = (iy + 0.5) * h; c[2] = (iz + 0.5) * h;
}

static int leaf_coord(double v, int side) {
    int i = (int)floor(v * side);
    if (i < 0) i = 0;
    if (i > side - 1) i = side - 1;
    return i;
}

static int fmm_uniform_impl(int64_t n, const double* x, const double* y, const double* z, const double* q,
                            const double* px, const double* py, const double* pz, int depth, int p, int basis,
                            int64_t nsample, const int64_t* sample, double* pot, double* ax, double* ay,
                            double* az) {
    orc_init();
    if (p < 0 || p > ORC_PMAX || depth < 0 || depth > 10 || basis < 0 || basis > 2) return -1;
    int side = 1 << depth;
    int64_t nleaf = (int64_t)side * side * side;
    /* basis 2, the TG variant (Sec. 3): multipoles in full symmetric storage
       (P2M, M2M without a detracer), M2L from them to a traceless local
       expansion (D is traceless, so is L; its independent components are
       kept), L2L and L2P on traceless storage */
    const int tg = basis == 2;
    const int bM = tg ? 0 : basis, bL = tg ? 1 : basis;
    int nc = orc_ncoef(p, bM) > orc_ncoef(p, bL) ? orc_ncoef(p, bM) : orc_ncoef(p, bL);
    uni_t U;
    U.depth = depth; U.p = p; U.basis = basis; U.nc = nc; U.n = n;
    U.x = x; U.y = y; U.z = z; U.q = q;

    /* leaf assignment and stable bucket sort */
    int64_t* leaf = (int64_t*)malloc(sizeof(int64_t) * (n > 0 ? n : 1));
    U.leaf_start = (int64_t*)calloc(nleaf + 1, sizeof(int64_t));
    U.order = (int64_t*)malloc(sizeof(int64_t) * (n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) {
        leaf[i] = cell_id(depth, leaf_coord(x[i], side), leaf_coord(y[i], side),
                          leaf_coord(z[i], side));
        U.leaf_start[leaf[i] + 1]++;
    }
    for (int64_t c = 0; c < nleaf; ++c) U.leaf_start[c + 1] += U.leaf_start[c];
    {
        int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * nleaf);
        memcpy(fill, U.leaf_start, sizeof(int64_t) * nleaf);
        for (int64_t i = 0; i < n; ++i) U.order[fill[leaf[i]]++] = i;
        free(fill);
    }

    /* which leaves / cells are needed (sampled mode) */
    char** need = (char**)malloc(sizeof(char*) * (depth + 1));
    for (int l = 0; l <= depth; ++l) {
        int64_t nce = (int64_t)1 << (3 * l);
        need[l] = (char*)calloc(nce, 1);
    }
    int64_t ntarg = nsample >= 0 ? nsample : n;
    for (int64_t t = 0; t < ntarg; ++t) {
        int64_t i = nsample >= 0 ? sample[t] : t;
        int ix = leaf_coord(x[i], side), iy = leaf_coord(y[i], side), iz = leaf_coord(z[i], side);
        for (int l = depth; l >= 0; --l) {
            need[l][cell_id(l, ix, iy, iz)] = 1;
            ix >>= 1; iy >>= 1; iz >>= 1;
        }
    }

    /* upward pass: P2M at leaves, M2M bottom-up (App. C) */
    U.M = (double**)malloc(sizeof(double*) * (depth + 1));
    U.L = (double**)malloc(sizeof(double*) * (depth + 1));
    for (int l = 0; l <= depth; ++l) {
        int64_t nce = (int64_t)1 << (3 * l);
        U.M[l] = (double*)calloc(nce * nc, sizeof(double));
        U.L[l] = (double*)calloc(nce * nc, sizeof(double));
    }
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t c = 0; c < nleaf; ++c) {
        int64_t b = U.leaf_start[c], e = U.leaf_start[c + 1];
        if (b == e) continue;
        int ix = (int)(c % side), iy = (int)((c / side) % side), iz = (int)(c / ((int64_t)side * side));
        double zc[3];
        cell_centre(depth, ix, iy, iz, zc);
        int64_t cnt = e - b;
        double* buf = (double*)malloc(sizeof(double) * 4 * cnt);
        for (int64_t a = 0; a < cnt; ++a) {
            int64_t i = U.order[b + a];
            buf[a] = x[i]; buf[cnt + a] = y[i]; buf[2 * cnt + a] = z[i]; buf[3 * cnt + a] = q[i];
        }
        orc_p2m(p, bM, cnt, buf, buf + cnt, buf + 2 * cnt, buf + 3 * cnt, zc, U.M[depth] + c * nc);
        if (px) {
            double* pb = (double*)malloc(sizeof(double) * 3 * cnt);
            for (int64_t a = 0; a < cnt; ++a) {
                int64_t i = U.order[b + a];
                pb[a] = px[i]; pb[cnt + a] = py[i]; pb[2 * cnt + a] = pz[i];
            }
            orc_p2m_dipole(p, bM, cnt, buf, buf + cnt, buf + 2 * cnt, pb, pb + cnt, pb + 2 * cnt, zc,
                           U.M[depth] + c * nc);
            free(pb);
        }
        free(buf);
    }
    for (int l = depth - 1; l >= 0; --l) {
        int s = 1 << l;
        int64_t nce = (int64_t)s * s * s;
#pragma omp parallel for schedule(dynamic, 16)
        for (int64_t c = 0; c < nce; ++c) {
            int ix = (int)(c % s), iy = (int)((c / s) % s), iz = (int)(c / ((int64_t)s * s));
            double zp[3];
            cell_centre(l, ix, iy, iz, zp);
            for (int ch = 0; ch < 8; ++ch) {
                int cx = 2 * ix + (ch & 1), cy = 2 * iy + ((ch >> 1) & 1), cz = 2 * iz + (ch >> 2);
                double zch[3], d[3];
                cell_centre(l + 1, cx, cy, cz, zch);
                d[0] = zch[0] - zp[0]; d[1] = zch[1] - zp[1]; d[2] = zch[2] - zp[2];
                orc_m2m(p, bM, U.M[l + 1] + cell_id(l + 1, cx, cy, cz) * nc, d, U.M[l] + c * nc);
            }
        }
    }

    /* interaction phase: M2L over the interaction lists at levels 2..depth */
    for (int l = 2; l <= depth; ++l) {
        int s = 1 << l;
        int64_t nce = (int64_t)s * s * s;
#pragma omp parallel for schedule(dynamic, 16)
        for (int64_t c = 0; c < nce; ++c) {
            if (!need[l][c]) continue;
            int ix = (int)(c % s), iy = (int)((c / s) % s), iz = (int)(c / ((int64_t)s * s));
            double zt[3];
            cell_centre(l, ix, iy, iz, zt);
            int px = ix >> 1, py = iy >> 1, pz = iz >> 1;
            for (int jz = 2 * pz - 2; jz <= 2 * pz + 3; ++jz)
                for (int jy = 2 * py - 2; jy <= 2 * py + 3; ++jy)
                    for (int jx = 2 * px - 2; jx <= 2 * px + 3; ++jx) {
                        if (jx < 0 || jy < 0 || jz < 0 || jx >= s || jy >= s || jz >= s) continue;
                        if (abs(jx - ix) <= 1 && abs(jy - iy) <= 1 && abs(jz - iz) <= 1) continue;
                        double zs[3], r[3];
                        cell_centre(l, jx, jy, jz, zs);
                        r[0] = zt[0] - zs[0]; r[1] = zt[1] - zs[1]; r[2] = zt[2] - zs[2];
                        if (tg) {
                            double Ls[NS_MAX];
                            for (int i = 0; i < NS_MAX; ++i) Ls[i] = 0.0;
                            orc_m2l(p, 0, U.M[l] + cell_id(l, jx, jy, jz) * nc, r, Ls);
                            add_out(p, 1, Ls, U.L[l] + c * nc);
                        } else {
                            orc_m2l(p, basis, U.M[l] + cell_id(l, jx, jy, jz) * nc, r, U.L[l] + c * nc);
                        }
                    }
        }
    }

    /* downward pass: L2L from level 2 to the leaves (App. C) */
    for (int l = 3; l <= depth; ++l) {
        int s = 1 << l;
        int64_t nce = (int64_t)s * s * s;
#pragma omp parallel for schedule(static)
        for (int64_t c = 0; c < nce; ++c) {
            if (!need[l][c]) continue;
            int ix = (int)(c % s), iy = (int)((c / s) % s), iz = (int)(c / ((int64_t)s * s));
            double zc[3], zp[3], d[3];
            cell_centre(l, ix, iy, iz, zc);
            cell_centre(l - 1, ix >> 1, iy >> 1, iz >> 1, zp);
            d[0] = zc[0] - zp[0]; d[1] = zc[1] - zp[1]; d[2] = zc[2] - zp[2];
            orc_l2l(p, bL, U.L[l - 1] + cell_id(l - 1, ix >> 1, iy >> 1, iz >> 1) * nc, d,
                    U.L[l] + c * nc);
        }
    }

    /* evaluation: L2P at leaves plus direct near field over adjacent leaves */
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t t = 0; t < ntarg; ++t) {
        int64_t i = nsample >= 0 ? sample[t] : t;
        int ix = leaf_coord(x[i], side), iy = leaf_coord(y[i], side), iz = leaf_coord(z[i], side);
        double zc[3], rb[3], o[4] = {0.0, 0.0, 0.0, 0.0};
        cell_centre(depth, ix, iy, iz, zc);
        rb[0] = x[i] - zc[0]; rb[1] = y[i] - zc[1]; rb[2] = z[i] - zc[2];
        if (depth >= 2) orc_l2p(p, bL, U.L[depth] + cell_id(depth, ix, iy, iz) * nc, rb, o);
        double ph = o[0], gx = o[1], gy = o[2], gz = o[3];
        for (int jz = iz - 1; jz <= iz + 1; ++jz)
            for (int jy = iy - 1; jy <= iy + 1; ++jy)
                for (int jx = ix - 1; jx <= ix + 1; ++jx) {
                    if (jx < 0 || jy < 0 || jz < 0 || jx >= side || jy >= side || jz >= side) continue;
                    int64_t lc = cell_id(depth, jx, jy, jz);
                    for (int64_t a = U.leaf_start[lc]; a < U.leaf_start[lc + 1]; ++a) {
                        int64_t j = U.order[a];
                        if (j == i) continue;
                        double dx = x[j] - x[i], dy = y[j] - y[i], dz = z[j] - z[i];
                        double r2 = dx * dx + dy * dy + dz * dz;
                        if (r2 == 0.0) continue;
                        double ir = 1.0 / sqrt(r2), ir3 = ir * ir * ir;
                        ph += q[j] * ir;
                        gx += q[j] * dx * ir3; gy += q[j] * dy * ir3; gz += q[j] * dz * ir3;
                        if (px) {   /* dipole source; d = x_i - x_j = -(dx, dy, dz) */
                            double ir5 = ir3 * ir * ir;
                            double pd = -(px[j] * dx + py[j] * dy + pz[j] * dz);
                            ph += pd * ir3;
                            gx += px[j] * ir3 + 3.0 * pd * dx * ir5;
                            gy += py[j] * ir3 + 3.0 * pd * dy * ir5;
                            gz += pz[j] * ir3 + 3.0 * pd * dz * ir5;
                        }
                    }
                }
        pot[t] = -ph; ax[t] = gx; ay[t] = gy; az[t] = gz;
    }

    for (int l = 0; l <= depth; ++l) { free(U.M[l]); free(U.L[l]); free(need[l]); }
    free(U.M); free(U.L); free(need);
    free(leaf); free(U.leaf_start); free(U.order);
    return 0;
}

int orc_fmm_uniform(int64_t n, const double* x, const double* y, const double* z,
                    const double* q, int depth, int p, int basis, int64_t nsample,
                    const int64_t* sample, double* pot, double* ax, double* ay,
                    double* az) {
    return fmm_uniform_impl(n, x, y, z, q, NULL, NULL, NULL, depth, p, basis, nsample, sample, pot, ax, ay, az);
}

/* The uniform FMM with point dipoles (px, py, pz) beside the charges q:    */
/* P2M adds the shifted pure dipoles (orc_p2m_dipole), the near field adds  */
/* the dipole terms of orc_direct_dipole; the other operators are the same. */
int orc_fmm_uniform_dipole(int64_t n, const double* x, const double* y, const double* z, const double* q,
                           const double* px, const double* py, const double* pz, int depth, int p, int basis,
                           int64_t nsample, const int64_t* sample, double* pot, double* ax, double* ay,
                           double* az) {
    return fmm_uniform_impl(n, x, y, z, q, px, py, pz, depth, p, basis, nsample, sample, pot, ax, ay, az);
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Adaptive octree FMM (App. C with an octree): the bounding cube of the      */
/* data (anchored at the coordinate minima, side = largest extent enlarged by */
/* 1e-12 relative), Morton keys with 21 bits per axis, particles sorted by    */
/* (key, index); a cell holding more than max_leaf particles is split into    */
/* its non-empty octants (children kept in octant order), down to level 21.   */
/* Expansion centres are geometric cell centres (App. C); the enclosing       */
/* radius of a leaf is the largest particle distance from its centre, of an   */
/* inner cell max over children of (|z_child - z| + r_child).                 */
/* Interaction lists come from a directed dual-tree traversal (App. C, after  */
/* Dehnen): start from (root, root); a self pair of an inner cell expands to  */
/* all ordered pairs of its children; a pair (A target, B source) is accepted */
/* for M2L when theta |z_A - z_B| > r_A + r_B (the MAC, evaluated squared), goes to P2P when both */
/* are leaves, and otherwise the larger cell (by radius; the target on ties)  */
/* is opened, or the one that is not a leaf.  theta = 0 accepts nothing, so   */
/* the method reduces to the direct sum.                                       */
/* ------------------------------------------------------------------------ */
typedef struct {
    int level, ix, iy, iz;
    int64_t b, e;          /* particle range in sorted order */
    int64_t child0;        /* first child node, -1 for leaves */
    int nchild;
    int64_t parent;
    double z[3], r;
} anode_t;

static uint64_t spread21(uint64_t v) {
    uint64_t r = 0;
    for (int j = 0; j < 21; ++j) r |= ((v >> j) & 1ull) << (3 * j);
    return r;
}

typedef struct { uint64_t key; int64_t idx; } kv_t;
static int kv_cmp(const void* a, const void* b) {
    const kv_t* p = (const kv_t*)a;
    const kv_t* q = (const kv_t*)b;
    if (p->key != q->key) return p->key < q->key ? -1 : 1;
    return p->idx < q->idx ? -1 : (p->idx > q->idx);
}

typedef struct { int64_t a, b; } pair_t;
typedef struct { pair_t* v; int64_t n, cap; } plist_t;
static void pl_push(plist_t* l, int64_t a, int64_t b) {
    if (l->n == l->cap) {
        l->cap = l->cap ? 2 * l->cap : 1024;
        l->v = (pair_t*)realloc(l->v, sizeof(pair_t) * l->cap);
    }
    l->v[l->n].a = a; l->v[l->n].b = b; l->n++;
}

static double dist3(const double* a, const double* b) {
    double dx = a[0] - b[0], dy = a[1] - b[1], dz = a[2] - b[2];
    return sqrt(dx * dx + dy * dy + dz * dz);
}

static int pair_cmp(const void* a, const void* b) {
    const pair_t* p = (const pair_t*)a;
    const pair_t* q = (const pair_t*)b;
    if (p->a != q->a) return p->a < q->a ? -1 : 1;
    return p->b < q->b ? -1 : (p->b > q->b);
}

typedef struct {
    int64_t n, nn;
    kv_t* kv;        /* particles sorted by (key, index) */
    anode_t* nd;     /* nodes, level by level (parents before children) */
    plist_t m2l;     /* (target, source), sorted by target then source */
    plist_t p2p;     /* (target leaf, source leaf), traversal order */
} atree_t;

static void atree_free(atree_t* T) {
    free(T->kv); free(T->nd); free(T->m2l.v); free(T->p2p.v);
    memset(T, 0, sizeof(*T));
}

/* Interaction lists of a built tree (T->nd with centres and radii): the
 * directed dual traversal described above. */
static void atree_lists(atree_t* T, double theta) {
    const anode_t* nd = T->nd;
    plist_t qa = {0, 0, 0}, qb = {0, 0, 0}, m2l = {0, 0, 0}, p2p = {0, 0, 0};
    pl_push(&qa, 0, 0);
    while (qa.n) {
        qb.n = 0;
        for (int64_t k = 0; k < qa.n; ++k) {
            const int64_t A = qa.v[k].a, B = qa.v[k].b;
            const int la = nd[A].nchild == 0, lb = nd[B].nchild == 0;
            if (A == B) {
                if (la) pl_push(&p2p, A, A);
                else
                    for (int i = 0; i < nd[A].nchild; ++i)
                        for (int j = 0; j < nd[A].nchild; ++j) pl_push(&qb, nd[A].child0 + i, nd[A].child0 + j);
                continue;
            }
            /* the MAC of App. C, theta |z_A - z_B| > r_A + r_B, compared squared
               (both sides are non-negative): theta^2 |z_A - z_B|^2 > (r_A + r_B)^2 */
            {
                const double dx = nd[A].z[0] - nd[B].z[0], dy = nd[A].z[1] - nd[B].z[1],
                             dz = nd[A].z[2] - nd[B].z[2];
                const double d2 = dx * dx + dy * dy + dz * dz;
                const double sr = nd[A].r + nd[B].r;
                if (theta * theta * d2 > sr * sr) { pl_push(&m2l, A, B); continue; }
            }
            if (la && lb) { pl_push(&p2p, A, B); continue; }
            if (!la && (lb || nd[A].r >= nd[B].r)) {
                for (int i = 0; i < nd[A].nchild; ++i) pl_push(&qb, nd[A].child0 + i, B);
            } else {
                for (int j = 0; j < nd[B].nchild; ++j) pl_push(&qb, A, nd[B].child0 + j);
            }
        }
        plist_t t = qa; qa = qb; qb = t;
    }
    free(qa.v); free(qb.v);
    if (m2l.n > 1) qsort(m2l.v, m2l.n, sizeof(pair_t), pair_cmp);
    T->m2l = m2l;
    T->p2p = p2p;
}

/* Octree, geometry and interaction lists as described above (n > 0).
 * com != 0 (the AP variant, Sec. 3): expansion centres are centres of mass
 * instead of geometric centres, computed bottom-up in a fixed order -- a
 * leaf sums q_a x_a and q_a over its particles in sorted order, an inner
 * cell sums Q_c z_c and Q_c over its children in octant order, z = S/Q --
 * and a cell whose total charge is 0 keeps its geometric centre.  The
 * radii and the traversal then use these centres. */
static void atree_build(atree_t* T, int64_t n, const double* x, const double* y, const double* z, const double* q,
                        int max_leaf, double theta, int com) {
    memset(T, 0, sizeof(*T));
    T->n = n;
    /* bounding cube */
    double lo[3] = {x[0], y[0], z[0]}, hi[3] = {x[0], y[0], z[0]};
    for (int64_t i = 0; i < n; ++i) {
        const double v[3] = {x[i], y[i], z[i]};
        for (int d = 0; d < 3; ++d) { if (v[d] < lo[d]) lo[d] = v[d]; if (v[d] > hi[d]) hi[d] = v[d]; }
    }
    double side = 0.0;
    for (int d = 0; d < 3; ++d) if (hi[d] - lo[d] > side) side = hi[d] - lo[d];
    if (side == 0.0) side = 1.0;
    side = side * (1.0 + 1e-12);
    const double scale = 2097152.0 / side; /* 2^21 */
    kv_t* kv = (kv_t*)malloc(sizeof(kv_t) * n);
    for (int64_t i = 0; i < n; ++i) {
        const double v[3] = {x[i], y[i], z[i]};
        uint64_t key = 0;
        for (int d = 0; d < 3; ++d) {
            int64_t c = (int64_t)floor((v[d] - lo[d]) * scale);
            if (c < 0) c = 0;
            if (c > 2097151) c = 2097151;
            key |= spread21((uint64_t)c) << d;
        }
        kv[i].key = key; kv[i].idx = i;
    }
    qsort(kv, n, sizeof(kv_t), kv_cmp);
    /* tree, level by level */
    int64_t cap = 1024, nn = 1;
    anode_t* nd = (anode_t*)malloc(sizeof(anode_t) * cap);
    nd[0].level = 0; nd[0].ix = nd[0].iy = nd[0].iz = 0; nd[0].b = 0; nd[0].e = n;
    nd[0].child0 = -1; nd[0].nchild = 0; nd[0].parent = -1;
    int64_t lvl_b = 0, lvl_e = 1;
    while (lvl_b < lvl_e) {
        for (int64_t c = lvl_b; c < lvl_e; ++c) {
            if (nd[c].e - nd[c].b <= max_leaf || nd[c].level >= 21) continue;
            const int L = nd[c].level;
            const int shift = 3 * (20 - L);
            nd[c].child0 = nn;
            int64_t s = nd[c].b;
            for (int oct = 0; oct < 8; ++oct) {
                int64_t e = s;
                while (e < nd[c].e && (int)((kv[e].key >> shift) & 7ull) == oct) ++e;
                if (e > s) {
                    if (nn == cap) { cap *= 2; nd = (anode_t*)realloc(nd, sizeof(anode_t) * cap); }
                    anode_t* ch = &nd[nn++];
                    ch->level = L + 1;
                    ch->ix = 2 * nd[c].ix + (oct & 1);
                    ch->iy = 2 * nd[c].iy + ((oct >> 1) & 1);
                    ch->iz = 2 * nd[c].iz + ((oct >> 2) & 1);
                    ch->b = s; ch->e = e; ch->child0 = -1; ch->nchild = 0; ch->parent = c;
                    nd[c].nchild++;
                }
                s = e;
            }
        }
        lvl_b = lvl_e;
        lvl_e = nn;
    }
    /* geometry: centres, radii (children after parents in the array) */
    for (int64_t c = 0; c < nn; ++c) {
        const double h = side / (double)(1ull << nd[c].level);
        nd[c].z[0] = lo[0] + (nd[c].ix + 0.5) * h;
        nd[c].z[1] = lo[1] + (nd[c].iy + 0.5) * h;
        nd[c].z[2] = lo[2] + (nd[c].iz + 0.5) * h;
    }
    if (com) {
        double* Q = (double*)calloc(nn, sizeof(double));
        for (int64_t c = nn - 1; c >= 0; --c) {   /* children follow parents: reverse order is bottom-up */
            double S[3] = {0.0, 0.0, 0.0}, Qc = 0.0;
            if (nd[c].nchild == 0) {
                for (int64_t a = nd[c].b; a < nd[c].e; ++a) {
                    const int64_t i = kv[a].idx;
                    Qc += q[i];
                    S[0] += q[i] * x[i]; S[1] += q[i] * y[i]; S[2] += q[i] * z[i];
                }
            } else {
                for (int k = 0; k < nd[c].nchild; ++k) {
                    const int64_t ch = nd[c].child0 + k;
                    Qc += Q[ch];
                    S[0] += Q[ch] * nd[ch].z[0]; S[1] += Q[ch] * nd[ch].z[1]; S[2] += Q[ch] * nd[ch].z[2];
                }
            }
            Q[c] = Qc;
            if (Qc != 0.0) { nd[c].z[0] = S[0] / Qc; nd[c].z[1] = S[1] / Qc; nd[c].z[2] = S[2] / Qc; }
        }
        free(Q);
    }
    for (int64_t c = nn - 1; c >= 0; --c) {
        double r = 0.0;
        if (nd[c].nchild == 0) {
            for (int64_t a = nd[c].b; a < nd[c].e; ++a) {
                const int64_t i = kv[a].idx;
                const double v[3] = {x[i], y[i], z[i]};
                const double d = dist3(v, nd[c].z);
                if (d > r) r = d;
            }
        } else {
            for (int k = 0; k < nd[c].nchild; ++k) {
                const anode_t* ch = &nd[nd[c].child0 + k];
                const double d = dist3(ch->z, nd[c].z) + ch->r;
                if (d > r) r = d;
            }
        }
        nd[c].r = r;
    }
    T->nn = nn; T->kv = kv; T->nd = nd;
    atree_lists(T, theta);
}

/* ------------------------------------------------------------------------ */
/* Binary median-split tree (App. C): a cell holding more than max_leaf      */
/* particles is split across the longest axis of its particles' bounding    */
/* box (the first of x, y, z on ties) into two children with equal numbers  */
/* of particles (the lower floor(n/2) by that coordinate, equal coordinates */
/* ordered by the particles' original index), the lower child first.  The   */
/* paper does not say how ties are split; by original index the split of a  */
/* cell depends only on its set of particles.                               */
/* Cells are shrink-wrapped: the expansion centre is the centre of the       */
/* bounding box of the cell's particles, (lo + hi) / 2 per axis; radii as   */
/* for the octree.  Nodes are numbered level by level (breadth first).       */
/* ------------------------------------------------------------------------ */
static const double* g_sort_coord;   /* coordinate array of the stable sort below */
static void merge_sort_kv(kv_t* v, kv_t* tmp, int64_t n) {
    if (n < 2) return;
    const int64_t h = n / 2;
    merge_sort_kv(v, tmp, h);
    merge_sort_kv(v + h, tmp, n - h);
    int64_t i = 0, j = h, k = 0;
    while (i < h && j < n) {
        /* order by (coordinate, original index): equal coordinates by index */
        const double cj = g_sort_coord[v[j].idx], ci = g_sort_coord[v[i].idx];
        if (cj < ci || (cj == ci && v[j].idx < v[i].idx)) tmp[k++] = v[j++];
        else tmp[k++] = v[i++];
    }
    while (i < h) tmp[k++] = v[i++];
    while (j < n) tmp[k++] = v[j++];
    memcpy(v, tmp, sizeof(kv_t) * n);
}

static void node_bbox(const kv_t* kv, const anode_t* c, const double* x, const double* y, const double* z,
                      double lo[3], double hi[3]) {
    const int64_t i0 = kv[c->b].idx;
    lo[0] = hi[0] = x[i0]; lo[1] = hi[1] = y[i0]; lo[2] = hi[2] = z[i0];
    for (int64_t a = c->b; a < c->e; ++a) {
        const int64_t i = kv[a].idx;
        const double v[3] = {x[i], y[i], z[i]};
        for (int d = 0; d < 3; ++d) { if (v[d] < lo[d]) lo[d] = v[d]; if (v[d] > hi[d]) hi[d] = v[d]; }
    }
}

static void btree_build(atree_t* T, int64_t n, const double* x, const double* y, const double* z, int max_leaf,
                        double theta) {
    memset(T, 0, sizeof(*T));
    T->n = n;
    kv_t* kv = (kv_t*)malloc(sizeof(kv_t) * n);
    kv_t* tmp = (kv_t*)malloc(sizeof(kv_t) * n);
    for (int64_t i = 0; i < n; ++i) { kv[i].key = 0; kv[i].idx = i; }
    int64_t cap = 1024, nn = 1;
    anode_t* nd = (anode_t*)malloc(sizeof(anode_t) * cap);
    memset(&nd[0], 0, sizeof(anode_t));
    nd[0].b = 0; nd[0].e = n; nd[0].child0 = -1; nd[0].parent = -1;
    int64_t lvl_b = 0, lvl_e = 1;
    while (lvl_b < lvl_e) {
        for (int64_t c = lvl_b; c < lvl_e; ++c) {
            double lo[3], hi[3];
            node_bbox(kv, &nd[c], x, y, z, lo, hi);
            nd[c].z[0] = (lo[0] + hi[0]) * 0.5; nd[c].z[1] = (lo[1] + hi[1]) * 0.5; nd[c].z[2] = (lo[2] + hi[2]) * 0.5;
            const int64_t cnt = nd[c].e - nd[c].b;
            if (cnt <= max_leaf) continue;
            int axis = 0;
            for (int d = 1; d < 3; ++d) if (hi[d] - lo[d] > hi[axis] - lo[axis]) axis = d;
            g_sort_coord = axis == 0 ? x : axis == 1 ? y : z;
            merge_sort_kv(kv + nd[c].b, tmp, cnt);
            const int64_t mid = nd[c].b + cnt / 2;
            if (nn + 2 > cap) { cap *= 2; nd = (anode_t*)realloc(nd, sizeof(anode_t) * cap); }
            nd[c].child0 = nn;
            nd[c].nchild = 2;
            for (int k = 0; k < 2; ++k) {
                anode_t* ch = &nd[nn++];
                memset(ch, 0, sizeof(anode_t));
                ch->level = nd[c].level + 1;
                ch->b = k ? mid : nd[c].b;
                ch->e = k ? nd[c].e : mid;
                ch->child0 = -1; ch->nchild = 0; ch->parent = c;
            }
        }
        lvl_b = lvl_e;
        lvl_e = nn;
    }
    free(tmp);
    for (int64_t c = nn - 1; c >= 0; --c) {
        double r = 0.0;
        if (nd[c].nchild == 0) {
            for (int64_t a = nd[c].b; a < nd[c].e; ++a) {
                const int64_t i = kv[a].idx;
                const double v[3] = {x[i], y[i], z[i]};
                const double d = dist3(v, nd[c].z);
                if (d > r) r = d;
            }
        } else {
            for (int k = 0; k < nd[c].nchild; ++k) {
                const anode_t* ch = &nd[nd[c].child0 + k];
                const double d = dist3(ch->z, nd[c].z) + ch->r;
                if (d > r) r = d;
            }
        }
        nd[c].r = r;
    }
    T->nn = nn; T->kv = kv; T->nd = nd;
    atree_lists(T, theta);
}

/* Upward pass: P2M at the leaves (Eq. P2M), M2M to the root (Eq. M2M). */
static void atree_multipoles(const atree_t* T, const double* x, const double* y, const double* z, const double* q,
                             int p, int basis, double* M) {
    const int nc = orc_ncoef(p, basis);
    const anode_t* nd = T->nd;
    const kv_t* kv = T->kv;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t c = 0; c < T->nn; ++c) {
        if (nd[c].nchild) continue;
        const int64_t cnt = nd[c].e - nd[c].b;
        double* buf = (double*)malloc(sizeof(double) * 4 * cnt);
        for (int64_t a = 0; a < cnt; ++a) {
            const int64_t i = kv[nd[c].b + a].idx;
            buf[a] = x[i]; buf[cnt + a] = y[i]; buf[2 * cnt + a] = z[i]; buf[3 * cnt + a] = q[i];
        }
        orc_p2m(p, basis, cnt, buf, buf + cnt, buf + 2 * cnt, buf + 3 * cnt, nd[c].z, M + c * nc);
        free(buf);
    }
    for (int64_t c = T->nn - 1; c >= 0; --c) {   /* children follow parents: reverse order is bottom-up */
        if (!nd[c].nchild) continue;
        for (int k = 0; k < nd[c].nchild; ++k) {
            const int64_t ch = nd[c].child0 + k;
            double d[3] = {nd[ch].z[0] - nd[c].z[0], nd[ch].z[1] - nd[c].z[1], nd[ch].z[2] - nd[c].z[2]};
            orc_m2m(p, basis, M + ch * nc, d, M + c * nc);
        }
    }
}

/* Adaptive FMM.  pair_p (optional, npair_p entries) gives each M2L pair its
 * own truncation order 0 <= p_k <= p, in the order of orc_adaptive_pairs
 * (target, then source): the pair contributes the terms |n| + |m| <= p_k of
 * Eq. M2L (ranks 0..p_k of the stored expansions, which are prefixes of the
 * order-p storage).  Every other operator runs at order p. */
static int fmm_adaptive_impl(int64_t n, const double* x, const double* y, const double* z, const double* q,
                             int max_leaf, double theta, int p, int basis, const signed char* pair_p,
                             int64_t npair_p, int64_t nsample, const int64_t* sample, double* pot, double* ax,
                             double* ay, double* az, int64_t* stats, int ap, int binary) {
    orc_init();
    if (p < 0 || p > ORC_PMAX || max_leaf < 1 || theta < 0.0 || n < 0) return -1;
    int64_t ntarg = nsample >= 0 ? nsample : n;
    if (n == 0) return 0;
    atree_t T;
    if (binary)
        btree_build(&T, n, x, y, z, max_leaf, theta);
    else
        atree_build(&T, n, x, y, z, q, max_leaf, theta, ap != 0);
    const int64_t nn = T.nn;
    const anode_t* nd = T.nd;
    const kv_t* kv = T.kv;
    if (pair_p) {
        if (npair_p != T.m2l.n) { atree_free(&T); return -2; }
        for (int64_t k = 0; k < npair_p; ++k)
            if (pair_p[k] < 0 || pair_p[k] > p) { atree_free(&T); return -1; }
    }
    if (stats) {
        /* stats: nodes, M2L pairs, P2P pairs, leaves, and the number of ordered
           particle pairs the lists cover (n^2 when every pair is covered once) */
        stats[0] = nn; stats[1] = T.m2l.n; stats[2] = T.p2p.n; stats[3] = 0; stats[4] = 0;
        for (int64_t c = 0; c < nn; ++c) stats[3] += nd[c].nchild == 0;
        for (int64_t k = 0; k < T.m2l.n; ++k)
            stats[4] += (nd[T.m2l.v[k].a].e - nd[T.m2l.v[k].a].b) * (nd[T.m2l.v[k].b].e - nd[T.m2l.v[k].b].b);
        for (int64_t k = 0; k < T.p2p.n; ++k)
            stats[4] += (nd[T.p2p.v[k].a].e - nd[T.p2p.v[k].a].b) * (nd[T.p2p.v[k].b].e - nd[T.p2p.v[k].b].b);
    }
    /* which nodes feed sampled targets */
    int64_t* pos_of = (int64_t*)malloc(sizeof(int64_t) * n);   /* sorted position of particle */
    for (int64_t a = 0; a < n; ++a) pos_of[kv[a].idx] = a;
    int64_t* leaf_of = (int64_t*)malloc(sizeof(int64_t) * n);   /* leaf of sorted position */
    for (int64_t c = 0; c < nn; ++c)
        if (nd[c].nchild == 0)
            for (int64_t a = nd[c].b; a < nd[c].e; ++a) leaf_of[a] = c;
    char* need = (char*)calloc(nn, 1);
    for (int64_t t = 0; t < ntarg; ++t) {
        int64_t c = leaf_of[pos_of[nsample >= 0 ? sample[t] : t]];
        while (c >= 0 && !need[c]) { need[c] = 1; c = nd[c].parent; }
    }
    /* upward pass */
    const int nc = orc_ncoef(p, basis);
    double* M = (double*)calloc((size_t)nn * nc, sizeof(double));
    double* L = (double*)calloc((size_t)nn * nc, sizeof(double));
    atree_multipoles(&T, x, y, z, q, p, basis, M);
    if (ap == 1 && p >= 1)   /* AP: about the centre of mass the dipole vanishes; it is set to exactly 0 */
        for (int64_t c = 0; c < nn; ++c)
            for (int t = 1; t <= 3; ++t) M[c * nc + t] = 0.0;
    /* interaction phase: the sorted M2L list is already grouped by target */
    int64_t* cnt = (int64_t*)calloc(nn + 1, sizeof(int64_t));
    for (int64_t k = 0; k < T.m2l.n; ++k) cnt[T.m2l.v[k].a + 1]++;
    for (int64_t c = 0; c < nn; ++c) cnt[c + 1] += cnt[c];
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t c = 0; c < nn; ++c) {
        if (!need[c]) continue;
        double* Lk = (double*)malloc(sizeof(double) * nc);
        for (int64_t k = cnt[c]; k < cnt[c + 1]; ++k) {
            const int64_t s = T.m2l.v[k].b;
            double r[3] = {nd[c].z[0] - nd[s].z[0], nd[c].z[1] - nd[s].z[1], nd[c].z[2] - nd[s].z[2]};
            if (!pair_p) {
                orc_m2l(p, basis, M + s * nc, r, L + c * nc);
            } else {
                /* order p_k on the rank prefix, added into the order-p L */
                const int pk = pair_p[k];
                const int nck = orc_ncoef(pk, basis);
                memset(Lk, 0, sizeof(double) * nc);
                orc_m2l(pk, basis, M + s * nc, r, Lk);
                for (int t = 0; t < nck; ++t) L[c * nc + t] += Lk[t];
            }
        }
        free(Lk);
    }
    for (int64_t c = 0; c < nn; ++c) {   /* parents precede children: forward order is top-down */
        if (!nd[c].nchild || !need[c]) continue;
        for (int k = 0; k < nd[c].nchild; ++k) {
            const int64_t ch = nd[c].child0 + k;
            if (!need[ch]) continue;
            double d[3] = {nd[ch].z[0] - nd[c].z[0], nd[ch].z[1] - nd[c].z[1], nd[ch].z[2] - nd[c].z[2]};
            orc_l2l(p, basis, L + c * nc, d, L + ch * nc);
        }
    }
    /* near-field lists by target leaf */
    int64_t* pc = (int64_t*)calloc(nn + 1, sizeof(int64_t));
    for (int64_t k = 0; k < T.p2p.n; ++k) pc[T.p2p.v[k].a + 1]++;
    for (int64_t c = 0; c < nn; ++c) pc[c + 1] += pc[c];
    int64_t* psrc = (int64_t*)malloc(sizeof(int64_t) * (T.p2p.n > 0 ? T.p2p.n : 1));
    {
        int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (nn + 1));
        memcpy(fill, pc, sizeof(int64_t) * (nn + 1));
        for (int64_t k = 0; k < T.p2p.n; ++k) psrc[fill[T.p2p.v[k].a]++] = T.p2p.v[k].b;
        free(fill);
    }
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t t = 0; t < ntarg; ++t) {
        const int64_t i = nsample >= 0 ? sample[t] : t;
        const int64_t c = leaf_of[pos_of[i]];
        double rb[3] = {x[i] - nd[c].z[0], y[i] - nd[c].z[1], z[i] - nd[c].z[2]}, o[4];
        orc_l2p(p, basis, L + c * nc, rb, o);
        double ph = o[0], gx = o[1], gy = o[2], gz = o[3];
        for (int64_t k = pc[c]; k < pc[c + 1]; ++k) {
            const int64_t s = psrc[k];
            for (int64_t a = nd[s].b; a < nd[s].e; ++a) {
                const int64_t j = kv[a].idx;
                if (j == i) continue;
                double dx = x[j] - x[i], dy = y[j] - y[i], dz = z[j] - z[i];
                double r2 = dx * dx + dy * dy + dz * dz;
                if (r2 == 0.0) continue;
                double ir = 1.0 / sqrt(r2), ir3 = ir * ir * ir;
                ph += q[j] * ir;
                gx += q[j] * dx * ir3; gy += q[j] * dy * ir3; gz += q[j] * dz * ir3;
            }
        }
        /* AP: only the gradient is evaluated (Sec. 3); the potential is not */
        pot[t] = ap == 1 ? 0.0 : -ph; ax[t] = gx; ay[t] = gy; az[t] = gz;
    }
    atree_free(&T);
    free(pos_of); free(leaf_of); free(need); free(M); free(L); free(cnt); free(pc); free(psrc);
    return 0;
}

int orc_fmm_adaptive_orders(int64_t n, const double* x, const double* y, const double* z, const double* q,
                            int max_leaf, double theta, int p, int basis, const signed char* pair_p,
                            int64_t npair_p, int64_t nsample, const int64_t* sample, double* pot, double* ax,
                            double* ay, double* az, int64_t* stats /* [5] or NULL */) {
    return fmm_adaptive_impl(n, x, y, z, q, max_leaf, theta, p, basis, pair_p, npair_p, nsample, sample, pot, ax, ay,
                             az, stats, 0, 0);
}

int orc_fmm_adaptive(int64_t n, const double* x, const double* y, const double* z, const double* q,
                     int max_leaf, double theta, int p, int basis, int64_t nsample, const int64_t* sample,
                     double* pot, double* ax, double* ay, double* az, int64_t* stats /* [5] or NULL */) {
    return orc_fmm_adaptive_orders(n, x, y, z, q, max_leaf, theta, p, basis, NULL, 0, nsample, sample, pot, ax,
                                   ay, az, stats);
}

/* The AP variant (Sec. 3, astrophysics): the adaptive FMM in the fully
 * traceless form with centre-of-mass expansion centres, the dipole of every
 * multipole set to 0 (it vanishes about the centre of mass), and only the
 * gradient evaluated (pot is written as 0).  basis must be traceless. */
int orc_fmm_adaptive_ap(int64_t n, const double* x, const double* y, const double* z, const double* q, int max_leaf,
                        double theta, int p, int64_t nsample, const int64_t* sample, double* pot, double* ax,
                        double* ay, double* az, int64_t* stats) {
    return fmm_adaptive_impl(n, x, y, z, q, max_leaf, theta, p, 1, NULL, 0, nsample, sample, pot, ax, ay, az, stats,
                             1, 0);
}

/* The FMM on the binary median-split tree (App. C): the operators, the
 * traversal and the lists as for the octree; expansion centres at the
 * centres of the cells' shrink-wrapped bounding boxes. */
int orc_fmm_btree(int64_t n, const double* x, const double* y, const double* z, const double* q, int max_leaf,
                  double theta, int p, int basis, int64_t nsample, const int64_t* sample, double* pot, double* ax,
                  double* ay, double* az, int64_t* stats) {
    return fmm_adaptive_impl(n, x, y, z, q, max_leaf, theta, p, basis, NULL, 0, nsample, sample, pot, ax, ay, az,
                             stats, 0, 1);
}

/* The FT variant on the AP tree (centre-of-mass centres, dipole kept and the
 * potential evaluated), for comparison with the AP variant. */
int orc_fmm_adaptive_com(int64_t n, const double* x, const double* y, const double* z, const double* q, int max_leaf,
                         double theta, int p, int64_t nsample, const int64_t* sample, double* pot, double* ax,
                         double* ay, double* az, int64_t* stats) {
    return fmm_adaptive_impl(n, x, y, z, q, max_leaf, theta, p, 1, NULL, 0, nsample, sample, pot, ax, ay, az, stats,
                             2, 0);
}

/* ------------------------------------------------------------------------ */
/* Per-pair data for choosing the M2L order of each pair (learned order;      */
/* the paper fixes one p per run, so everything below is an addition on top  */
/* of its operators, each quantity written out from its definition).         */
/*                                                                            */
/* Pairs come in the order (target, then source).  For a pair with source A,  */
/* target B, offset d = z_B - z_A, radii r_A, r_B, particle counts n_A, n_B   */
/* and full symmetric multipoles (Eq. P2M/M2M, any order >= 4):               */
/*   a = max(r_A/|d|, 1e-6),  b = max(r_B/|d|, 1e-6)                          */
/*   f0 = ln(a + b)   (the MAC ratio of App. C)                               */
/*   f1 = ln a,  f2 = ln b                                                    */
/*   f3..f6 = ln max(|M_A^(j)| / (|M_A,0| r_A^j), 1e-6),  j = 1..4            */
/*   f7..f8 = the same for the target's own multipole M_B, j = 1..2           */
/*   f9 = ln min(n_A, 1024),  f10 = ln min(n_B, 1024) (counts saturate, so a */
/*         model trained on small sets sees no unseen values on large ones)  */
/*   f11 = ln max(g_AB / T_B, 1e-12): the pair's share of a far-field          */
/*         magnitude estimate, g_AB = |M_A,0| / |d|^2 and T_B the sum of g     */
/*         over the M2L lists of B and of all its ancestors                   */
/* where |M^(j)|^2 = sum_{|m|=j} j!/m! M_m^2 is the Frobenius norm of the     */
/* rank-j symmetric tensor (a ratio with a zero denominator counts as 0).     */
/*                                                                            */
/* Label of the pair at order p (p = 2..10): the error of the force the       */
/* pair's order-p M2L (followed by L2P at order p) produces at target         */
/* particles y_j of B, against the direct sum g over A's particles, relative  */
/* to the total force a at those particles (direct sum over all particles,    */
/* the particle itself excluded):                                             */
/*   e_p = sqrt(sum_j |g_p(y_j) - g(y_j)|^2 / sum_j |a(y_j)|^2),              */
/*   label_p = log10(max(e_p, 1e-12)).                                        */
/* The y_j are all of B's particles when n_B <= 64, else the 64 at sorted     */
/* positions b_B + floor(j n_B / 64), j = 0..63.                              */
/* The source multipole is the order-10 one, so every p <= 10 reads its rank  */
/* prefix.                                                                    */
/* ------------------------------------------------------------------------ */
#define ORC_NF 12
#define ORC_NLAB 9

static double rank_norm(const double* M, int j) {
    /* Frobenius norm of the rank-j block of a full symmetric polytensor */
    const int off = orc_ncoef_sym(j - 1);
    double s = 0.0;
    for (int t = 0; t < (j + 1) * (j + 2) / 2; ++t) {
        const int* n = g_sym[off + t];
        const double mult = g_fact[j] / mfact(n[0], n[1], n[2]);
        s += mult * M[off + t] * M[off + t];
    }
    return sqrt(s);
}

static double shape_feature(const double* M, int j, double r) {
    const double m0 = fabs(M[0]);
    double g = 0.0;
    if (m0 > 0.0 && r > 0.0) g = rank_norm(M, j) / (m0 * ipow(r, j));
    return log(g > 1e-6 ? g : 1e-6);
}

/* Relative force error at the points (xt, yt, zt) of the order-p M2L of a
 * source multipole M (full symmetric, order >= p, about zA) towards zB,
 * followed by L2P at order p, against the exact field g of the given source
 * particles (the definition of the label above, for one p). */
static double pair_error(int p, const double* M, const double zA[3], const double zB[3], int nt,
                         const double (*yv)[3], const double (*g)[3], double* Lp /* ncoef_sym(p) */) {
    const double d[3] = {zB[0] - zA[0], zB[1] - zA[1], zB[2] - zA[2]};
    memset(Lp, 0, sizeof(double) * orc_ncoef_sym(p));
    orc_m2l(p, 0, M, d, Lp);
    double num = 0.0, den = 0.0;
    for (int j = 0; j < nt; ++j) {
        const double rb[3] = {yv[j][0] - zB[0], yv[j][1] - zB[1], yv[j][2] - zB[2]};
        double o[4];
        orc_l2p(p, 0, Lp, rb, o);
        for (int c = 0; c < 3; ++c) {
            num += (o[1 + c] - g[j][c]) * (o[1 + c] - g[j][c]);
            den += g[j][c] * g[j][c];
        }
    }
    return den > 0.0 ? sqrt(num / den) : 0.0;
}

/* The same from source particles (P2M about zA at order p) and up to 64
 * target points; used to check the per-pair labels. */
double orc_pair_error(int p, int64_t na, const double* xa, const double* ya, const double* za, const double* qa,
                      const double zA[3], const double zB[3], int nt, const double* xt, const double* yt,
                      const double* zt) {
    orc_init();
    if (p < 0 || p > ORC_PMAX || nt < 1 || nt > 64) return -1.0;
    const int nc = orc_ncoef_sym(p);
    double* M = (double*)calloc(nc, sizeof(double));
    double* Lp = (double*)malloc(sizeof(double) * nc);
    double yv[64][3], g[64][3];
    orc_p2m(p, 0, na, xa, ya, za, qa, zA, M);
    for (int j = 0; j < nt; ++j) {
        yv[j][0] = xt[j]; yv[j][1] = yt[j]; yv[j][2] = zt[j];
        g[j][0] = g[j][1] = g[j][2] = 0.0;
        for (int64_t i = 0; i < na; ++i) {
            const double dx = xa[i] - yv[j][0], dy = ya[i] - yv[j][1], dz = za[i] - yv[j][2];
            const double r2 = dx * dx + dy * dy + dz * dz;
            const double ir = 1.0 / sqrt(r2), ir3 = ir * ir * ir;
            g[j][0] += qa[i] * dx * ir3; g[j][1] += qa[i] * dy * ir3; g[j][2] += qa[i] * dz * ir3;
        }
    }
    const double e = pair_error(p, M, zA, zB, nt, (const double (*)[3])yv, (const double (*)[3])g, Lp);
    free(M); free(Lp);
    return e;
}

/* The adaptive tree itself: per node (centre x, y, z, radius), the range
 * [b, e) of sorted positions it holds and its parent (-1 for the root);
 * order[a] = the particle at sorted position a.  Returns the node count
 * (arrays written when cap allows). */
static int64_t adaptive_tree_impl(int64_t n, const double* x, const double* y, const double* z, const double* q,
                                  int com, int max_leaf, int64_t cap, double* zr, int64_t* range, int64_t* order,
                                  int64_t* parent) {
    orc_init();
    if (max_leaf < 1 || n < 1) return -1;
    atree_t T;
    if (com == 2)
        btree_build(&T, n, x, y, z, max_leaf, 0.0);
    else
        atree_build(&T, n, x, y, z, q, max_leaf, 0.0, com);
    const int64_t nn = T.nn;
    if (cap >= nn) {
        for (int64_t c = 0; c < nn; ++c) {
            if (zr) { zr[4 * c] = T.nd[c].z[0]; zr[4 * c + 1] = T.nd[c].z[1]; zr[4 * c + 2] = T.nd[c].z[2];
                      zr[4 * c + 3] = T.nd[c].r; }
            if (range) { range[2 * c] = T.nd[c].b; range[2 * c + 1] = T.nd[c].e; }
            if (parent) parent[c] = T.nd[c].parent;
        }
        if (order) for (int64_t a = 0; a < n; ++a) order[a] = T.kv[a].idx;
    }
    atree_free(&T);
    return nn;
}

int64_t orc_adaptive_tree(int64_t n, const double* x, const double* y, const double* z, int max_leaf, int64_t cap,
                          double* zr, int64_t* range, int64_t* order, int64_t* parent) {
    return adaptive_tree_impl(n, x, y, z, NULL, 0, max_leaf, cap, zr, range, order, parent);
}

/* The binary median-split tree (App. C). */
int64_t orc_btree(int64_t n, const double* x, const double* y, const double* z, int max_leaf, int64_t cap, double* zr,
                  int64_t* range, int64_t* order, int64_t* parent) {
    return adaptive_tree_impl(n, x, y, z, NULL, 2, max_leaf, cap, zr, range, order, parent);
}

/* The tree with centre-of-mass centres (the AP variant's geometry). */
int64_t orc_adaptive_tree_com(int64_t n, const double* x, const double* y, const double* z, const double* q,
                              int max_leaf, int64_t cap, double* zr, int64_t* range, int64_t* order, int64_t* parent) {
    return adaptive_tree_impl(n, x, y, z, q, 1, max_leaf, cap, zr, range, order, parent);
}

int orc_ncols_features(void) { return ORC_NF; }
int orc_ncols_labels(void) { return ORC_NLAB; }

int64_t orc_adaptive_pairs(int64_t n, const double* x, const double* y, const double* z, const double* q,
                           int max_leaf, double theta, int64_t cap, int64_t* tgt, int64_t* src, double* feat,
                           double* lab) {
    orc_init();
    if (max_leaf < 1 || theta < 0.0 || n < 0) return -1;
    if (n == 0) return 0;
    atree_t T;
    atree_build(&T, n, x, y, z, q, max_leaf, theta, 0);
    const int64_t np = T.m2l.n;
    if (cap < np || (!tgt && !src && !feat && !lab)) { atree_free(&T); return np; }
    const anode_t* nd = T.nd;
    const kv_t* kv = T.kv;
    const int P = 10, nc = orc_ncoef_sym(P);
    double* M = NULL;
    if (feat || lab) {
        M = (double*)calloc((size_t)T.nn * nc, sizeof(double));
        atree_multipoles(&T, x, y, z, q, P, 0, M);
    }
    /* far-field magnitude estimate T_B (feature f11) */
    double* Tf = NULL;
    if (feat) {
        double* S = (double*)calloc((size_t)T.nn, sizeof(double));
        Tf = (double*)calloc((size_t)T.nn, sizeof(double));
        for (int64_t k = 0; k < np; ++k) {
            const int64_t B = T.m2l.v[k].a, A = T.m2l.v[k].b;
            const double dd = dist3(nd[A].z, nd[B].z);
            S[B] += fabs(M[A * nc]) / (dd * dd);
        }
        for (int64_t c = 0; c < T.nn; ++c) Tf[c] = S[c] + (nd[c].parent >= 0 ? Tf[nd[c].parent] : 0.0);
        free(S);
    }
    /* total force at every particle (label denominators), caller order */
    double* at[4] = {NULL, NULL, NULL, NULL};
    if (lab) {
        for (int c = 0; c < 4; ++c) at[c] = (double*)malloc(sizeof(double) * n);
        orc_direct(n, x, y, z, q, -1, NULL, at[0], at[1], at[2], at[3]);
    }
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t k = 0; k < np; ++k) {
        const int64_t B = T.m2l.v[k].a, A = T.m2l.v[k].b;
        if (tgt) tgt[k] = B;
        if (src) src[k] = A;
        const double d[3] = {nd[B].z[0] - nd[A].z[0], nd[B].z[1] - nd[A].z[1], nd[B].z[2] - nd[A].z[2]};
        const double dn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        if (feat) {
            double* f = feat + k * ORC_NF;
            double a = nd[A].r / dn, b = nd[B].r / dn;
            if (a < 1e-6) a = 1e-6;
            if (b < 1e-6) b = 1e-6;
            f[0] = log(a + b);
            f[1] = log(a);
            f[2] = log(b);
            for (int j = 1; j <= 4; ++j) f[2 + j] = shape_feature(M + A * nc, j, nd[A].r);
            for (int j = 1; j <= 2; ++j) f[6 + j] = shape_feature(M + B * nc, j, nd[B].r);
            f[9] = log((double)(nd[A].e - nd[A].b < 1024 ? nd[A].e - nd[A].b : 1024));
            f[10] = log((double)(nd[B].e - nd[B].b < 1024 ? nd[B].e - nd[B].b : 1024));
            {
                const double share = Tf[B] > 0.0 ? fabs(M[A * nc]) / (dn * dn) / Tf[B] : 0.0;
                f[11] = log(share > 1e-12 ? share : 1e-12);
            }
        }
        if (lab) {
            const int64_t nB = nd[B].e - nd[B].b;
            const int ny = nB <= 64 ? (int)nB : 64;
            double yv[64][3], g[64][3];
            for (int j = 0; j < ny; ++j) {
                const int64_t sp = nd[B].b + (nB <= 64 ? j : (int64_t)j * nB / 64);
                const int64_t t = kv[sp].idx;
                yv[j][0] = x[t]; yv[j][1] = y[t]; yv[j][2] = z[t];
                g[j][0] = g[j][1] = g[j][2] = 0.0;
                for (int64_t s = nd[A].b; s < nd[A].e; ++s) {
                    const int64_t i = kv[s].idx;
                    const double dx = x[i] - yv[j][0], dy = y[i] - yv[j][1], dz = z[i] - yv[j][2];
                    const double r2 = dx * dx + dy * dy + dz * dz;
                    const double ir = 1.0 / sqrt(r2), ir3 = ir * ir * ir;
                    g[j][0] += q[i] * dx * ir3; g[j][1] += q[i] * dy * ir3; g[j][2] += q[i] * dz * ir3;
                }
            }
            /* relative to the pair's own force -> relative to the total force */
            double own = 0.0, tot = 0.0;
            for (int j = 0; j < ny; ++j) {
                const int64_t sp = nd[B].b + (nB <= 64 ? j : (int64_t)j * nB / 64);
                const int64_t t = kv[sp].idx;
                own += g[j][0] * g[j][0] + g[j][1] * g[j][1] + g[j][2] * g[j][2];
                tot += at[1][t] * at[1][t] + at[2][t] * at[2][t] + at[3][t] * at[3][t];
            }
            const double scale = tot > 0.0 ? sqrt(own / tot) : 0.0;
            double* Lp = (double*)malloc(sizeof(double) * nc);
            for (int p = 2; p <= P; ++p) {
                const double e = scale * pair_error(p, M + A * nc, nd[A].z, nd[B].z, ny, (const double (*)[3])yv,
                                                    (const double (*)[3])g, Lp);
                lab[k * ORC_NLAB + (p - 2)] = log10(e > 1e-12 ? e : 1e-12);
            }
            free(Lp);
        }
    }
    free(M);
    free(Tf);
    for (int c = 0; c < 4; ++c) free(at[c]);
    atree_free(&T);
    return np;
}
