/*
 * hdd_oracle.c — plain CPU reference of the method, complex128 throughout.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by tests/, __graft_entry__.smoke() and bench.py's
 * CPU-baseline leg, never by the product path.  It shares no code with the CUDA library.
 *
 * Each routine follows the paper's definitions literally (element-by-element assembly of the
 * weak form, explicit sparse Z_j = Z_j^y (x) Z_j^x, E_j = Z_j^T A_j Z_j formed by sparse
 * products, textbook banded LU with partial pivoting, restarted GMRES/FGMRES with classical
 * Gram-Schmidt applied twice and complex Givens rotations).  Threads (OpenMP) share only
 * independent work: whole subdomain solves, and the independent dot products / vector elements
 * of the outer orthogonalisation; every value is computed by one thread in a fixed order, so
 * results do not depend on the thread count.
 */
#include "hdd_oracle.h"

#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex zc;

/* ------------------------------------------------------------------------------------------ */
/* real CSR                                                                                    */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
    int nr, nc, nnz;
    int *rp, *ci;
    double *v;
    double *vi;      /* imaginary parts (same pattern), NULL for a real matrix */
} csr;

static void csr_free(csr *a) {
    free(a->rp); free(a->ci); free(a->v); free(a->vi);
    memset(a, 0, sizeof(*a));
}

/* y = A x for complex x (real or complex matrix). */
static void csr_mv(const csr *a, const zc *x, zc *y) {
    for (int r = 0; r < a->nr; r++) {
        zc s = 0;
        if (a->vi)
            for (int t = a->rp[r]; t < a->rp[r + 1]; t++) s += CMPLX(a->v[t], a->vi[t]) * x[a->ci[t]];
        else
            for (int t = a->rp[r]; t < a->rp[r + 1]; t++) s += a->v[t] * x[a->ci[t]];
        y[r] = s;
    }
}

static csr csr_transpose(const csr *a) {
    csr t;
    t.nr = a->nc; t.nc = a->nr; t.nnz = a->nnz;
    t.rp = (int *)calloc((size_t)t.nr + 1, sizeof(int));
    t.ci = (int *)malloc(sizeof(int) * (size_t)(a->nnz > 0 ? a->nnz : 1));
    t.v = (double *)malloc(sizeof(double) * (size_t)(a->nnz > 0 ? a->nnz : 1));
    t.vi = a->vi ? (double *)malloc(sizeof(double) * (size_t)(a->nnz > 0 ? a->nnz : 1)) : NULL;
    for (int k = 0; k < a->nnz; k++) t.rp[a->ci[k] + 1]++;
    for (int r = 0; r < t.nr; r++) t.rp[r + 1] += t.rp[r];
    int *pos = (int *)malloc(sizeof(int) * (size_t)(t.nr + 1));
    memcpy(pos, t.rp, sizeof(int) * (size_t)(t.nr + 1));
    for (int r = 0; r < a->nr; r++)
        for (int k = a->rp[r]; k < a->rp[r + 1]; k++) {
            int d = pos[a->ci[k]]++;
            t.ci[d] = r;
            t.v[d] = a->v[k];
            if (a->vi) t.vi[d] = a->vi[k];
        }
    free(pos);
    return t;
}

/* C = A B (Gustavson row-by-row product with a dense accumulator; columns sorted).  Complex
 * if either factor is: (a + i a')(b + i b') = (ab - a'b') + i (ab' + a'b). */
static csr csr_matmul(const csr *a, const csr *b) {
    csr c;
    const int cplx = a->vi != NULL || b->vi != NULL;
    c.nr = a->nr; c.nc = b->nc;
    c.rp = (int *)calloc((size_t)c.nr + 1, sizeof(int));
    double *acc = (double *)calloc((size_t)b->nc, sizeof(double));
    double *acci = cplx ? (double *)calloc((size_t)b->nc, sizeof(double)) : NULL;
    int *mark = (int *)malloc(sizeof(int) * (size_t)b->nc);
    for (int j = 0; j < b->nc; j++) mark[j] = -1;
    int cap = 16 * (a->nr + 1), nnz = 0;
    c.ci = (int *)malloc(sizeof(int) * (size_t)cap);
    c.v = (double *)malloc(sizeof(double) * (size_t)cap);
    c.vi = cplx ? (double *)malloc(sizeof(double) * (size_t)cap) : NULL;
    int *cols = (int *)malloc(sizeof(int) * (size_t)b->nc);
    for (int r = 0; r < a->nr; r++) {
        int nc = 0;
        for (int t = a->rp[r]; t < a->rp[r + 1]; t++) {
            int k = a->ci[t];
            double av = a->v[t], ai = a->vi ? a->vi[t] : 0.0;
            for (int u = b->rp[k]; u < b->rp[k + 1]; u++) {
                int j = b->ci[u];
                if (mark[j] != r) {
                    mark[j] = r; acc[j] = 0.0; cols[nc++] = j;
                    if (cplx) acci[j] = 0.0;
                }
                if (cplx) {
                    double bv = b->v[u], bi = b->vi ? b->vi[u] : 0.0;
                    acc[j] += av * bv - ai * bi;
                    acci[j] += av * bi + ai * bv;
                } else {
                    acc[j] += av * b->v[u];
                }
            }
        }
        /* insertion sort of the row's column list */
        for (int i = 1; i < nc; i++) {
            int key = cols[i], q = i - 1;
            while (q >= 0 && cols[q] > key) { cols[q + 1] = cols[q]; q--; }
            cols[q + 1] = key;
        }
        if (nnz + nc > cap) {
            while (nnz + nc > cap) cap *= 2;
            c.ci = (int *)realloc(c.ci, sizeof(int) * (size_t)cap);
            c.v = (double *)realloc(c.v, sizeof(double) * (size_t)cap);
            if (cplx) c.vi = (double *)realloc(c.vi, sizeof(double) * (size_t)cap);
        }
        for (int i = 0; i < nc; i++) {
            c.ci[nnz] = cols[i]; c.v[nnz] = acc[cols[i]];
            if (cplx) c.vi[nnz] = acci[cols[i]];
            nnz++;
        }
        c.rp[r + 1] = nnz;
    }
    c.nnz = nnz;
    free(acc); free(acci); free(mark); free(cols);
    return c;
}

/* ------------------------------------------------------------------------------------------ */
/* banded LU with partial pivoting (Gaussian elimination restricted to the band; the row     */
/* interchanges widen the upper band to kl+ku).  Row-band storage: element (r,c) with         */
/* -kl <= c-r <= kl+ku sits at ab[r*W + (c - r + kl)], W = 2kl+ku+1.                          */
/* ------------------------------------------------------------------------------------------ */
#define AB(r, c) ab[(size_t)(r) * W + (size_t)((c) - (r) + kl)]

int or_band_lu(int m, int kl, int ku, double *ab, int *piv) {
    const int W = 2 * kl + ku + 1;
    for (int j = 0; j < m; j++) {
        int rlast = j + kl < m - 1 ? j + kl : m - 1;
        int clast = j + kl + ku < m - 1 ? j + kl + ku : m - 1;
        int p = j;
        double amax = fabs(AB(j, j));
        for (int r = j + 1; r <= rlast; r++)
            if (fabs(AB(r, j)) > amax) { amax = fabs(AB(r, j)); p = r; }
        piv[j] = p;
        if (!(amax > 0.0) || !isfinite(amax)) return OR_ERR_SINGULAR;
        if (p != j)
            for (int c = j; c <= clast; c++) {
                double t = AB(j, c); AB(j, c) = AB(p, c); AB(p, c) = t;
            }
        for (int r = j + 1; r <= rlast; r++) {
            double l = AB(r, j) / AB(j, j);
            AB(r, j) = l;
            for (int c = j + 1; c <= clast; c++) AB(r, c) -= l * AB(j, c);
        }
    }
    return OR_OK;
}

static void band_solve_z(int m, int kl, int ku, const double *ab, const int *piv, zc *b) {
    const int W = 2 * kl + ku + 1;
    for (int j = 0; j < m; j++) {
        int p = piv[j];
        if (p != j) { zc t = b[j]; b[j] = b[p]; b[p] = t; }
        int rlast = j + kl < m - 1 ? j + kl : m - 1;
        for (int r = j + 1; r <= rlast; r++) b[r] -= AB(r, j) * b[j];
    }
    for (int r = m - 1; r >= 0; r--) {
        int clast = r + kl + ku < m - 1 ? r + kl + ku : m - 1;
        zc s = b[r];
        for (int c = r + 1; c <= clast; c++) s -= AB(r, c) * b[c];
        b[r] = s / AB(r, r);
    }
}

void or_band_solve(int m, int kl, int ku, const double *ab, const int *piv, double *b_c128) {
    band_solve_z(m, kl, ku, ab, piv, (zc *)b_c128);
}

/* The same elimination for a complex band (the impedance boundary makes A_j and E_j complex
 * symmetric): the pivot is the entry of largest modulus in the column. */
static int band_lu_c(int m, int kl, int ku, zc *ab, int *piv) {
    const int W = 2 * kl + ku + 1;
    for (int j = 0; j < m; j++) {
        int rlast = j + kl < m - 1 ? j + kl : m - 1;
        int clast = j + kl + ku < m - 1 ? j + kl + ku : m - 1;
        int p = j;
        double amax = cabs(AB(j, j));
        for (int r = j + 1; r <= rlast; r++)
            if (cabs(AB(r, j)) > amax) { amax = cabs(AB(r, j)); p = r; }
        piv[j] = p;
        if (!(amax > 0.0) || !isfinite(amax)) return OR_ERR_SINGULAR;
        if (p != j)
            for (int c = j; c <= clast; c++) {
                zc t = AB(j, c); AB(j, c) = AB(p, c); AB(p, c) = t;
            }
        for (int r = j + 1; r <= rlast; r++) {
            zc l = AB(r, j) / AB(j, j);
            AB(r, j) = l;
            for (int c = j + 1; c <= clast; c++) AB(r, c) -= l * AB(j, c);
        }
    }
    return OR_OK;
}

static void band_solve_c(int m, int kl, int ku, const zc *ab, const int *piv, zc *b) {
    const int W = 2 * kl + ku + 1;
    for (int j = 0; j < m; j++) {
        int p = piv[j];
        if (p != j) { zc t = b[j]; b[j] = b[p]; b[p] = t; }
        int rlast = j + kl < m - 1 ? j + kl : m - 1;
        for (int r = j + 1; r <= rlast; r++) b[r] -= AB(r, j) * b[j];
    }
    for (int r = m - 1; r >= 0; r--) {
        int clast = r + kl + ku < m - 1 ? r + kl + ku : m - 1;
        zc s = b[r];
        for (int c = r + 1; c <= clast; c++) s -= AB(r, c) * b[c];
        b[r] = s / AB(r, r);
    }
}

#undef AB

int or_band_lu_z(int m, int kl, int ku, double *ab_c128, int *piv) {
    return band_lu_c(m, kl, ku, (zc *)ab_c128, piv);
}
void or_band_solve_z(int m, int kl, int ku, const double *ab_c128, const int *piv, double *b_c128) {
    band_solve_c(m, kl, ku, (const zc *)ab_c128, piv, (zc *)b_c128);
}

/* ------------------------------------------------------------------------------------------ */
/* problem                                                                                     */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
    int m, kl, ku;
    double *ab;              /* real band, or NULL when the matrix is complex */
    zc *abz;                 /* complex band, or NULL when the matrix is real */
    int *piv;
} bandlu;

static int bandlu_factor(bandlu *f) {
    return f->abz ? band_lu_c(f->m, f->kl, f->ku, f->abz, f->piv)
                  : or_band_lu(f->m, f->kl, f->ku, f->ab, f->piv);
}
static void bandlu_solve(const bandlu *f, zc *b) {
    if (f->abz) band_solve_c(f->m, f->kl, f->ku, f->abz, f->piv, b);
    else band_solve_z(f->m, f->kl, f->ku, f->ab, f->piv, b);
}
static void bandlu_free(bandlu *f) {
    free(f->ab); free(f->abz); free(f->piv);
    f->ab = NULL; f->abz = NULL; f->piv = NULL;
}

typedef struct {
    int ix0, ix1, iy0, iy1;  /* local interior node box (inclusive, global node indices) */
    int ox0, ox1, oy0, oy1;  /* owned nodes (partition of unity D_j = ownership indicator) */
    int nx, ny, n;
    int mx, my, m;
    int *gidx;               /* local -> global unknown index (R_j) */
    csr A;                   /* A_j = R_j A R_j^T */
    csr Z, Zt;               /* deflation matrix Z_j (n x m) and its transpose */
    bandlu E;                /* factored E_j = Z_j^T A_j Z_j */
    double *Edense;          /* E_j before factoring, kept only for small m (tests) */
    double *Edense_i;        /* its imaginary part (complex E_j only) */
    bandlu Aex;              /* factored A_j for the direct local solve */
} subdomain;

/* Grid coarse space of the two-level variant: P1 on the mesh of N/c intervals, interpolation P
 * (fine interior nodes x coarse interior nodes), and the coarse operator A_H = K_H - k² M_H^lumped
 * in band form, factored. */
typedef struct {
    int have, c, Nc, mc, nH, kl;
    csr P, Pt;
    double *ab;
    int *piv;
} cgrid;

struct or_problem {
    cgrid cg;
    int N, n, diag;
    int bc;                  /* 0: Dirichlet (Eq. 1); 1: impedance (Sommerfeld) on all four sides */
    int lo, hi;              /* node indices 0..N that are unknowns: lo..hi in both directions */
    double k, h;
    csr A, K, M, B;          /* B: boundary mass matrix ∫_∂Ω φ_a φ_b ds (empty for bc = 0) */
    int Sx, Sy, nsub, overlap;
    subdomain *sub;
    int have_defl, have_exact;
};

static int nthreads_req = 0;
void or_set_threads(int t) { nthreads_req = t; }
int or_get_threads(void) {
#ifdef _OPENMP
    return nthreads_req > 0 ? nthreads_req : omp_get_max_threads();
#else
    return 1;
#endif
}

/* -- Eq. 2: P1 assembly, element by element ----------------------------------------------- */
typedef struct { int *col; double *val; int *cnt; } rowacc;

static void acc_add(rowacc *a, int row, int col, double v) {
    int base = row * 8;
    for (int t = 0; t < a->cnt[row]; t++)
        if (a->col[base + t] == col) { a->val[base + t] += v; return; }
    a->col[base + a->cnt[row]] = col;
    a->val[base + a->cnt[row]] = v;
    a->cnt[row]++;
}

static csr acc_to_csr(rowacc *a, int n) {
    csr c;
    c.nr = c.nc = n;
    c.rp = (int *)malloc(sizeof(int) * (size_t)(n + 1));
    c.rp[0] = 0;
    for (int r = 0; r < n; r++) c.rp[r + 1] = c.rp[r] + a->cnt[r];
    c.nnz = c.rp[n];
    c.ci = (int *)malloc(sizeof(int) * (size_t)c.nnz);
    c.v = (double *)malloc(sizeof(double) * (size_t)c.nnz);
    c.vi = NULL;
    for (int r = 0; r < n; r++) {
        int base = r * 8, cnt = a->cnt[r];
        int *cc = a->col + base;
        double *vv = a->val + base;
        for (int i = 1; i < cnt; i++) {           /* insertion sort by column */
            int kc = cc[i]; double kv = vv[i]; int q = i - 1;
            while (q >= 0 && cc[q] > kc) { cc[q + 1] = cc[q]; vv[q + 1] = vv[q]; q--; }
            cc[q + 1] = kc; vv[q + 1] = kv;
        }
        memcpy(c.ci + c.rp[r], cc, sizeof(int) * (size_t)cnt);
        memcpy(c.v + c.rp[r], vv, sizeof(double) * (size_t)cnt);
    }
    return c;
}

/* Unknown index of node (i, j), x fastest.  Dirichlet (bc 0): interior nodes 1 <= i, j <= N-1
 * only, -1 on the boundary (eliminated, u = 0 there).  Impedance (bc 1): every node
 * 0 <= i, j <= N is an unknown. */
static int node_index(int N, int bc, int i, int j) {
    if (bc) {
        if (i < 0 || i > N || j < 0 || j > N) return -1;
        return i + j * (N + 1);
    }
    if (i < 1 || i > N - 1 || j < 1 || j > N - 1) return -1;
    return (i - 1) + (j - 1) * (N - 1);
}

/* Element matrices of the bilinear form a(u,v) = ∫ ∇u·∇v - k² u v (Eq. 2) on one triangle:
 * stiffness K_T[a][b] = ∇φ_a·∇φ_b |T| and consistent mass M_T[a][b] = |T|(1+δ_ab)/12. */
static void element_matrices(const double xy[3][2], double Ke[3][3], double Me[3][3]) {
    double x0 = xy[0][0], y0 = xy[0][1], x1 = xy[1][0], y1 = xy[1][1], x2 = xy[2][0], y2 = xy[2][1];
    double det = (x1 - x0) * (y2 - y0) - (x2 - x0) * (y1 - y0);
    double area = 0.5 * fabs(det);
    double g[3][2] = {{(y1 - y2) / det, (x2 - x1) / det},
                      {(y2 - y0) / det, (x0 - x2) / det},
                      {(y0 - y1) / det, (x1 - x0) / det}};
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) {
            Ke[a][b] = (g[a][0] * g[b][0] + g[a][1] * g[b][1]) * area;
            Me[a][b] = area * (a == b ? 2.0 : 1.0) / 12.0;
        }
}

/* Element matrix of the boundary term ∫_e φ_a φ_b ds on one boundary edge e of length |e|
 * (1D P1 mass): |e|(1+δ_ab)/6. */
static void edge_mass(const double xy[2][2], double Be[2][2]) {
    double len = hypot(xy[1][0] - xy[0][0], xy[1][1] - xy[0][1]);
    for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2; b++) Be[a][b] = len * (a == b ? 2.0 : 1.0) / 6.0;
}

or_problem *or_create(int N, double k, int diag) { return or_create_bc(N, k, diag, 0); }

/* bc 1: the first-order absorbing (Sommerfeld) condition ∂u/∂n - i k u = 0 on all of ∂Ω.
 * Integrating -Δu by parts then leaves -i k ∫_∂Ω u v ds in the bilinear form of Eq. 2 (no
 * conjugation, so A = K - k²M - i k B is complex symmetric, not Hermitian), and every node
 * of the mesh, boundary nodes included, is an unknown. */
or_problem *or_create_bc(int N, double k, int diag, int bc) {
    if (N < 2 || bc < 0 || bc > 1) return NULL;
    or_problem *p = (or_problem *)calloc(1, sizeof(or_problem));
    p->N = N; p->k = k; p->diag = diag; p->h = 1.0 / N; p->bc = bc;
    p->lo = bc ? 0 : 1;
    p->hi = bc ? N : N - 1;
    p->n = (p->hi - p->lo + 1) * (p->hi - p->lo + 1);
    int n = p->n;
    rowacc aA, aK, aM, aB;
    rowacc *accs[4] = {&aA, &aK, &aM, &aB};
    for (int q = 0; q < 4; q++) {
        accs[q]->col = (int *)malloc(sizeof(int) * 8 * (size_t)n);
        accs[q]->val = (double *)malloc(sizeof(double) * 8 * (size_t)n);
        accs[q]->cnt = (int *)calloc((size_t)n, sizeof(int));
    }
    const double h = p->h, k2 = k * k;
    for (int cj = 0; cj < N; cj++)
        for (int ci = 0; ci < N; ci++) {
            /* two triangles per cell, split along SW-NE (diag 0) or NW-SE (diag 1) */
            int tri[2][3][2];
            if (diag == 0) {
                int t0[3][2] = {{ci, cj}, {ci + 1, cj}, {ci + 1, cj + 1}};
                int t1[3][2] = {{ci, cj}, {ci + 1, cj + 1}, {ci, cj + 1}};
                memcpy(tri[0], t0, sizeof(t0)); memcpy(tri[1], t1, sizeof(t1));
            } else {
                int t0[3][2] = {{ci, cj}, {ci + 1, cj}, {ci, cj + 1}};
                int t1[3][2] = {{ci + 1, cj}, {ci + 1, cj + 1}, {ci, cj + 1}};
                memcpy(tri[0], t0, sizeof(t0)); memcpy(tri[1], t1, sizeof(t1));
            }
            for (int t = 0; t < 2; t++) {
                double xy[3][2], Ke[3][3], Me[3][3];
                int gi[3];
                for (int a = 0; a < 3; a++) {
                    xy[a][0] = tri[t][a][0] * h;
                    xy[a][1] = tri[t][a][1] * h;
                    gi[a] = node_index(N, bc, tri[t][a][0], tri[t][a][1]);
                }
                element_matrices(xy, Ke, Me);
                for (int a = 0; a < 3; a++) {
                    if (gi[a] < 0) continue;  /* Dirichlet nodes eliminated (u = 0 there) */
                    for (int b = 0; b < 3; b++) {
                        if (gi[b] < 0) continue;
                        acc_add(&aK, gi[a], gi[b], Ke[a][b]);
                        acc_add(&aM, gi[a], gi[b], Me[a][b]);
                        acc_add(&aA, gi[a], gi[b], Ke[a][b] - k2 * Me[a][b]);
                    }
                }
            }
        }
    if (bc) {
        /* the 4N boundary edges: bottom, top (along x), left, right (along y) */
        for (int side = 0; side < 4; side++)
            for (int e = 0; e < N; e++) {
                int nd[2][2];
                if (side < 2) { int j = side == 0 ? 0 : N; nd[0][0] = e; nd[0][1] = j; nd[1][0] = e + 1; nd[1][1] = j; }
                else { int i = side == 2 ? 0 : N; nd[0][0] = i; nd[0][1] = e; nd[1][0] = i; nd[1][1] = e + 1; }
                double xy[2][2], Be[2][2];
                int gi[2];
                for (int a = 0; a < 2; a++) {
                    xy[a][0] = nd[a][0] * h;
                    xy[a][1] = nd[a][1] * h;
                    gi[a] = node_index(N, bc, nd[a][0], nd[a][1]);
                }
                edge_mass(xy, Be);
                for (int a = 0; a < 2; a++)
                    for (int b = 0; b < 2; b++) acc_add(&aB, gi[a], gi[b], Be[a][b]);
            }
    }
    p->A = acc_to_csr(&aA, n);
    p->K = acc_to_csr(&aK, n);
    p->M = acc_to_csr(&aM, n);
    p->B = acc_to_csr(&aB, n);
    if (bc) {
        /* Im A = -k B on A's pattern (every boundary edge is the side of a triangle, so B's
         * pattern lies inside A's) */
        p->A.vi = (double *)calloc((size_t)(p->A.nnz > 0 ? p->A.nnz : 1), sizeof(double));
        for (int r = 0; r < n; r++)
            for (int t = p->B.rp[r]; t < p->B.rp[r + 1]; t++) {
                int q = p->A.rp[r];
                while (q < p->A.rp[r + 1] && p->A.ci[q] != p->B.ci[t]) q++;
                if (q < p->A.rp[r + 1]) p->A.vi[q] = -k * p->B.v[t];
            }
    }
    for (int q = 0; q < 4; q++) { free(accs[q]->col); free(accs[q]->val); free(accs[q]->cnt); }
    return p;
}

static void free_sub(subdomain *s) {
    free(s->gidx);
    csr_free(&s->A); csr_free(&s->Z); csr_free(&s->Zt);
    bandlu_free(&s->E); free(s->Edense); free(s->Edense_i);
    bandlu_free(&s->Aex);
}

void or_destroy(or_problem *p) {
    if (!p) return;
    csr_free(&p->cg.P); csr_free(&p->cg.Pt); free(p->cg.ab); free(p->cg.piv);
    csr_free(&p->A); csr_free(&p->K); csr_free(&p->M); csr_free(&p->B);
    if (p->sub) { for (int s = 0; s < p->nsub; s++) free_sub(&p->sub[s]); free(p->sub); }
    free(p);
}

int or_n(const or_problem *p) { return p->n; }

static const csr *pick(const or_problem *p, int which) {
    return which == 0 ? &p->A : which == 1 ? &p->K : which == 2 ? &p->M : &p->B;
}
int or_nnz(const or_problem *p, int which) { return pick(p, which)->nnz; }
void or_get_csr(const or_problem *p, int which, int *rowptr, int *col, double *val) {
    const csr *a = pick(p, which);
    memcpy(rowptr, a->rp, sizeof(int) * (size_t)(a->nr + 1));
    memcpy(col, a->ci, sizeof(int) * (size_t)a->nnz);
    memcpy(val, a->v, sizeof(double) * (size_t)a->nnz);
}
void or_get_csr_imag(const or_problem *p, int which, double *val) {
    const csr *a = pick(p, which);
    if (a->vi) memcpy(val, a->vi, sizeof(double) * (size_t)a->nnz);
    else memset(val, 0, sizeof(double) * (size_t)a->nnz);
}
void or_apply_global(const or_problem *p, int which, const double *x, double *y) {
    csr_mv(pick(p, which), (const zc *)x, (zc *)y);
}

/* -- right-hand sides (§3) -------------------------------------------------------------------- */
/* Point source: F(v) = amp · v(x_c), with x_c snapped to the nearest node that is an unknown
 * (an interior node for Dirichlet, any node for the impedance condition). */
void or_rhs_point(const or_problem *p, double x, double y, double amp, double *f) {
    int N = p->N;
    int i = (int)floor(x * N + 0.5), j = (int)floor(y * N + 0.5);
    if (i < p->lo) i = p->lo;
    if (i > p->hi) i = p->hi;
    if (j < p->lo) j = p->lo;
    if (j > p->hi) j = p->hi;
    ((zc *)f)[node_index(N, p->bc, i, j)] += amp;
}

/* F += M g_I, g_I the interpolant in V^h of the Gaussian bump (its nodal values at the
 * unknowns; zero on the boundary for Dirichlet). */
void or_rhs_gauss(const or_problem *p, double cx, double cy, double sigma, double amp, double *f) {
    int N = p->N;
    zc *g = (zc *)calloc((size_t)p->n, sizeof(zc));
    zc *mg = (zc *)malloc(sizeof(zc) * (size_t)p->n);
    for (int j = p->lo; j <= p->hi; j++)
        for (int i = p->lo; i <= p->hi; i++) {
            double dx = i * p->h - cx, dy = j * p->h - cy;
            g[node_index(N, p->bc, i, j)] = amp * exp(-(dx * dx + dy * dy) / (2.0 * sigma * sigma));
        }
    csr_mv(&p->M, g, mg);
    for (int t = 0; t < p->n; t++) ((zc *)f)[t] += mg[t];
    free(g); free(mg);
}

/* F = M f_I with f = (2π² - k²) sin(πx) sin(πy): exact solution u = sin(πx) sin(πy).  With
 * the impedance condition u still vanishes on ∂Ω but ∂u/∂n = -π sin(πs) on every side (s the
 * coordinate along the side), so the boundary datum g = ∂u/∂n - i k u = -π sin(πs) is added as
 * F += B g_I. */
void or_rhs_manufactured(const or_problem *p, double *f) {
    int N = p->N;
    zc *g = (zc *)malloc(sizeof(zc) * (size_t)p->n);
    for (int j = p->lo; j <= p->hi; j++)
        for (int i = p->lo; i <= p->hi; i++)
            g[node_index(N, p->bc, i, j)] = (2.0 * M_PI * M_PI - p->k * p->k) * sin(M_PI * i * p->h) *
                                            sin(M_PI * j * p->h);
    csr_mv(&p->M, g, (zc *)f);
    if (p->bc) {
        zc *bg = (zc *)malloc(sizeof(zc) * (size_t)p->n);
        for (int j = 0; j <= N; j++)
            for (int i = 0; i <= N; i++) {
                double v = 0.0;
                if (j == 0 || j == N) v += -M_PI * sin(M_PI * i * p->h);
                if (i == 0 || i == N) v += -M_PI * sin(M_PI * j * p->h);
                g[node_index(N, 1, i, j)] = v;
            }
        csr_mv(&p->B, g, bg);
        for (int t = 0; t < p->n; t++) ((zc *)f)[t] += bg[t];
        free(bg);
    }
    free(g);
}

/* -- domain decomposition (Eq. 3, §3) --------------------------------------------------------- */
int or_setup_dd(or_problem *p, int Sx, int Sy, int overlap, const int *ifx, const int *ify) {
    int N = p->N;
    if (Sx < 1 || Sy < 1 || overlap < 1) return OR_ERR_ARG;
    if (ifx[0] != 0 || ifx[Sx] != N || ify[0] != 0 || ify[Sy] != N) return OR_ERR_ARG;
    for (int q = 0; q < Sx; q++) if (ifx[q + 1] - ifx[q] < 2) return OR_ERR_ARG;
    for (int q = 0; q < Sy; q++) if (ify[q + 1] - ify[q] < 2) return OR_ERR_ARG;
    if (p->sub) { for (int s = 0; s < p->nsub; s++) free_sub(&p->sub[s]); free(p->sub); }
    p->Sx = Sx; p->Sy = Sy; p->nsub = Sx * Sy; p->overlap = overlap;
    p->sub = (subdomain *)calloc((size_t)p->nsub, sizeof(subdomain));
    p->have_defl = p->have_exact = 0;
    for (int py = 0; py < Sy; py++)
        for (int px = 0; px < Sx; px++) {
            subdomain *sd = &p->sub[px + py * Sx];
            /* subdomain = cells [a_p - δ, a_{p+1} + δ]; the unknowns among its nodes, less those
             * on its artificial boundary, form the local box (lo..hi: the global unknown range) */
            const int lo = p->lo, hi = p->hi;
            sd->ix0 = ifx[px] - overlap + 1 < lo ? lo : ifx[px] - overlap + 1;
            sd->ix1 = ifx[px + 1] + overlap - 1 > hi ? hi : ifx[px + 1] + overlap - 1;
            sd->iy0 = ify[py] - overlap + 1 < lo ? lo : ify[py] - overlap + 1;
            sd->iy1 = ify[py + 1] + overlap - 1 > hi ? hi : ify[py + 1] + overlap - 1;
            /* owned nodes a_p <= i < a_{p+1} (the last subdomain also owns hi): each unknown
             * owned exactly once */
            sd->ox0 = ifx[px] < lo ? lo : ifx[px];
            sd->ox1 = px == Sx - 1 ? hi : ifx[px + 1] - 1;
            sd->oy0 = ify[py] < lo ? lo : ify[py];
            sd->oy1 = py == Sy - 1 ? hi : ify[py + 1] - 1;
            sd->nx = sd->ix1 - sd->ix0 + 1;
            sd->ny = sd->iy1 - sd->iy0 + 1;
            sd->n = sd->nx * sd->ny;
            sd->mx = sd->nx / 2;
            sd->my = sd->ny / 2;
            sd->m = sd->mx * sd->my;
            sd->gidx = (int *)malloc(sizeof(int) * (size_t)sd->n);
            for (int j = 0; j < sd->ny; j++)
                for (int i = 0; i < sd->nx; i++)
                    sd->gidx[i + j * sd->nx] = node_index(N, p->bc, sd->ix0 + i, sd->iy0 + j);
            /* A_j = R_j A R_j^T: rows and columns of the box, extracted from the assembled A */
            int *g2l = (int *)malloc(sizeof(int) * (size_t)p->n);
            for (int t = 0; t < p->n; t++) g2l[t] = -1;
            for (int t = 0; t < sd->n; t++) g2l[sd->gidx[t]] = t;
            sd->A.nr = sd->A.nc = sd->n;
            sd->A.rp = (int *)malloc(sizeof(int) * (size_t)(sd->n + 1));
            sd->A.ci = (int *)malloc(sizeof(int) * 8 * (size_t)sd->n);
            sd->A.v = (double *)malloc(sizeof(double) * 8 * (size_t)sd->n);
            sd->A.vi = p->A.vi ? (double *)malloc(sizeof(double) * 8 * (size_t)sd->n) : NULL;
            int nnz = 0;
            sd->A.rp[0] = 0;
            for (int t = 0; t < sd->n; t++) {
                int g = sd->gidx[t];
                for (int q = p->A.rp[g]; q < p->A.rp[g + 1]; q++) {
                    int lc = g2l[p->A.ci[q]];
                    if (lc >= 0) {
                        sd->A.ci[nnz] = lc; sd->A.v[nnz] = p->A.v[q];
                        if (sd->A.vi) sd->A.vi[nnz] = p->A.vi[q];
                        nnz++;
                    }
                }
                sd->A.rp[t + 1] = nnz;
            }
            sd->A.nnz = nnz;
            free(g2l);
        }
    return OR_OK;
}

int or_nsub(const or_problem *p) { return p->nsub; }
void or_sub_box(const or_problem *p, int s, int *b) {
    const subdomain *sd = &p->sub[s];
    b[0] = sd->ix0; b[1] = sd->ix1; b[2] = sd->iy0; b[3] = sd->iy1;
    b[4] = sd->ox0; b[5] = sd->ox1; b[6] = sd->oy0; b[7] = sd->oy1;
}
int or_sub_n(const or_problem *p, int s) { return p->sub[s].n; }
int or_sub_m(const or_problem *p, int s) { return p->sub[s].m; }

void or_sub_restrict(const or_problem *p, int s, const double *v, double *vs) {
    const subdomain *sd = &p->sub[s];
    for (int t = 0; t < sd->n; t++) ((zc *)vs)[t] = ((const zc *)v)[sd->gidx[t]];
}
void or_sub_apply_A(const or_problem *p, int s, const double *v, double *w) {
    csr_mv(&p->sub[s].A, (const zc *)v, (zc *)w);
}
int or_sub_nnz(const or_problem *p, int s, int which) {
    return which == 0 ? p->sub[s].A.nnz : p->sub[s].Z.nnz;
}
void or_sub_get_csr(const or_problem *p, int s, int which, int *rowptr, int *col, double *val) {
    const csr *a = which == 0 ? &p->sub[s].A : &p->sub[s].Z;
    memcpy(rowptr, a->rp, sizeof(int) * (size_t)(a->nr + 1));
    memcpy(col, a->ci, sizeof(int) * (size_t)a->nnz);
    memcpy(val, a->v, sizeof(double) * (size_t)a->nnz);
}
void or_sub_get_csr_imag(const or_problem *p, int s, int which, double *val) {
    const csr *a = which == 0 ? &p->sub[s].A : &p->sub[s].Z;
    if (a->vi) memcpy(val, a->vi, sizeof(double) * (size_t)a->nnz);
    else memset(val, 0, sizeof(double) * (size_t)a->nnz);
}

/* -- Eq. 4, Eq. 5: deflation matrix and coarse matrix ---------------------------------------- */
/* 1D quadratic rational Bézier deflation matrix (n x n/2): column i (1-based) carries
 * (1,4,6,4,1)/8 on fine rows 2i-2 .. 2i+2, truncated to 1..n (zero Dirichlet outside). */
static double z1d(int fine0, int coarse0) {
    static const double w[5] = {1.0, 4.0, 6.0, 4.0, 1.0};
    int t = (fine0 + 1) - (2 * (coarse0 + 1) - 2);
    return (t >= 0 && t <= 4) ? w[t] / 8.0 : 0.0;
}

/* Z_j = Z_j^y ⊗ Z_j^x (Eq. 5), lexicographic ordering with x fastest, built entry by entry. */
static csr build_Z(int nx, int ny) {
    int mx = nx / 2, my = ny / 2, n = nx * ny;
    csr z;
    z.nr = n; z.nc = mx * my;
    z.rp = (int *)malloc(sizeof(int) * (size_t)(n + 1));
    z.ci = (int *)malloc(sizeof(int) * 9 * (size_t)n);
    z.v = (double *)malloc(sizeof(double) * 9 * (size_t)n);
    z.vi = NULL;
    int nnz = 0;
    z.rp[0] = 0;
    for (int fy = 0; fy < ny; fy++)
        for (int fx = 0; fx < nx; fx++) {
            for (int cy = 0; cy < my; cy++) {
                double wy = z1d(fy, cy);
                if (wy == 0.0) continue;
                for (int cx = 0; cx < mx; cx++) {
                    double wx = z1d(fx, cx);
                    if (wx == 0.0) continue;
                    z.ci[nnz] = cx + cy * mx;
                    z.v[nnz] = wy * wx;
                    nnz++;
                }
            }
            z.rp[fx + fy * nx + 1] = nnz;
        }
    z.nnz = nnz;
    return z;
}

/* Store a square sparse matrix in row-band form (kl, ku taken from its actual nonzeros). */
static void csr_to_band(const csr *a, bandlu *b) {
    int kl = 0, ku = 0;
    for (int r = 0; r < a->nr; r++)
        for (int t = a->rp[r]; t < a->rp[r + 1]; t++) {
            int d = a->ci[t] - r;
            if (-d > kl) kl = -d;
            if (d > ku) ku = d;
        }
    int W = 2 * kl + ku + 1;
    b->m = a->nr; b->kl = kl; b->ku = ku;
    b->ab = NULL; b->abz = NULL;
    if (a->vi) b->abz = (zc *)calloc((size_t)a->nr * (size_t)W, sizeof(zc));
    else b->ab = (double *)calloc((size_t)a->nr * (size_t)W, sizeof(double));
    b->piv = (int *)malloc(sizeof(int) * (size_t)(a->nr > 0 ? a->nr : 1));
    for (int r = 0; r < a->nr; r++)
        for (int t = a->rp[r]; t < a->rp[r + 1]; t++) {
            size_t at = (size_t)r * W + (size_t)(a->ci[t] - r + kl);
            if (a->vi) b->abz[at] = CMPLX(a->v[t], a->vi[t]);
            else b->ab[at] = a->v[t];
        }
}

int or_setup_deflation(or_problem *p) {
    if (!p->sub) return OR_ERR_STATE;
    int status = OR_OK;
#pragma omp parallel for schedule(dynamic) num_threads(or_get_threads())
    for (int s = 0; s < p->nsub; s++) {
        subdomain *sd = &p->sub[s];
        csr_free(&sd->Z); csr_free(&sd->Zt);
        bandlu_free(&sd->E); free(sd->Edense); free(sd->Edense_i);
        sd->Edense = NULL; sd->Edense_i = NULL;
        sd->Z = build_Z(sd->nx, sd->ny);
        sd->Zt = csr_transpose(&sd->Z);
        csr AZ = csr_matmul(&sd->A, &sd->Z);
        csr E = csr_matmul(&sd->Zt, &AZ);    /* E_j = Z_j^T A_j Z_j (Eq. 4) */
        if (sd->m <= 400) {
            sd->Edense = (double *)calloc((size_t)sd->m * (size_t)sd->m, sizeof(double));
            for (int r = 0; r < E.nr; r++)
                for (int t = E.rp[r]; t < E.rp[r + 1]; t++)
                    sd->Edense[(size_t)r * sd->m + E.ci[t]] = E.v[t];
            if (E.vi) {
                sd->Edense_i = (double *)calloc((size_t)sd->m * (size_t)sd->m, sizeof(double));
                for (int r = 0; r < E.nr; r++)
                    for (int t = E.rp[r]; t < E.rp[r + 1]; t++)
                        sd->Edense_i[(size_t)r * sd->m + E.ci[t]] = E.vi[t];
            }
        }
        csr_to_band(&E, &sd->E);
        int st = bandlu_factor(&sd->E);
        if (st != OR_OK) {
#pragma omp critical
            status = st;
        }
        csr_free(&AZ); csr_free(&E);
    }
    if (status == OR_OK) p->have_defl = 1;
    return status;
}

int or_setup_exact(or_problem *p) {
    if (!p->sub) return OR_ERR_STATE;
    int status = OR_OK;
#pragma omp parallel for schedule(dynamic) num_threads(or_get_threads())
    for (int s = 0; s < p->nsub; s++) {
        subdomain *sd = &p->sub[s];
        bandlu_free(&sd->Aex);
        csr_to_band(&sd->A, &sd->Aex);
        int st = bandlu_factor(&sd->Aex);
        if (st != OR_OK) {
#pragma omp critical
            status = st;
        }
    }
    if (status == OR_OK) p->have_exact = 1;
    return status;
}

void or_sub_E_band(const or_problem *p, int s, int *kl_ku) {
    kl_ku[0] = p->sub[s].E.kl; kl_ku[1] = p->sub[s].E.ku;
}
void or_sub_E_dense(const or_problem *p, int s, double *E) {
    const subdomain *sd = &p->sub[s];
    if (sd->Edense) memcpy(E, sd->Edense, sizeof(double) * (size_t)sd->m * (size_t)sd->m);
}
void or_sub_E_dense_imag(const or_problem *p, int s, double *E) {
    const subdomain *sd = &p->sub[s];
    if (sd->Edense_i) memcpy(E, sd->Edense_i, sizeof(double) * (size_t)sd->m * (size_t)sd->m);
    else if (sd->Edense) memset(E, 0, sizeof(double) * (size_t)sd->m * (size_t)sd->m);
}
void or_sub_apply_Z(const or_problem *p, int s, const double *c, double *f) {
    csr_mv(&p->sub[s].Z, (const zc *)c, (zc *)f);
}
void or_sub_apply_Zt(const or_problem *p, int s, const double *f, double *c) {
    csr_mv(&p->sub[s].Zt, (const zc *)f, (zc *)c);
}
int or_sub_coarse_solve(const or_problem *p, int s, const double *y, double *x) {
    const subdomain *sd = &p->sub[s];
    memcpy(x, y, sizeof(zc) * (size_t)sd->m);
    bandlu_solve(&sd->E, (zc *)x);
    return OR_OK;
}

/* Q_j r = Z_j E_j^{-1} Z_j^T r (Eq. 4). */
static void apply_Q(const subdomain *sd, const zc *r, zc *out, zc *cw) {
    csr_mv(&sd->Zt, r, cw);
    bandlu_solve(&sd->E, cw);
    csr_mv(&sd->Z, cw, out);
}

/* P_j v = v - A_j Q_j v (Eq. 4).  work: 2n + m. */
static void apply_P(const subdomain *sd, const zc *v, zc *out, zc *work) {
    zc *q = work, *aq = work + sd->n, *cw = work + 2 * sd->n;
    apply_Q(sd, v, q, cw);
    csr_mv(&sd->A, q, aq);
    for (int t = 0; t < sd->n; t++) out[t] = v[t] - aq[t];
}

/* w = P_j A_j v.  work: 3n + m. */
static void apply_PA(const subdomain *sd, const zc *v, zc *w, zc *work) {
    zc *t = work + 2 * sd->n + sd->m;
    csr_mv(&sd->A, v, t);
    apply_P(sd, t, w, work);
}

void or_sub_apply_PA(const or_problem *p, int s, const double *v, double *w) {
    const subdomain *sd = &p->sub[s];
    zc *work = (zc *)malloc(sizeof(zc) * (size_t)(3 * sd->n + sd->m));
    apply_PA(sd, (const zc *)v, (zc *)w, work);
    free(work);
}
void or_sub_apply_P(const or_problem *p, int s, const double *v, double *w) {
    const subdomain *sd = &p->sub[s];
    zc *work = (zc *)malloc(sizeof(zc) * (size_t)(2 * sd->n + sd->m));
    apply_P(sd, (const zc *)v, (zc *)w, work);
    free(work);
}

/* -- Krylov helpers ---------------------------------------------------------------------------- */
static double nrm2(const zc *x, int n) {
    double s = 0.0;
    for (int t = 0; t < n; t++) s += creal(x[t]) * creal(x[t]) + cimag(x[t]) * cimag(x[t]);
    return sqrt(s);
}
static zc dotc(const zc *a, const zc *b, int n) {    /* a^H b */
    zc s = 0;
    for (int t = 0; t < n; t++) s += conj(a[t]) * b[t];
    return s;
}

/* Classical Gram-Schmidt applied twice: w ⟂ V[0..j], h[0..j] = accumulated coefficients.
 * With par != 0 (the global outer vectors) the independent dot products and the independent
 * vector elements are shared among threads; every value is still computed by one thread in
 * the same order, so the result does not depend on the thread count. */
static double cgs2(const zc *V, int n, int j, zc *w, zc *h, zc *htmp, int par) {
    for (int l = 0; l <= j; l++) h[l] = 0;
    for (int pass = 0; pass < 2; pass++) {
#pragma omp parallel for schedule(static) num_threads(or_get_threads()) if (par)
        for (int l = 0; l <= j; l++) htmp[l] = dotc(V + (size_t)l * n, w, n);
#pragma omp parallel for schedule(static) num_threads(or_get_threads()) if (par)
        for (int t = 0; t < n; t++) {
            zc s = w[t];
            for (int l = 0; l <= j; l++) s -= htmp[l] * V[(size_t)l * n + t];
            w[t] = s;
        }
        for (int l = 0; l <= j; l++) h[l] += htmp[l];
    }
    return nrm2(w, n);
}

/* The outer orthogonalisation exactly as or_solve runs it (threads over the independent dots
 * and elements): w is made orthogonal to the nv vectors of V (n x nv, column-major) by CGS2,
 * h[0..nv) receives the coefficients, the return value is ||w||.  Exposed for pins. */
double or_cgs2(const double *V_c128, int n, int nv, double *w_c128, double *h_c128) {
    if (nv < 1 || n < 1) return nrm2((const zc *)w_c128, n > 0 ? n : 0);
    zc *htmp = (zc *)malloc(sizeof(zc) * (size_t)nv);
    double r = cgs2((const zc *)V_c128, n, nv - 1, (zc *)w_c128, (zc *)h_c128, htmp, 1);
    free(htmp);
    return r;
}

/* Complex Givens rotation G = [c s; -conj(s) c] with c real, chosen so that
 * G [a; b] = [r; 0] (the standard complex form, cf. Bindel, Demmel, Kahan & Marques,
 * ACM TOMS 28 (2002)), magnitudes taken with hypot. */
static void givens(zc a, zc b, double *c, zc *s, zc *r) {
    double aa = cabs(a), bb = cabs(b);
    if (bb == 0.0) { *c = 1.0; *s = 0.0; *r = a; return; }
    if (aa == 0.0) { *c = 0.0; *s = conj(b) / bb; *r = bb; return; }
    double t = hypot(aa, bb);
    zc ph = a / aa;
    *c = aa / t;
    *s = ph * conj(b) / t;
    *r = ph * t;
}

/* Back substitution with the k x k upper triangle of H (column-major, leading dim ldh). */
static void upper_solve(const zc *H, int ldh, int k, const zc *g, zc *y) {
    for (int i = k - 1; i >= 0; i--) {
        zc s = g[i];
        for (int l = i + 1; l < k; l++) s -= H[i + (size_t)l * ldh] * y[l];
        y[i] = s / H[i + (size_t)i * ldh];
    }
}

/* -- inner solve: restarted GMRES on P_j A_j u = P_j f (Eq. 4), relative tolerance on the
 *    deflated residual ||P_j (f - A_j u)|| / ||P_j f|| (§3), then the solution of A_j x = f is
 *    completed as x = u + Q_j (f - A_j u). ---------------------------------------------------- */
static int sub_gmres(const subdomain *sd, const zc *f, const zc *x0, double tol, int restart,
                     int maxit, zc *x, int *its_out) {
    const int n = sd->n, R = restart;
    zc *V = (zc *)malloc(sizeof(zc) * (size_t)n * (size_t)(R + 1));
    zc *H = (zc *)calloc((size_t)(R + 1) * (size_t)R, sizeof(zc));
    zc *g = (zc *)malloc(sizeof(zc) * (size_t)(R + 1));
    zc *sn = (zc *)malloc(sizeof(zc) * (size_t)R);
    double *cs = (double *)malloc(sizeof(double) * (size_t)R);
    zc *y = (zc *)malloc(sizeof(zc) * (size_t)(R + 1));
    zc *htmp = (zc *)malloc(sizeof(zc) * (size_t)(R + 1));
    zc *u = (zc *)malloc(sizeof(zc) * (size_t)n);
    zc *r = (zc *)malloc(sizeof(zc) * (size_t)n);
    zc *w = (zc *)malloc(sizeof(zc) * (size_t)n);
    zc *work = (zc *)malloc(sizeof(zc) * (size_t)(3 * n + sd->m));
    int status = OR_OK, total = 0;

    apply_P(sd, f, r, work);
    double ref = nrm2(r, n);                       /* ||P_j f|| */
    for (int t = 0; t < n; t++) u[t] = x0 ? x0[t] : 0.0;

    for (;;) {
        /* true deflated residual of the current iterate */
        csr_mv(&sd->A, u, w);
        for (int t = 0; t < n; t++) w[t] = f[t] - w[t];
        apply_P(sd, w, r, work);
        double beta = nrm2(r, n);
        if (!isfinite(beta)) { status = OR_ERR_NONFINITE; break; }
        if (beta <= tol * ref || total >= maxit) break;
        for (int t = 0; t < n; t++) V[t] = r[t] / beta;
        for (int l = 0; l <= R; l++) g[l] = 0;
        g[0] = beta;
        int kcols = 0, done = 0;
        for (int i = 0; i < R; i++) {
            zc *hcol = H + (size_t)i * (R + 1);
            apply_PA(sd, V + (size_t)i * n, w, work);
            double hn = cgs2(V, n, i, w, hcol, htmp, 0);
            total++;
            for (int l = 0; l < i; l++) {          /* previous rotations */
                zc a = hcol[l], b = hcol[l + 1];
                hcol[l] = cs[l] * a + sn[l] * b;
                hcol[l + 1] = -conj(sn[l]) * a + cs[l] * b;
            }
            zc rr;
            givens(hcol[i], (zc)hn, &cs[i], &sn[i], &rr);
            hcol[i] = rr;
            hcol[i + 1] = 0;
            g[i + 1] = -conj(sn[i]) * g[i];
            g[i] = cs[i] * g[i];
            kcols = i + 1;
            int breakdown = !(hn > 0.0);
            if (!breakdown)
                for (int t = 0; t < n; t++) V[(size_t)(i + 1) * n + t] = w[t] / hn;
            if (cabs(g[i + 1]) <= tol * ref || total >= maxit || breakdown) { done = 1; break; }
        }
        upper_solve(H, R + 1, kcols, g, y);
        for (int l = 0; l < kcols; l++) {
            const zc *v = V + (size_t)l * n;
            for (int t = 0; t < n; t++) u[t] += y[l] * v[t];
        }
        if (done) break;
    }
    /* completion x = u + Q_j (f - A_j u) */
    csr_mv(&sd->A, u, w);
    for (int t = 0; t < n; t++) w[t] = f[t] - w[t];
    apply_Q(sd, w, r, work);
    for (int t = 0; t < n; t++) x[t] = u[t] + r[t];
    *its_out = total;
    free(V); free(H); free(g); free(sn); free(cs); free(y); free(htmp);
    free(u); free(r); free(w); free(work);
    return status;
}

int or_sub_solve(const or_problem *p, int s, const double *f, const double *x0, double tol,
                 int restart, int maxit, double *x, int *its) {
    if (!p->have_defl) return OR_ERR_STATE;
    return sub_gmres(&p->sub[s], (const zc *)f, (const zc *)x0, tol, restart, maxit, (zc *)x, its);
}

int or_sub_solve_exact(const or_problem *p, int s, const double *f, double *x) {
    if (!p->have_exact) return OR_ERR_STATE;
    const subdomain *sd = &p->sub[s];
    memcpy(x, f, sizeof(zc) * (size_t)sd->n);
    bandlu_solve(&sd->Aex, (zc *)x);
    return OR_OK;
}

/* -- RAS (Eq. 3): z = Σ_j R_j^T D_j A_j^{-1} R_j v, D_j the ownership indicator ------------ */
int or_ras_apply(const or_problem *p, const double *v_, double *z_, double inner_tol,
                 int inner_restart, int inner_maxit, long long *its_total, int *its_max,
                 long long *hits) {
    const zc *v = (const zc *)v_;
    zc *z = (zc *)z_;
    if (inner_tol > 0 && !p->have_defl) return OR_ERR_STATE;
    if (inner_tol <= 0 && !p->have_exact) return OR_ERR_STATE;
    long long tot = 0, nh = 0;
    int mx = 0, status = OR_OK;
#pragma omp parallel for schedule(dynamic) num_threads(or_get_threads()) \
    reduction(+ : tot, nh) reduction(max : mx)
    for (int s = 0; s < p->nsub; s++) {
        const subdomain *sd = &p->sub[s];
        zc *fs = (zc *)malloc(sizeof(zc) * (size_t)sd->n);
        zc *xs = (zc *)malloc(sizeof(zc) * (size_t)sd->n);
        for (int t = 0; t < sd->n; t++) fs[t] = v[sd->gidx[t]];
        int its = 0, st;
        if (inner_tol > 0) {
            st = sub_gmres(sd, fs, NULL, inner_tol, inner_restart, inner_maxit, xs, &its);
        } else {
            memcpy(xs, fs, sizeof(zc) * (size_t)sd->n);
            bandlu_solve(&sd->Aex, xs);
            st = OR_OK;
        }
        if (st != OR_OK) {
#pragma omp critical
            status = st;
        }
        tot += its;
        if (its > mx) mx = its;
        if (inner_tol > 0 && its >= inner_maxit) nh++;
        for (int j = sd->oy0; j <= sd->oy1; j++)
            for (int i = sd->ox0; i <= sd->ox1; i++) {
                int l = (i - sd->ix0) + (j - sd->iy0) * sd->nx;
                z[sd->gidx[l]] = xs[l];
            }
        free(fs); free(xs);
    }
    if (its_total) *its_total = tot;
    if (its_max) *its_max = mx;
    if (hits) *hits = nh;
    return status;
}

/* -- outer solve: restarted flexible GMRES, right-preconditioned by RAS (§3; Saad, SIAM J.
 *    Sci. Comput. 14 (1993)).  Stops on ||f - A x|| <= tol ||f||, checked on the true
 *    residual at every restart and at exit. --------------------------------------------------- */
/* ------------------------------------------------------------------------------------------ */
/* Two-level variant (the paper's §4 names a coarse space as the next step): the grid coarse    */
/* space — P1 on a coarser mesh of the same triangulation, H = c h — with P1 interpolation P, */
/* restriction Pᵀ and the coarse operator rediscretised on that mesh with its mass lumped      */
/* (A_H = K_H - k² diag(row sums of M_H)), solved exactly by banded LU.                        */
/* ------------------------------------------------------------------------------------------ */
int or_setup_coarse_grid(or_problem *p, int c) {
    if (!p || p->bc != 0 || c < 2 || p->N % c != 0 || p->N / c < 2) return OR_ERR_ARG;
    cgrid *g = &p->cg;
    csr_free(&g->P); csr_free(&g->Pt); free(g->ab); free(g->piv);
    memset(g, 0, sizeof(*g));
    const int N = p->N, Nc = N / c, mc = Nc - 1, nH = mc * mc;
    g->c = c; g->Nc = Nc; g->mc = mc; g->nH = nH;
    /* P: value at each fine interior node of the coarse piecewise-linear function, by barycentric
     * coordinates in the coarse triangle that contains the node */
    rowacc acc;
    acc.col = (int *)malloc(sizeof(int) * 8 * (size_t)p->n);
    acc.val = (double *)malloc(sizeof(double) * 8 * (size_t)p->n);
    acc.cnt = (int *)calloc((size_t)p->n, sizeof(int));
    for (int j = 1; j < N; j++)
        for (int i = 1; i < N; i++) {
            const int cx0 = i / c, cy0 = j / c;
            const double a = (double)(i - cx0 * c) / c, b = (double)(j - cy0 * c) / c;
            int vx[3], vy[3];
            double wt[3];
            if (p->diag == 0) {          /* triangles (cx0,cy0),(cx0+1,cy0),(cx0+1,cy0+1) and (cx0,cy0),(cx0+1,cy0+1),(cx0,cy0+1) */
                if (a >= b) { vx[0] = cx0; vy[0] = cy0; wt[0] = 1 - a; vx[1] = cx0 + 1; vy[1] = cy0; wt[1] = a - b;
                              vx[2] = cx0 + 1; vy[2] = cy0 + 1; wt[2] = b; }
                else { vx[0] = cx0; vy[0] = cy0; wt[0] = 1 - b; vx[1] = cx0 + 1; vy[1] = cy0 + 1; wt[1] = a;
                       vx[2] = cx0; vy[2] = cy0 + 1; wt[2] = b - a; }
            } else {                     /* triangles (cx0,cy0),(cx0+1,cy0),(cx0,cy0+1) and (cx0+1,cy0),(cx0+1,cy0+1),(cx0,cy0+1) */
                if (a + b <= 1) { vx[0] = cx0; vy[0] = cy0; wt[0] = 1 - a - b; vx[1] = cx0 + 1; vy[1] = cy0; wt[1] = a;
                                  vx[2] = cx0; vy[2] = cy0 + 1; wt[2] = b; }
                else { vx[0] = cx0 + 1; vy[0] = cy0; wt[0] = 1 - b; vx[1] = cx0 + 1; vy[1] = cy0 + 1; wt[1] = a + b - 1;
                       vx[2] = cx0; vy[2] = cy0 + 1; wt[2] = 1 - a; }
            }
            const int r = (i - 1) + (j - 1) * (N - 1);
            for (int t = 0; t < 3; t++) {
                if (wt[t] == 0.0 || vx[t] < 1 || vy[t] < 1 || vx[t] > mc || vy[t] > mc) continue;
                acc_add(&acc, r, (vx[t] - 1) + (vy[t] - 1) * mc, wt[t]);
            }
        }
    g->P = acc_to_csr(&acc, p->n);
    g->P.nc = nH;
    g->Pt = csr_transpose(&g->P);
    free(acc.col); free(acc.val); free(acc.cnt);
    /* A_H from the coarse mesh's own element assembly, mass lumped, in band storage */
    or_problem *q = or_create(Nc, p->k, p->diag);
    if (!q) return OR_ERR_ARG;
    const int kl = mc + 1, W = 3 * kl + 1;
    g->kl = kl;
    g->ab = (double *)calloc((size_t)nH * W, sizeof(double));
    g->piv = (int *)malloc(sizeof(int) * (size_t)nH);
    double *ab = g->ab;
    const double k2 = p->k * p->k;
#define AB(r, col) ab[(size_t)(r) * W + (size_t)((col) - (r) + kl)]
    /* lumped mass: the integral of the coarse hat function, i.e. the row sum of the full mass
     * matrix with the boundary columns included = area of its support / 3 = 6 (H^2/2) / 3 = H^2 at
     * every interior node (summing only the interior columns would lose mass next to the boundary) */
    const double H = 1.0 / Nc, mlump = H * H;
    for (int r = 0; r < nH; r++) {
        for (int t = q->K.rp[r]; t < q->K.rp[r + 1]; t++) AB(r, q->K.ci[t]) += q->K.v[t];
        AB(r, r) -= k2 * mlump;
    }
#undef AB
    or_destroy(q);
    int st = or_band_lu(nH, kl, kl, ab, g->piv);
    if (st != OR_OK) return st;
    g->have = 1;
    return OR_OK;
}

int or_cg_n(const or_problem *p) { return p->cg.have ? p->cg.nH : 0; }
void or_cg_apply_P(const or_problem *p, const double *uH, double *u) {
    csr_mv(&p->cg.P, (const zc *)uH, (zc *)u);
}
void or_cg_apply_Pt(const or_problem *p, const double *v, double *vH) {
    csr_mv(&p->cg.Pt, (const zc *)v, (zc *)vH);
}
/* xH = A_H⁻¹ yH */
void or_cg_solve(const or_problem *p, const double *yH, double *xH) {
    memcpy(xH, yH, sizeof(zc) * (size_t)p->cg.nH);
    band_solve_z(p->cg.nH, p->cg.kl, p->cg.kl, p->cg.ab, p->cg.piv, (zc *)xH);
}

int or_solve(const or_problem *p, const double *f_, double *x_, const or_solve_params *prm,
             or_stats *st, double *hist, int hcap) {
    const zc *f = (const zc *)f_;
    zc *x = (zc *)x_;
    const int n = p->n;
    const int R = prm->outer_restart < prm->outer_maxit ? prm->outer_restart : prm->outer_maxit;
    memset(st, 0, sizeof(*st));
    for (int t = 0; t < n; t++) x[t] = 0;
    double fn = nrm2(f, n);
    if (fn == 0.0) { st->rel_res_true = 0.0; return OR_OK; }
    zc *V = (zc *)malloc(sizeof(zc) * (size_t)n * (size_t)(R + 1));
    zc *Zb = (zc *)malloc(sizeof(zc) * (size_t)n * (size_t)R);
    zc *H = (zc *)calloc((size_t)(R + 1) * (size_t)R, sizeof(zc));
    zc *g = (zc *)malloc(sizeof(zc) * (size_t)(R + 1));
    zc *sn = (zc *)malloc(sizeof(zc) * (size_t)R);
    double *cs = (double *)malloc(sizeof(double) * (size_t)R);
    zc *y = (zc *)malloc(sizeof(zc) * (size_t)(R + 1));
    zc *htmp = (zc *)malloc(sizeof(zc) * (size_t)(R + 1));
    zc *r = (zc *)malloc(sizeof(zc) * (size_t)n);
    zc *w = (zc *)malloc(sizeof(zc) * (size_t)n);
    const int two = prm->two_level != 0;
    if (two && !p->cg.have) {
        free(V); free(Zb); free(H); free(g); free(sn); free(cs); free(y); free(htmp); free(r); free(w);
        st->status = OR_ERR_STATE;
        return OR_ERR_STATE;
    }
    const int nH = two ? p->cg.nH : 1;
    zc *vH = (zc *)malloc(sizeof(zc) * (size_t)nH), *xH = (zc *)malloc(sizeof(zc) * (size_t)nH);
    zc *tv = (zc *)malloc(sizeof(zc) * (size_t)(two ? n : 1)), *z2 = (zc *)malloc(sizeof(zc) * (size_t)(two ? n : 1));
    int status = OR_OK, total = 0, nh = 0;
    long long inner_tot = 0, hits = 0;
    int inner_max = 0;
    double relres = 1.0;

    for (;;) {
        csr_mv(&p->A, x, w);
        for (int t = 0; t < n; t++) r[t] = f[t] - w[t];
        double beta = nrm2(r, n);
        relres = beta / fn;
        if (!isfinite(beta)) { status = OR_ERR_NONFINITE; break; }
        if (relres <= prm->outer_tol) break;
        if (total >= prm->outer_maxit) { status = OR_ERR_NO_CONVERGENCE; break; }
        for (int t = 0; t < n; t++) V[t] = r[t] / beta;
        for (int l = 0; l <= R; l++) g[l] = 0;
        g[0] = beta;
        int kcols = 0;
        for (int j = 0; j < R; j++) {
            zc *hcol = H + (size_t)j * (R + 1);
            zc *zj = Zb + (size_t)j * n;
            long long it_tot = 0, it_hits = 0;
            int it_max = 0;
            const zc *vj = V + (size_t)j * n;
            int s2;
            if (two) {
                /* coarse correction z0 = P A_H⁻¹ Pᵀ v, then RAS on the residual v - A z0 */
                csr_mv(&p->cg.Pt, vj, vH);
                memcpy(xH, vH, sizeof(zc) * (size_t)nH);
                band_solve_z(nH, p->cg.kl, p->cg.kl, p->cg.ab, p->cg.piv, xH);
                csr_mv(&p->cg.P, xH, zj);
                csr_mv(&p->A, zj, w);
                for (int t = 0; t < n; t++) tv[t] = vj[t] - w[t];
                s2 = or_ras_apply(p, (const double *)tv, (double *)z2, prm->inner_tol, prm->inner_restart,
                                  prm->inner_maxit, &it_tot, &it_max, &it_hits);
                for (int t = 0; t < n; t++) zj[t] += z2[t];
            } else {
                s2 = or_ras_apply(p, (const double *)vj, (double *)zj, prm->inner_tol, prm->inner_restart,
                                  prm->inner_maxit, &it_tot, &it_max, &it_hits);
            }
            if (s2 != OR_OK) { status = s2; break; }
            inner_tot += it_tot; hits += it_hits;
            if (it_max > inner_max) inner_max = it_max;
            csr_mv(&p->A, zj, w);
            double hn = cgs2(V, n, j, w, hcol, htmp, 1);
            total++;
            for (int l = 0; l < j; l++) {
                zc a = hcol[l], b = hcol[l + 1];
                hcol[l] = cs[l] * a + sn[l] * b;
                hcol[l + 1] = -conj(sn[l]) * a + cs[l] * b;
            }
            zc rr;
            givens(hcol[j], (zc)hn, &cs[j], &sn[j], &rr);
            hcol[j] = rr;
            hcol[j + 1] = 0;
            g[j + 1] = -conj(sn[j]) * g[j];
            g[j] = cs[j] * g[j];
            kcols = j + 1;
            if (hist && nh < hcap) hist[nh++] = cabs(g[j + 1]) / fn;
            int breakdown = !(hn > 0.0);
            if (!breakdown)
                for (int t = 0; t < n; t++) V[(size_t)(j + 1) * n + t] = w[t] / hn;
            if (cabs(g[j + 1]) <= prm->outer_tol * fn || total >= prm->outer_maxit || breakdown)
                break;
        }
        if (status != OR_OK) break;
        upper_solve(H, R + 1, kcols, g, y);
        for (int l = 0; l < kcols; l++) {
            const zc *zl = Zb + (size_t)l * n;
            for (int t = 0; t < n; t++) x[t] += y[l] * zl[t];
        }
    }
    st->outer_its = total;
    st->status = status;
    st->rel_res_true = relres;
    st->inner_its_total = inner_tot;
    st->inner_its_avg = total > 0 ? (double)inner_tot / ((double)total * p->nsub) : 0.0;
    st->inner_its_max = inner_max;
    st->inner_maxit_hits = hits;
    st->n_history = nh;
    free(V); free(Zb); free(H); free(g); free(sn); free(cs); free(y); free(htmp); free(r); free(w);
    free(vH); free(xH); free(tv); free(z2);
    return status;
}
