/*
 * hdd_oracle.h — plain, slow CPU reference of the method (TEST INFRASTRUCTURE ONLY).
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may load this
 * library.  It shares no code, header or table with the CUDA path.
 *
 * Everything is complex128 (C99 double complex); real matrices are real CSR.
 * Model problem: -Δu - k²u = f on (0,1)², u = 0 on the boundary (§2, Eq. 1), P1 elements on
 * a uniform mesh with N intervals per side (Eq. 2).  Variant (§3 names the solver fit for
 * Sommerfeld problems as well): the first-order absorbing condition ∂u/∂n - i k u = 0 on all
 * of ∂Ω instead, which makes A complex symmetric and every mesh node an unknown.  One-level RAS (Eq. 3) wrapped by FGMRES;
 * subdomain systems solved by GMRES preconditioned with two-level deflation (Eq. 4, Eq. 5).
 */
#ifndef HDD_ORACLE_H
#define HDD_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct or_problem or_problem;

enum {
    OR_OK = 0,
    OR_ERR_ARG = 1,
    OR_ERR_STATE = 2,
    OR_ERR_SINGULAR = 3,
    OR_ERR_NO_CONVERGENCE = 4,
    OR_ERR_NONFINITE = 5
};

typedef struct {
    double outer_tol;     /* relative residual ||f-Ax||/||f|| (§3) */
    int outer_restart;
    int outer_maxit;
    double inner_tol;     /* relative deflated residual; <= 0 selects the direct (LU) local solve */
    int inner_restart;
    int inner_maxit;
    int two_level;        /* 1: hybrid two-level preconditioner with the grid coarse space       */
} or_solve_params;

typedef struct {
    int outer_its;
    int status;
    double rel_res_true;
    long long inner_its_total;
    double inner_its_avg;     /* total inner its / (outer its x #subdomains) */
    int inner_its_max;
    long long inner_maxit_hits;
    int n_history;
} or_stats;

/* -- problem and assembly (Eq. 2) ------------------------------------------------------- */
or_problem *or_create(int N, double k, int diag);            /* Dirichlet                   */
or_problem *or_create_bc(int N, double k, int diag, int bc); /* bc: 0 Dirichlet, 1 impedance */
void or_destroy(or_problem *p);
int or_n(const or_problem *p);
int or_nnz(const or_problem *p, int which);           /* which: 0 = A, 1 = K, 2 = M, 3 = B  */
void or_get_csr(const or_problem *p, int which, int *rowptr, int *col, double *val);
void or_get_csr_imag(const or_problem *p, int which, double *val);   /* zeros if real     */
void or_apply_global(const or_problem *p, int which, const double *x_c128, double *y_c128);

/* -- right-hand sides (§3) ---------------------------------------------------------------- */
void or_rhs_point(const or_problem *p, double x, double y, double amp, double *f_c128);
void or_rhs_gauss(const or_problem *p, double cx, double cy, double sigma, double amp,
                  double *f_c128);
void or_rhs_manufactured(const or_problem *p, double *f_c128);

/* -- domain decomposition (Eq. 3, §3) ------------------------------------------------------ */
int or_setup_dd(or_problem *p, int Sx, int Sy, int overlap, const int *ifx, const int *ify);
int or_nsub(const or_problem *p);
void or_sub_box(const or_problem *p, int s, int *box8);     /* ix0 ix1 iy0 iy1 ox0 ox1 oy0 oy1 */
int or_sub_n(const or_problem *p, int s);
int or_sub_m(const or_problem *p, int s);
void or_sub_restrict(const or_problem *p, int s, const double *v_c128, double *vs_c128);
void or_sub_apply_A(const or_problem *p, int s, const double *v_c128, double *w_c128);
int or_sub_nnz(const or_problem *p, int s, int which);       /* 0 = A_s, 1 = Z_s            */
void or_sub_get_csr(const or_problem *p, int s, int which, int *rowptr, int *col, double *val);
void or_sub_get_csr_imag(const or_problem *p, int s, int which, double *val);

/* -- deflation (Eq. 4, Eq. 5) ------------------------------------------------------------- */
int or_setup_deflation(or_problem *p);
int or_setup_exact(or_problem *p);
void or_sub_E_band(const or_problem *p, int s, int *kl_ku);
void or_sub_E_dense(const or_problem *p, int s, double *E);  /* m x m row-major, unfactored */
void or_sub_E_dense_imag(const or_problem *p, int s, double *E);    /* its imaginary part  */
void or_sub_apply_Z(const or_problem *p, int s, const double *c_c128, double *f_c128);
void or_sub_apply_Zt(const or_problem *p, int s, const double *f_c128, double *c_c128);
int or_sub_coarse_solve(const or_problem *p, int s, const double *y_c128, double *x_c128);
void or_sub_apply_PA(const or_problem *p, int s, const double *v_c128, double *w_c128);
void or_sub_apply_P(const or_problem *p, int s, const double *v_c128, double *w_c128);
int or_sub_solve(const or_problem *p, int s, const double *f_c128, const double *x0_c128,
                 double tol, int restart, int maxit, double *x_c128, int *its);
int or_sub_solve_exact(const or_problem *p, int s, const double *f_c128, double *x_c128);

/* -- RAS preconditioner and outer FGMRES (Eq. 3, §3) -------------------------------------- */
int or_ras_apply(const or_problem *p, const double *v_c128, double *z_c128, double inner_tol,
                 int inner_restart, int inner_maxit, long long *inner_its_total,
                 int *inner_its_max, long long *maxit_hits);
int or_solve(const or_problem *p, const double *f_c128, double *x_c128, const or_solve_params *prm,
             or_stats *st, double *res_history, int history_cap);

/* -- two-level variant: grid coarse space (P1 on the mesh of N/c intervals, lumped mass) ----- */
/* z = Q v + M_RAS⁻¹ (v - A Q v), Q = P A_H⁻¹ Pᵀ (coarse correction first, then one-level RAS)   */
int or_setup_coarse_grid(or_problem *p, int c);             /* Dirichlet only; c | N        */
int or_cg_n(const or_problem *p);                           /* coarse unknowns (N/c - 1)²  */
void or_cg_apply_P(const or_problem *p, const double *uH_c128, double *u_c128);
void or_cg_apply_Pt(const or_problem *p, const double *v_c128, double *vH_c128);
void or_cg_solve(const or_problem *p, const double *yH_c128, double *xH_c128);

/* -- outer CGS2 as or_solve applies it (exposed for pins) ---------------------------------- */
double or_cgs2(const double *V_c128, int n, int nv, double *w_c128, double *h_c128);

/* -- banded LU with partial pivoting, row-band storage (exposed for pins) ----------------- */
int or_band_lu(int m, int kl, int ku, double *ab, int *piv);
void or_band_solve(int m, int kl, int ku, const double *ab, const int *piv, double *b_c128);
int or_band_lu_z(int m, int kl, int ku, double *ab_c128, int *piv);      /* complex band   */
void or_band_solve_z(int m, int kl, int ku, const double *ab_c128, const int *piv, double *b_c128);

void or_set_threads(int nthreads);
int or_get_threads(void);

#ifdef __cplusplus
}
#endif
#endif
