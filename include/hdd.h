/*
 * hdd.h — C ABI of the GB300 Helmholtz domain-decomposition solver.
 *
 * Problem (§2, Eq. 1): -Δu - k²u = f on (0,1)², u = 0 on ∂Ω, P1 finite elements on a uniform
 * mesh of N intervals per side with every cell split along one diagonal (Eq. 2).  The unknowns
 * are the (N-1)² interior nodes, index (i-1) + (j-1)(N-1) for node (i/N, j/N), x fastest.
 *
 * Solver (§3): flexible GMRES, right-preconditioned by one-level restricted additive Schwarz
 * M⁻¹ = Σ_j R_jᵀ D_j A_j⁻¹ R_j (Eq. 3) on an overlapping Cartesian partition; every local
 * system A_j ũ_j = f̃_j is solved inexactly by GMRES on P_j A_j ũ = P_j f̃ with the two-level
 * deflation P_j = I - A_j Z_j E_j⁻¹ Z_jᵀ, E_j = Z_jᵀ A_j Z_j (Eq. 4), Z_j = Z_jʸ ⊗ Z_jˣ built from
 * the quadratic rational Bézier stencil (1/8)[1 4 6 4 1] (Eq. 5).  All subdomain solves (and all
 * right-hand sides) run at once on the GPU.
 *
 * Conventions for every entry point:
 *  - Vectors passed as `*_dev` are caller-owned DEVICE pointers of interleaved complex128
 *    (re, im doubles), one vector of (N-1)² entries per right-hand side, stored RHS-major.
 *    They must be 16-byte aligned and live on the context's device.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is enqueued on it; calls
 *    that return statistics synchronise it before returning.
 *  - Every call returns an hdd_status and never aborts the process; after an error the context
 *    can still be destroyed.  hdd_last_error() gives a one-line description.
 *  - The library owns all of its internal device memory (allocated in the setup calls and in
 *    hdd_solve when larger work buffers are needed; freed by hdd_destroy).
 *  - A context is not thread-safe; use one context per host thread.
 *  - Required call order: hdd_create → hdd_assemble → hdd_setup_dd → hdd_setup_deflation
 *    (and/or hdd_setup_exact) → hdd_solve / test hooks.  Out-of-order calls return
 *    HDD_ERR_STATE.  Calling a setup step again invalidates the later ones.
 */
#ifndef HDD_H
#define HDD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hdd_ctx hdd_ctx;

typedef enum {
    HDD_OK = 0,
    HDD_ERR_INVALID_ARG = 1,     /* NULL pointer, size out of range, misaligned pointer      */
    HDD_ERR_STATE = 2,           /* call order violated                                      */
    HDD_ERR_OOM = 3,             /* device allocation failed                                 */
    HDD_ERR_CUDA = 4,            /* a CUDA runtime call failed                               */
    HDD_ERR_SINGULAR_COARSE = 5, /* zero pivot in the LU of some E_j (Eq. 4)                 */
    HDD_ERR_SINGULAR_LOCAL = 6,  /* zero pivot in the LU of some A_j (direct local solve)    */
    HDD_ERR_NO_CONVERGENCE = 7,  /* outer FGMRES reached outer_maxit above the tolerance     */
    HDD_ERR_BREAKDOWN = 8,       /* reserved                                                 */
    HDD_ERR_NONFINITE = 9,       /* NaN/Inf met in a residual                                */
    HDD_ERR_TIMEOUT = 10         /* a bounded device-side wait gave up (see hdd_cnn_infer)   */
} hdd_status;

/* Create a context on CUDA device `device`.  *out receives the handle. */
hdd_status hdd_create(hdd_ctx **out, int device);

/* Free every device and host resource of the context (NULL is accepted). */
void hdd_destroy(hdd_ctx *ctx);

/* Static string naming a status code. */
const char *hdd_status_str(hdd_status s);

/* Description of the most recent error on this context ("" if none). */
const char *hdd_last_error(const hdd_ctx *ctx);

/* ---------------------------------------------------------------------------------------- */
/* Assembly (§2, Eq. 2).  The matrix is never stored: with constant k and a uniform mesh the */
/* assembled P1 operator is the 7-point stencil                                              */
/*   centre 4 - k²h²/2, edge neighbours -1 - k²h²/12, the two corners joined by the cell      */
/*   diagonals -k²h²/12 (SW/NE for diag = 0, NW/SE for diag = 1),                            */
/* which every kernel applies matrix-free.                                                   */
/*                                                                                          */
/* bc = 1 selects the Sommerfeld variant (§3: the solver is meant for non-symmetric          */
/* Sommerfeld problems too): the first-order absorbing condition du/dn - i k u = 0 on all    */
/* four sides, so every mesh node 0 <= i, j <= N is an unknown ((N+1)² per vector, index     */
/* i + j(N+1)) and A = K - k²M - i k B, B the P1 boundary mass matrix (h/3 centre, h/6 along */
/* the side): complex symmetric, with the interior stencil above on interior rows.  Local    */
/* matrices keep these rows where a box meets the boundary of the square (Dirichlet on its   */
/* artificial sides); E and A_j are then complex and are factored as their real equivalents. */
/* The learned warm start serves bc = 0 only.                                               */
/* ---------------------------------------------------------------------------------------- */
typedef struct {
    double k;   /* wave number                                            */
    int N;      /* intervals per side, h = 1/N, 4 <= N <= 65536            */
    int diag;   /* 0: cells split along SW-NE, 1: along NW-SE              */
    int bc;     /* 0: u = 0 on the boundary (Eq. 1); 1: impedance, above  */
} hdd_assemble_params;

hdd_status hdd_assemble(hdd_ctx *ctx, const hdd_assemble_params *prm);

/* Rows of the impedance operator (bc = 1) by node class, as every kernel applies them; host
 * only (no context, no device).  Class c = cx + 3·cy with cx = 0 on x = 0, 2 on x = N, 1 in
 * between (cy the same in y), so class 4 is the interior.  Slot q of a row couples the node to
 * the neighbour at offset 0 (0,0), 1 (+1,0), 2 (-1,0), 3 (0,+1), 4 (0,-1), 5 and 6 the corners
 * joined by the cell diagonals: (+1,+1), (-1,-1) for diag = 0, (+1,-1), (-1,+1) for diag = 1.
 * coef_c128: 63 complex128 (interleaved re, im) entries of A = K - k²M - i k B at [c·7 + q];
 * mass: 63 doubles of M, or NULL.  HDD_ERR_INVALID_ARG for N < 4, diag not 0/1, k < 0 or a
 * NULL coef_c128. */
hdd_status hdd_stencil_rows(int N, double k, int diag, double *coef_c128, double *mass);

/* Load vector on the device (§3): point sources F += amp·e_c at the unknown node nearest to
 * (x, y) (clamped into the interior for bc = 0), and Gaussian bumps F += M g with g the nodal
 * values of amp·exp(-|x - c|²/(2σ²)) at the unknowns (the interpolant in V^h) and M the P1
 * mass matrix.  points: npoints triples (x, y, amp); bumps: nbumps quadruples (cx, cy, σ, amp),
 * both host arrays.  f_dev: one complex128 vector of (N-1)² (bc = 0) or (N+1)² (bc = 1)
 * entries, overwritten. */
hdd_status hdd_build_rhs(hdd_ctx *ctx, int npoints, const double *points, int nbumps,
                         const double *bumps, void *f_dev, void *stream);

/* y = A x for nrhs global complex128 vectors (x_dev, y_dev distinct). */
hdd_status hdd_apply_A(hdd_ctx *ctx, const void *x_dev, void *y_dev, int nrhs, void *stream);

/* ---------------------------------------------------------------------------------------- */
/* Decomposition (Eq. 3, §3).  Sx x Sy Cartesian subdomains with interfaces                  */
/* 0 = a_0 < a_1 < ... < a_S = N (node indices; NULL = uniform round(pN/S)).  Subdomain      */
/* (p, q) owns the interior nodes a_p <= i < a_{p+1}, a_q <= j < a_{q+1} (D_j = ownership    */
/* indicator) and its local box, after appending `overlap` element layers, is               */
/* max(1, a_p - δ + 1) <= i <= min(N-1, a_{p+1} + δ - 1) (same in y).  Subdomain index        */
/* s = p + q·Sx.  A_j = R_j A R_jᵀ is the stencil on the box with zero Dirichlet values      */
/* outside it.  With bc = 1 the unknowns run over 0..N: the box is clipped to [0, N] and the */
/* last subdomain in each direction also owns node N.                                        */
/* ---------------------------------------------------------------------------------------- */
typedef struct {
    int Sx, Sy;       /* 1 <= Sx, Sy <= 4096                                 */
    int overlap;      /* δ >= 1 element layers                                */
    const int *ifx;   /* host array of Sx+1 interfaces in x, or NULL          */
    const int *ify;   /* host array of Sy+1 interfaces in y, or NULL          */
} hdd_dd_params;

hdd_status hdd_setup_dd(hdd_ctx *ctx, const hdd_dd_params *prm);

/* Number of subdomains and, for subdomain s, the 12 ints
 * {ix0, ix1, iy0, iy1, ox0, ox1, oy0, oy1, nx, ny, mx, my}: local box, owned range,
 * box size, coarse size (mx = floor(nx/2)). */
hdd_status hdd_get_subdomain(const hdd_ctx *ctx, int s, int *info12);
int hdd_num_subdomains(const hdd_ctx *ctx);

/* Packed local layout used by the local test hooks: subdomain s occupies
 * [fine_off[s], fine_off[s] + nx·ny) of a packed fine vector (box x fastest) and
 * [coarse_off[s], coarse_off[s] + mx·my) of a packed coarse vector.  Host arrays of nsub+1. */
hdd_status hdd_get_offsets(const hdd_ctx *ctx, long long *fine_off, long long *coarse_off);

/* Batch nrhs independent right-hand sides (1..4096; default 1 after hdd_setup_dd): every
 * subsequent hdd_solve / hdd_ras_apply takes nrhs global vectors (RHS-major) and runs the local
 * solves of every (subdomain, RHS) pair in the same launches; the outer FGMRES iterations of the
 * right-hand sides run in lockstep, each with its own Krylov basis and stopping test.  The
 * packed local layout (hdd_get_offsets) then repeats per RHS.  Factors are kept. */
hdd_status hdd_setup_batch(hdd_ctx *ctx, int nrhs);
int hdd_num_rhs(const hdd_ctx *ctx);

/* ---------------------------------------------------------------------------------------- */
/* Deflation set-up (Eq. 4, Eq. 5).  For every distinct box shape: E = Zᵀ A Z (5x5 coarse   */
/* stencil, half-bandwidth 2·mx+2) is formed and LU-factorised with partial pivoting in FP64 */
/* on the device; subdomains with equal shape share one factor.  With bc = 1 a shape also    */
/* records which box sides lie on the boundary of the square, and the complex E is factored  */
/* as its real equivalent (order 2·mx·my, unknowns Re and Im interleaved).                   */
/* ---------------------------------------------------------------------------------------- */
hdd_status hdd_setup_deflation(hdd_ctx *ctx, void *stream);

/* ---------------------------------------------------------------------------------------- */
/* Two-level RAS (the coarse space the conclusions, §4, name as the next step).  The coarse   */
/* space is P1 on the mesh of N/c intervals with the same diagonal direction (H = c h): P     */
/* interpolates a coarse nodal vector to the fine interior nodes (the coarse hat functions    */
/* are φ = max(0, 1 - max(|ξ|, |η|, |ξ - η|)) for diag 0, |ξ + η| in place of |ξ - η| for diag */
/* 1, in units of H), Pᵀ restricts.  The coarse operator is rediscretised on that mesh with a */
/* lumped mass, A_H = K_H - k² H² I (every coarse hat integrates to H²), whose eigenvectors   */
/* are the discrete sine modes: A_H⁻¹ = S D⁻¹ S with S the orthonormal DST-I of order m =     */
/* N/c - 1 along each axis and D_pq = 4 sin²(pπ/2Nc) + 4 sin²(qπ/2Nc) - k²H².  The two-level   */
/* preconditioner is the hybrid z = Q v + M_RAS⁻¹(v - A Q v), Q = P A_H⁻¹ Pᵀ, applied by       */
/* hdd_solve and hdd_ras_apply when hdd_solve_params.two_level is 1.  Coarse vectors hold     */
/* m² complex entries, x fastest (node (I, J), 1 <= I, J <= m, at (I-1) + (J-1) m).           */
/* ---------------------------------------------------------------------------------------- */

/* Build P's tables and S, D⁻¹ (FP64 on the host, an FP32 copy beside them) for coarsening   */
/* factor c.  HDD_ERR_INVALID_ARG unless c >= 2 divides N with N/c >= 2, or for bc = 1;       */
/* HDD_ERR_SINGULAR_COARSE if some |D_pq| <= 1e-13 max |D| (k H on a coarse resonance).       */
/* Needs hdd_assemble; kept across hdd_setup_dd and hdd_setup_batch; synchronises the stream. */
hdd_status hdd_setup_coarse_grid(hdd_ctx *ctx, int c, void *stream);

/* Test hook: apply the stages set in `stages` to nrhs complex128 vectors, in this order:     */
/*   HDD_CG_RESTRICT  v (fine, nglob) → Pᵀ v (coarse, m²)                                       */
/*   HDD_CG_SOLVE     y (coarse) → A_H⁻¹ y (coarse; four DST passes and the diagonal scaling,  */
/*                    in FP32 for prec 64, FP64 for prec 128)                                  */
/*   HDD_CG_PROLONG   u (coarse) → P u (fine)                                                  */
/* in_dev and out_dev hold nrhs consecutive vectors of the stage's input and output lengths   */
/* (distinct device buffers, 16-byte aligned).  All three: out = Q in.                        */
#define HDD_CG_RESTRICT 1
#define HDD_CG_SOLVE 2
#define HDD_CG_PROLONG 4
hdd_status hdd_coarse_grid_op(hdd_ctx *ctx, int stages, int prec, const void *in_dev, void *out_dev,
                              void *stream);
/* m² of the coarse grid set up, 0 if none */
long long hdd_coarse_grid_size(const hdd_ctx *ctx);

/* Banded LU (FP64, partial pivoting) of every distinct A_j for the direct local solve
 * (inner_tol <= 0, the benchmark of §3.1); for bc = 1 of its real equivalent, as for E. */
hdd_status hdd_setup_exact(hdd_ctx *ctx, void *stream);

/* ---------------------------------------------------------------------------------------- */
/* Solve (§3).                                                                               */
/* ---------------------------------------------------------------------------------------- */
typedef struct {
    double outer_tol;    /* stop when ||f - A x|| <= outer_tol ||f|| (true residual)        */
    int outer_restart;   /* FGMRES restart length (>= outer_maxit means unrestarted)         */
    int outer_maxit;     /* total outer iterations                                          */
    double inner_tol;    /* relative deflated residual ||P(f̃ - A ũ)|| <= tol ||P f̃||;        */
                         /* <= 0 selects the direct (banded LU) local solve                 */
    int inner_restart;   /* GMRES restart length, 1..64                                      */
    int inner_maxit;     /* total inner iterations per local solve                          */
    int inner_prec;      /* 64: complex64 inner solves with FP32 accumulation;              */
                         /* 128: complex128 inner solves.  Coarse E and outer: FP64 always  */
    int warm_start;      /* 1: start every local solve from the learned guess (hdd_cnn_*);  */
                         /* 0: from zero.  The tolerance stays relative to ||P f̃||          */
    int outer_reorth32;  /* 1: the second CGS pass of the outer Arnoldi applies its         */
                         /* correction V h2 in FP32 from an FP32 copy of the basis whenever */
                         /* sum |h2| <= 2^-34 ||w'|| (error below the FP64 rounding of w'), */
                         /* FP64 otherwise; 0: FP64 always.  Dots, norms, H: FP64 always    */
    int two_level;       /* 1: hybrid two-level RAS with the grid coarse space of            */
                         /* hdd_setup_coarse_grid, z = Q v + M_RAS⁻¹(v - A Q v); 0: one-level */
                         /* RAS as in the paper (§3).  Ignored by hdd_autotune              */
} hdd_solve_params;

typedef struct {
    int outer_its;               /* outer FGMRES iterations (preconditioner applications)     */
    int status;                  /* hdd_status of the solve                                   */
    double rel_res_true;         /* ||f - A x|| / ||f|| recomputed at exit                    */
    long long inner_its_total;   /* Arnoldi steps summed over every local solve              */
    double inner_its_avg;        /* inner_its_total / (outer_its x #subdomains), as in §3    */
    int inner_its_max;           /* largest step count of one local solve                     */
    long long inner_maxit_hits;  /* local solves stopped by inner_maxit                       */
    double t_solve_ms;           /* wall time of the solve (host clock, stream synchronised) */
    int n_history;               /* entries in res_history                                    */
    const double *res_history;   /* |g_{j+1}|/||f|| per outer iteration; library-owned, valid */
                                 /* until the next hdd_solve or hdd_destroy                   */
    long long outer_reorth_fp64; /* outer iterations x RHS whose second CGS pass ran in FP64  */
                                 /* although outer_reorth32 was set (guard not met)           */
} hdd_solve_stats;

/* Solve A x = f for the batched right-hand sides (f_dev → x_dev: nrhs complex128 vectors,
 * distinct buffers).  stats may be NULL; outer_its counts lockstep iterations (the largest over
 * the right-hand sides), rel_res_true is the largest true relative residual, inner_its_avg the
 * average over all local solves, res_history that of the first RHS.  Returns
 * HDD_ERR_NO_CONVERGENCE (x holds the last iterates) when outer_maxit is reached. */
hdd_status hdd_solve(hdd_ctx *ctx, const void *f_dev, void *x_dev, const hdd_solve_params *prm,
                     hdd_solve_stats *stats, void *stream);

/* One application of the RAS preconditioner z = Σ_j R_jᵀ D_j ũ_j with ũ_j the inexact (or,
 * for inner_tol <= 0, direct) solution of A_j ũ_j = R_j v (Eq. 3): the inner-solve hot path on
 * its own.  v_dev, z_dev: nrhs global complex128 vectors.  inner_its (may be NULL): host array
 * of nsub x nrhs receiving each local solve's Arnoldi step count (task r·nsub + s).  With
 * prm->two_level = 1 it applies the hybrid two-level preconditioner z = Q v + M_RAS⁻¹(v - A Q v)
 * (needs hdd_setup_coarse_grid; inner_its then counts the local solves of M_RAS⁻¹). */
hdd_status hdd_ras_apply(hdd_ctx *ctx, const void *v_dev, void *z_dev,
                         const hdd_solve_params *prm, int *inner_its, void *stream);

/* Tile-shape autotuner (no counterpart in the paper).  The batched local kernels work on tiles
 * of a task's box: fine tiles of `fine_rows` box rows (fine_rows x box width <= 2048 nodes) and
 * coarse tiles of `coarse_rows` coarse rows; defaults 8 and 4.  This times one RAS application
 * (hdd_ras_apply with prm, on a fixed dense pseudo-random vector, best of two after a warm-up)
 * for every admissible pair of fine_rows in {4, 6, 8, 12, 16, 24} and coarse_rows in {2, 4, 8},
 * keeps the fastest pair for every later call on this context (until hdd_setup_dd /
 * hdd_setup_batch rebuild the tiles with it), and returns it with its time (outputs may be
 * NULL).  Tile shapes change the order of the per-tile partial sums, so results change at
 * rounding level.  Needs hdd_setup_deflation (or hdd_setup_exact for inner_tol <= 0);
 * allocates two global vectors for the duration of the call; synchronises the stream. */
hdd_status hdd_autotune(hdd_ctx *ctx, const hdd_solve_params *prm, void *stream, int *fine_rows,
                        int *coarse_rows, double *best_ms);

/* ---------------------------------------------------------------------------------------- */
/* Local test hooks on packed local vectors (layout of hdd_get_offsets), complex128.         */
/*   op 0: out = A_j in        (fine → fine, every subdomain)                                */
/*   op 1: out = Z_j in        (coarse → fine)                                               */
/*   op 2: out = Z_jᵀ in       (fine → coarse)                                               */
/*   op 3: out = E_j⁻¹ in      (coarse → coarse, FP64 factors)                               */
/*   op 4: out = P_j A_j in    (fine → fine)                                                 */
/*   op 5: out = R_j in        (global → fine; `in` is a global vector)                      */
/*   op 6: out = A_j⁻¹ in      (fine → fine, direct solve; needs hdd_setup_exact)            */
/* prec: 64 runs the fine arithmetic of ops 0, 1, 2, 4 in complex64 (inputs rounded to FP32, */
/* outputs widened back) and the banded solves of ops 3 and 6 in double-FP32 arithmetic (the  */
/* form the complex64 inner iteration uses, HDD_OPT_COARSE_DF); 128: complex128 / FP64. */
hdd_status hdd_local_op(hdd_ctx *ctx, int op, int prec, const void *in_dev, void *out_dev,
                        void *stream);

/* ---------------------------------------------------------------------------------------- */
/* Learned warm start (no counterpart in the paper).  A 4-layer 3x3 convolutional network with  */
/* 32 channels, BF16 weights and FP32 accumulation maps a restricted right-hand side f̃ of a     */
/* subdomain (channels Re f̃/σ, Im f̃/σ, k·h with σ = RMS(f̃), zero padding at the box edge) to an */
/* initial guess ũ₀ = σ·(a + i b) for its deflated GMRES.  Layers 4→32, 32→32, 32→32 (ReLU)    */
/* and 32→2; parameters are one FP32 array of hdd_cnn_num_params() values, per layer the       */
/* weights W[cout][ky·3+kx][cin] then the biases (the first layer's fourth input channel is    */
/* zero).  Training minimises the mean over subdomains of the relative deflated residual the   */
/* local GMRES starts from, ||P_j(f̂ - A_j(a + i b))||² / ||P_j f̂||² with f̂ = f̃/σ (Eq. 4), with */
/* Adam (β = 0.9, 0.999, ε = 1e-8) on FP32 master weights.  Images are the packed local       */
/* vectors of hdd_get_offsets (complex128 here); the solver applies the network in its own   */
/* precision.  Because FGMRES is flexible, any guess keeps the outer tolerance exact.         */
/* ---------------------------------------------------------------------------------------- */
int hdd_cnn_num_params(void);
/* Load parameters (host FP32 array), reset Adam's moments.  HDD_ERR_INVALID_ARG for a problem
 * assembled with bc = 1: the network serves the Dirichlet problem only. */
hdd_status hdd_cnn_set_params(hdd_ctx *ctx, const float *params);
/* Read the FP32 master parameters. */
hdd_status hdd_cnn_get_params(hdd_ctx *ctx, float *params);
/* Parameter file I/O (the format warmstart.save writes): "HDDCNN01", the parameter count and
 * the CRC-32 (IEEE 802.3 / zlib) of the payload as little-endian u32, then the FP32 parameters
 * little-endian.  load checks magic, count and CRC (HDD_ERR_INVALID_ARG naming the defect) and
 * then acts as hdd_cnn_set_params; save writes the current master parameters (needs
 * hdd_cnn_set_params or a load first). */
hdd_status hdd_warmstart_load(hdd_ctx *ctx, const char *path);
hdd_status hdd_warmstart_save(hdd_ctx *ctx, const char *path);
/* x0 = guess for every packed right-hand side f (complex128 packed local vectors). */
hdd_status hdd_cnn_forward(hdd_ctx *ctx, const void *f_dev, void *x0_dev, void *stream);
/* Inference as the solver's warm start runs it: layer 1 on the CUDA cores, layers 2-4 as      */
/* implicit GEMMs on the tensor cores (tcgen05, BF16 operands, FP32 accumulation in TMEM), with */
/* the activations between layers rounded to BF16.  Same arguments as hdd_cnn_forward, which  */
/* keeps FP32 activations (the training forward).  HDD_ERR_TIMEOUT if a bounded device wait    */
/* gave up (synchronises the stream to read that flag).  If the wait's own drain of the copies  */
/* and MMAs in flight also gave up, that work may outlive the CTA that issued it, so the error  */
/* is fatal: the context then refuses every later call with HDD_ERR_TIMEOUT, and the caller    */
/* should destroy it and discard its CUDA context. */
hdd_status hdd_cnn_infer(hdd_ctx *ctx, const void *f_dev, void *x0_dev, void *stream);
/* Training loss of the batch f (every packed subdomain image) and, if grad != NULL, its
 * gradient w.r.t. every parameter (host FP32 array); synchronises the device.  Needs
 * hdd_setup_deflation (the loss applies P_j). */
hdd_status hdd_cnn_loss_grad(hdd_ctx *ctx, const void *f_dev, double *loss, float *grad);
/* One Adam step with learning rate lr on the batch f; *loss receives the loss before the step. */
hdd_status hdd_cnn_train_step(hdd_ctx *ctx, const void *f_dev, float lr, double *loss, void *stream);
/* Copy outer Krylov vector j of the last solve (nrhs global vectors) to v_dev: the restricted
 * Arnoldi vectors are the right-hand sides the local solves see (training inputs). */
hdd_status hdd_get_outer_vector(hdd_ctx *ctx, int j, void *v_dev, void *stream);

/* ---------------------------------------------------------------------------------------- */
/* Profiling.  With profiling on, every kernel launch is bracketed by a pair of CUDA events on */
/* the launching stream; durations are summed per kernel family together with the family's   */
/* algorithmic bytes (data the step must read and write once) and floating-point operations. */
/* ---------------------------------------------------------------------------------------- */
typedef struct {
    char name[40];       /* family, e.g. "coarse_solve_fp64"                          */
    long long launches;
    double ms;           /* sum of per-launch event durations                         */
    double bytes;        /* algorithmic bytes, summed over launches                   */
    double flops;        /* algorithmic floating-point operations, summed            */
    int bound;           /* 0: memory bandwidth, 1: FP64 arithmetic, 2: FP32 arithmetic  */
} hdd_kernel_stat;

/* Synchronise the device, clear the counters and switch event timing on (1) or off (0). */
hdd_status hdd_profile(hdd_ctx *ctx, int enable);
/* Number of kernel families (entries readable with hdd_profile_get). */
int hdd_profile_count(const hdd_ctx *ctx);
/* Synchronise the device and read family i. */
hdd_status hdd_profile_get(hdd_ctx *ctx, int i, hdd_kernel_stat *out);
/* Kernel launches made by this context since creation (counted whether or not profiling is on). */
long long hdd_launch_count(const hdd_ctx *ctx);

/* Implementation choices of one context (no counterpart in the paper; every choice computes   */
/* the same method).  HDD_OPT_COARSE_LOOKAHEAD (1): the FP64 block solves of E_j (Eq. 4) and    */
/* A_j use the look-ahead kernel (value 1, the default) or the plain blocked kernel (0); both   */
/* apply the same precomputed block operators, summed in a different fixed order.              */
/* HDD_OPT_FUSED_INNER (2): each inner Arnoldi step runs as one cluster-resident kernel per     */
/* step between the coarse solves (1, the default, where every box fits its plan) or as the    */
/* separate stencil / CGS / Givens kernels (0).  HDD_OPT_OUTER_DOTS_DF (3): with the guarded    */
/* FP32 second outer CGS pass (outer_reorth32 = 1), the dot products of both outer CGS passes  */
/* run in double-FP32 arithmetic (error-free products and sums, as accurate as FP64 sums) from  */
/* hi/lo FP32 copies of the basis (1, the default; another 8 bytes per basis entry) or in FP64  */
/* (0).  HDD_OPT_OUTER_UPDATE_DF (4): with HDD_OPT_OUTER_DOTS_DF, the first-pass update         */
/* w' = w - V h1 also runs in double-FP32 arithmetic from those copies, widened to FP64 every   */
/* 32 basis vectors (1, the default: 16 bytes per basis entry on the FP32 pipe; worst-case      */
/* error 3.6e-12 Σ|v h| against 1.4e-13 for the FP64 sum at 1270 vectors, removed from the      */
/* basis directions by the second pass) or in FP64 (0).  Hessenberg entries, norms, w and the   */
/* solution stay FP64.  HDD_OPT_OUTER_DCGS2 (5): with both double-FP32 options, the outer      */
/* Arnoldi uses delayed CGS2 (Świrydowicz et al., low-synchronisation Gram-Schmidt): the second */
/* pass of basis vector j runs fused with the first pass of step j+1, so a step makes two passes */
/* over the basis instead of four (1, the default), or the plain CGS2 above (0); both compute   */
/* the same FGMRES iteration up to rounding.  outer_reorth32 = 0 runs every outer step in FP64 */
/* (plain CGS2) whatever these say.  HDD_OPT_COARSE_DF (6): the coarse solves E_j⁻¹ of the    */
/* complex64 inner iteration run in double-FP32 arithmetic on the FP32 pipe (1, the default:    */
/* operators as (hi, lo) FP32 pairs, 2^-48 relative, forward error about κ(E_j)·2^-48) or in   */
/* FP64 (0).  Complex128 inner solves and the direct local solve always use FP64.              */
/* HDD_OPT_COARSE_SPIKE (7): those double-FP32 solves split each banded solve over 2 or 4 SMs   */
/* (the SPIKE algorithm on the blocked operators, spike matrices formed at hdd_setup_deflation  */
/* in FP64 by the host) when the active chains leave SMs free (1, the default) or not (0).     */
/* HDD_OPT_OUTER_DOTS_BIASED (8): with delayed CGS2, the first-pass dot products V^H w of its  */
/* fused pass keep every high accumulator offset by a power of two above four times the sum    */
/* it will take (bounded from the largest |entry| of each basis vector and of the chunk of w), */
/* so one fma and one exact subtraction replace the two-sum: a quarter fewer FP32 instructions */
/* in the pass, those dots within a few 1e-12 of Σ|v w| instead of about 1e-15 (1, the        */
/* default: the delayed second pass, which keeps the two-sum, measures and removes what the   */
/* first pass left) or the two-sum for both (0).                                              */
/* HDD_ERR_INVALID_ARG for an unknown key or a value other than 0 or 1.  Takes effect from the  */
/* next call that solves.                                                                       */
#define HDD_OPT_COARSE_LOOKAHEAD 1
#define HDD_OPT_FUSED_INNER 2
#define HDD_OPT_OUTER_DOTS_DF 3
#define HDD_OPT_OUTER_UPDATE_DF 4
#define HDD_OPT_OUTER_DCGS2 5
#define HDD_OPT_COARSE_DF 6
#define HDD_OPT_COARSE_SPIKE 7
#define HDD_OPT_OUTER_DOTS_BIASED 8
hdd_status hdd_set_option(hdd_ctx *ctx, int key, int value);

/* ---------------------------------------------------------------------------------------- */
/* Deflated operator without device allocation.                                             */
/*                                                                                          */
/* The paper has no counterpart: this entry point exists for callers that cannot call        */
/* cudaMalloc, e.g. code running inside a captured CUDA graph, under an allocator that must  */
/* not be re-entered, or in an embedding that owns all device memory up front.               */
/*                                                                                          */
/* out = P_j A_j in for every subdomain j (the same operator and packed layout as            */
/* hdd_local_op op 4, complex128).  in_dev, out_dev: caller-owned packed local vectors       */
/* (hdd_get_offsets), distinct, 16-byte aligned.  The two complex128 coarse work vectors live */
/* in a fixed array inside the library (16 MiB, present on every GPU that loads the library  */
/* until the process exits): the packed coarse length Σ m_x·m_y must not exceed 524288, else */
/* HDD_ERR_INVALID_ARG.  The call allocates nothing; the first call from a CUDA context     */
/* looks up that array's device address in it (make the first call before any stream        */
/* capture; after cudaDeviceReset the first call from the new context looks it up again).    */
/* Each context has its own copy of the array, and every call made in one context shares     */
/* that copy, which keeps the last call's contents: calls that may overlap on the GPU in one  */
/* context (other streams, other host threads) race; serialise them.  Work is enqueued on     */
/* `stream`; no synchronisation.                                                            */
/* ---------------------------------------------------------------------------------------- */
hdd_status hdd_apply_PA_noalloc(hdd_ctx *ctx, const void *in_dev, void *out_dev, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* HDD_H */
