// hdd_common.cuh — shared definitions of the GB300 solver library (device + host launchers).
//
// Layout in HBM
//  * global vectors: complex128, (N-1)² interior nodes, x fastest;
//  * packed local vectors: every (subdomain, right-hand side) "task" owns a contiguous slab of
//    nx·ny fine entries (box, x fastest) at Task::foff and mx·my coarse entries at Task::coff;
//  * Krylov bases: basis vector k of every task at base + k·ld (ld = total packed length), so
//    one kernel sweeps the same vector of all tasks with coalesced accesses;
//  * FP64 banded factors (one per distinct box shape): L stored by column (kl multipliers per
//    column), U stored by column above the diagonal with its true extent, reciprocal pivots.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace hdd {

// ------------------------------------------------------------------------------------------
// complex helpers (storage as float2 / double2)
// ------------------------------------------------------------------------------------------
// ------------------------------------------------------------------------------------------
// double-FP32 ("df") arithmetic on the FP32 pipe: a value is an unevaluated pair (hi, lo) of
// FP32 numbers.  df_acc adds the product (xh + xl)(yh + yl) to the accumulator (sh, sl): the
// product of the high parts exactly (p + e, e = fma(xh, yh, -p)), the two cross terms, and a
// Knuth two-sum of p into sh (the compensated dot product of Ogita, Rump & Oishi, SIAM J. Sci.
// Comput. 2005, on split inputs).  The _rn intrinsics keep the compiler from contracting the
// error-free steps into fused multiply-adds.
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ void df_acc(float &sh, float &sl, float xh, float xl, float yh, float yl) {
    const float p = __fmul_rn(xh, yh);
    const float e = fmaf(xh, yh, -p);                 // exact: xh·yh = p + e
    const float c = fmaf(xh, yl, fmaf(xl, yh, e));
    const float t = __fadd_rn(sh, p);                 // two-sum: sh + p = t + err exactly
    const float bb = __fsub_rn(t, sh);
    const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, bb)), __fsub_rn(p, bb));
    sh = t;
    sl = __fadd_rn(sl, __fadd_rn(err, c));
}

// The same sum with a biased high accumulator (6 instructions instead of 12).  sh starts at a
// power of two M >= 4 Σ|xh·yh| over every product the accumulator will take, so it stays within
// [3M/4, 5M/4]: t = fl(sh + xh·yh) (one fma) and q = t - sh is exact (Sterbenz), and the part of
// the product that t did not absorb, xh·yh - q, is formed by a second fma and added to sl with
// the cross terms.  That remainder is below ulp(M) and is itself rounded once (error <= 2^-24
// ulp(M)), so a sum of T products carries at most about T·2^-47·M more error than df_acc, i.e.
// a few 1e-12 of T·max|xh|·max|yh| when M is the bound's power of two.  The caller subtracts M
// (exact) when it is done.
__device__ __forceinline__ void df_acc_biased(float &sh, float &sl, float xh, float xl, float yh, float yl) {
    const float t = fmaf(xh, yh, sh);
    const float q = __fsub_rn(t, sh);
    sl = __fadd_rn(sl, fmaf(xh, yh, -q));
    sl = fmaf(xh, yl, sl);
    sl = fmaf(xl, yh, sl);
    sh = t;
}
// smallest power of two >= max(y, 2^-100) for finite y >= 0 (the bias M of df_acc_biased)
__device__ __forceinline__ float pow2_ceil(float y) {
    y = fmaxf(y, 0x1p-100f);
    return __uint_as_float((__float_as_uint(y) + 0x007FFFFFu) & 0xFF800000u);
}

// (sh, sl) += (bh, bl): two-sum of the high parts, the low parts added
__device__ __forceinline__ void df_add(float &sh, float &sl, float bh, float bl) {
    const float t = __fadd_rn(sh, bh);
    const float bb = __fsub_rn(t, sh);
    const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, bb)), __fsub_rn(bh, bb));
    sh = t;
    sl = __fadd_rn(sl, __fadd_rn(err, bl));
}

// the FP64 value x as a pair (hi, lo) with hi + lo = x to about 2^-48 relative
__device__ __forceinline__ float2 df_split(double x) {
    const float h = (float)x;
    return make_float2(h, (float)(x - (double)h));
}

template <typename R> struct C2;
template <> struct C2<float> { using T = float2; };
template <> struct C2<double> { using T = double2; };
template <typename R> using c2 = typename C2<R>::T;

template <typename R> __host__ __device__ __forceinline__ c2<R> mk(R re, R im) {
    c2<R> z; z.x = re; z.y = im; return z;
}
template <typename R> __device__ __forceinline__ c2<R> cadd(c2<R> a, c2<R> b) { return mk<R>(a.x + b.x, a.y + b.y); }
template <typename R> __device__ __forceinline__ c2<R> csub(c2<R> a, c2<R> b) { return mk<R>(a.x - b.x, a.y - b.y); }
template <typename R> __device__ __forceinline__ c2<R> cscale(R s, c2<R> a) { return mk<R>(s * a.x, s * a.y); }
template <typename R> __device__ __forceinline__ c2<R> cmul(c2<R> a, c2<R> b) {
    return mk<R>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// acc += conj(a) * b
template <typename R> __device__ __forceinline__ void cdotc_acc(c2<R> &acc, c2<R> a, c2<R> b) {
    acc.x = fma(a.x, b.x, acc.x); acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y); acc.y = fma(-a.y, b.x, acc.y);
}
// acc -= h * v
template <typename R> __device__ __forceinline__ void caxpy_neg(c2<R> &acc, c2<R> h, c2<R> v) {
    acc.x = fma(-h.x, v.x, acc.x); acc.x = fma(h.y, v.y, acc.x);
    acc.y = fma(-h.x, v.y, acc.y); acc.y = fma(-h.y, v.x, acc.y);
}
// acc += h * v
template <typename R> __device__ __forceinline__ void caxpy(c2<R> &acc, c2<R> h, c2<R> v) {
    acc.x = fma(h.x, v.x, acc.x); acc.x = fma(-h.y, v.y, acc.x);
    acc.y = fma(h.x, v.y, acc.y); acc.y = fma(h.y, v.x, acc.y);
}

template <typename R> __device__ __forceinline__ R shfl_xor(R v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }

// Division by a box dimension d (1 <= d <= 256) of an index 0 <= e < 2^24, as the high word of
// e·M with M = ceil(2^32/d): with M·d = 2^32 + r (0 <= r < d) the excess over e/d is
// e·r/(2^32·d) < e/2^32 < 1/d, too small to reach the next integer (checked on the CPU for every
// d <= 256).  Replaces the integer division in the row/column splits of the tile loops.
struct BoxDiv {
    unsigned m;
    __device__ __forceinline__ explicit BoxDiv(int d)
        : m(d > 1 ? (unsigned)((0x100000000ull + (unsigned)d - 1) / (unsigned)d) : 0u) {}
    __device__ __forceinline__ int q(int e) const { return m ? (int)__umulhi((unsigned)e, m) : e; }
};

// ------------------------------------------------------------------------------------------
// problem description shared with the kernels
// ------------------------------------------------------------------------------------------
struct Stencil {           // P1 operator K - k²M on the uniform mesh (Eq. 2), 7-point form
    double c0;             // centre
    double c1;             // E, W, N, S
    double c2;             // the two corners joined by the cell diagonals
    int diag;              // 0: diagonal pair (+1,+1)/(-1,-1); 1: (+1,-1)/(-1,+1)
    // bc = 1: impedance (first-order absorbing) condition du/dn - iku = 0 on all four sides.
    // Every mesh node 0..N is then an unknown and A = K - k²M - ik B (B: boundary mass); the
    // rows of nodes on the boundary differ from c0..c2 and are read, per node class
    // (node_class), from bcoef[cls·7 + slot] (complex A) and bmass[cls·7 + slot] (real M), with
    // the slots of stencil_slot.  Interior rows keep c0..c2.
    int bc = 0;
    int N = 0;                       // intervals per side
    const double2 *bcoef = nullptr;  // device table, 9 classes x 7 slots
    const double *bmass = nullptr;   // device table, 9 classes x 7 slots
};

// Class of mesh node (gx, gy): cx + 3·cy with cx = 0 on x = 0, 2 on x = N, 1 otherwise (cy the
// same in y); 4 is the interior class.
__host__ __device__ __forceinline__ int node_class(int N, int gx, int gy) {
    return (gx == 0 ? 0 : (gx == N ? 2 : 1)) + 3 * (gy == 0 ? 0 : (gy == N ? 2 : 1));
}
// Stencil slots: 0 centre, 1 E (+1,0), 2 W (-1,0), 3 N (0,+1), 4 S (0,-1), 5 and 6 the corners
// joined by the cell diagonals: (+1,+1), (-1,-1) for diag 0; (+1,-1), (-1,+1) for diag 1.
__host__ __device__ __forceinline__ void stencil_offset(int diag, int q, int &dx, int &dy) {
    const int ox[7] = {0, 1, -1, 0, 0, 1, -1};
    const int oy0[7] = {0, 0, 0, 1, -1, 1, -1}, oy1[7] = {0, 0, 0, 1, -1, -1, 1};
    dx = ox[q];
    dy = diag == 0 ? oy0[q] : oy1[q];
}
// slot of offset (dx, dy), -1 if it is not a stencil neighbour
__host__ __device__ __forceinline__ int stencil_slot(int diag, int dx, int dy) {
    for (int q = 0; q < 7; q++) {
        int ax, ay;
        stencil_offset(diag, q, ax, ay);
        if (ax == dx && ay == dy) return q;
    }
    return -1;
}

struct Task {              // one local solve: subdomain `sub` for right-hand side `rhs`
    int nx, ny, mx, my;    // box and coarse sizes
    int ix0, iy0;          // mesh node (i, j) of the box's local (0,0): >= 1 (Dirichlet), >= 0 (impedance)
    int ox0, ox1, oy0, oy1;// owned nodes (global, inclusive)
    int shape;             // index of the shared factor of E (and of A_j)
    int sub, rhs;
    int tile0, ntiles;     // fine tiles of this task
    long long foff, coff;  // packed fine / coarse offsets
    long long poff;        // frame offset of the padded planar CNN activations, (ny+2)(nx+2) per task
};

struct Tile {              // a block of fine rows (fine tiles) or coarse rows (coarse tiles)
    int task, r0, nr;
};

struct BlockFactor {        // FP64 banded LU with partial pivoting in blocked solve form
    int m;                 // order
    int nblk;              // blocks of BNB rows
    int wl, wu;            // widest left (L) / right (U) panel over the blocks, even
    long long perm_off;    // int perm[m]: (P b)[i] = b[perm[i]]
    long long meta_off;    // int4 per block: {forward operator offset, its panel width w_l,
                           //                  backward operator offset, its panel width w_u}
                           // offsets in doubles from the start of the operator array
};
constexpr int BNB = 16;    // rows per block of the blocked banded solve
// Row stride of a block operator with panel width w (BNB + w columns), padded with zeros to
// ≡ 2 (mod 16) entries: the 8-byte reads of a warp's 16 rows x 2 lanes then fall in distinct
// shared-memory banks whatever the panel width (an unpadded width ≡ 0 mod 16 put every row on
// the same banks).
__host__ __device__ __forceinline__ int op_stride(int w) {
    const int K = BNB + w;
    return K + ((2 - K) & 15);
}

constexpr int MAX_RESTART = 64;       // inner GMRES restart bound (Hessenberg in registers/smem)
constexpr int FINE_ROWS = 8;          // default fine rows per fine tile (hdd_autotune may change it)
constexpr int COARSE_ROWS = 4;        // default coarse rows per coarse tile
constexpr int FINE_EPT = 8;           // fine elements per thread: a fine tile holds <= 256·8 nodes
constexpr int LOCAL_THREADS = 256;    // threads per tile CTA

// per-task inner GMRES state (precision R)
template <typename R> struct InnerState {
    c2<R> *H;        // [task][(restart+1) * restart], column i holds rows 0..i+1
    R *cs;           // [task][restart]
    c2<R> *sn;       // [task][restart]
    c2<R> *g;        // [task][restart+1]
    R *ref;          // ||P f̃||
    int *its;        // Arnoldi steps so far (whole solve)
    int *kcols;      // columns in the current cycle
    int *conv;       // 1 once converged / finished
    int *restart;    // 1 if the task needs another cycle
};

// ------------------------------------------------------------------------------------------
// host-side launchers (defined in the kernel translation units)
// ------------------------------------------------------------------------------------------
template <typename R> struct LocalArgs {
    const Task *tasks; const Tile *ftiles; const Tile *ctiles;
    int ntasks, nftiles, nctiles;
    Stencil st;
    long long ld;      // packed fine length (all tasks): stride between basis vectors
    long long ldc;     // packed coarse length
    int max_nx;        // largest box width (shared-memory sizing), <= 256
    int gw;            // global grid width: N-1 (Dirichlet) or N+1 (impedance)
    int glo;           // mesh index of the first global unknown in x and y: 1 or 0
    int frows, crows;  // largest fine / coarse tile height (shared-memory sizing)
};

// local (batched over tasks), R = float or double
template <typename R> void launch_restrict(const LocalArgs<R> &a, const double2 *glob, long long nglob,
                                           c2<R> *out, const int *flag, cudaStream_t s);
template <typename R> void launch_scatter(const LocalArgs<R> &a, const c2<R> *x, double2 *glob,
                                          long long nglob, const int *flag, cudaStream_t s);
template <typename R> void launch_local_A(const LocalArgs<R> &a, const c2<R> *in, c2<R> *out,
                                          const c2<R> *f, const int *flag, cudaStream_t s);
template <typename R> void launch_zt(const LocalArgs<R> &a, const c2<R> *in, double2 *y, int apply_A,
                                     const int *flag, cudaStream_t s);
// out = add + sign · Z s
template <typename R> void launch_z(const LocalArgs<R> &a, const double2 *sc, const c2<R> *add,
                                    c2<R> *out, const int *flag, cudaStream_t s, R sign = 1);
template <typename R> void launch_prolong_stencil(const LocalArgs<R> &a, int mode, const c2<R> *in,
                                                  const double2 *sc, c2<R> *out, const c2<R> *V,
                                                  int nv, c2<R> *part, const int *flag,
                                                  cudaStream_t s);
template <typename R> void launch_cgs_update(const LocalArgs<R> &a, int pass, c2<R> *w, const c2<R> *V,
                                             int nv, const c2<R> *part_in, c2<R> *part_out,
                                             const int *flag, cudaStream_t s);
template <typename R> void launch_givens_normalize(const LocalArgs<R> &a, const InnerState<R> &S,
                                                   int restart, int i, c2<R> *w, const c2<R> *p1,
                                                   const c2<R> *p2, const c2<R> *p3,
                                                   const int *act_in, int *act_out, int *counter,
                                                   R tol, int maxit, cudaStream_t s);
template <typename R> void launch_init_cycle(const LocalArgs<R> &a, const InnerState<R> &S, int restart,
                                             c2<R> *v0, const c2<R> *p3, const int *flag,
                                             int *act_out, int *counter, R tol, int maxit,
                                             int set_ref, cudaStream_t s);
template <typename R> void launch_update_u(const LocalArgs<R> &a, const InnerState<R> &S, int restart,
                                           c2<R> *u, const c2<R> *V, const int *flag, int *rs_out,
                                           int *counter, int maxit, cudaStream_t s);
template <typename R> cudaError_t set_local_smem_limits(size_t bytes);
template <typename R> void launch_set_ref(const LocalArgs<R> &a, const InnerState<R> &S, const c2<R> *p3,
                                          const int *flag, cudaStream_t s);
template <typename R> void launch_coarse_combine(const LocalArgs<R> &a, const InnerState<R> &S,
                                                 int restart, const double2 *sbuf, double2 *sc,
                                                 const int *flag, cudaStream_t s);
size_t local_max_dynamic_smem(int max_nx, int bytes_per_c, int frows, int crows);
// one inner Arnoldi step per launch, one cluster of C CTAs per task (kernels_local.cu)
constexpr int STEP_ROWS_MAX = LOCAL_THREADS * FINE_EPT;   // box nodes a CTA of the fused step holds
size_t step_smem_bytes(int max_nx, int max_ny, int C, int bytes_per_c);
template <typename R>
cudaError_t launch_arnoldi_step(const LocalArgs<R> &la, int C, int i, int restart, c2<R> *V, const double2 *sc,
                                double2 *y, const InnerState<R> &S, const int *act_in, int *act_out,
                                int *counter, R tol, int maxit, size_t smem, cudaStream_t s);
template <typename R> int arnoldi_step_max_cluster(size_t smem, int C);
void launch_cast(long long n, const void *in, int in_double, void *out, int out_double, cudaStream_t s);
constexpr int LOCAL_LDP = MAX_RESTART + 2;   // partial-sum slots per fine tile

// coarse / banded FP64
void launch_assemble_E(const Stencil &st, int nx, int ny, int kl, int ku, double *ab, cudaStream_t s);
void launch_assemble_Aloc(const Stencil &st, int nx, int ny, int kl, int ku, double *ab, cudaStream_t s);
// complex E (resp. A_j) of a box with origin (gx0, gy0) under the impedance condition, written as
// its real equivalent: unknowns (Re x_0, Im x_0, Re x_1, ...), i.e. the complex vector read as
// doubles; order 2m, half-bandwidths kl2 = ku2 = 2·kl + 1 of the complex band kl
void launch_assemble_E_re2(const Stencil &st, int nx, int ny, int gx0, int gy0, int kl2, int ku2, double *ab,
                           cudaStream_t s);
void launch_assemble_Aloc_re2(const Stencil &st, int nx, int ny, int gx0, int gy0, int kl2, int ku2, double *ab,
                              cudaStream_t s);
void launch_band_lu(int nmat, const int *m, const int *kl, const int *ku, double *const *ab,
                    int *const *piv, int *info, cudaStream_t s);
void launch_factor_prepare(int m, int kl, int ku, const double *ab, const int *piv, int KLW,
                           double *Lp, int *lext, int *uext, int *perm, int *err, cudaStream_t s);
void launch_block_operators(int m, int kl, int ku, const double *ab, int KLW, const double *Lp,
                            const int4 *meta, double *Mall, cudaStream_t s);
struct BlockSolveCfg {       // shared-memory plan of the blocked solve over a set of factors
    int maxK = 0;          // widest operator row stride: op_stride(panel width)
    int cwy = 0, cwx = 0;  // circular y / x windows, powers of two >= BNB + widest left / right panel
    int ring = 0;          // operator ring depth (4 or 2), chosen by set_block_solve_smem
    int la_ring = 0;       // ring of the look-ahead kernel (6, 4 or 3; 0 if it does not fit)
    int lookahead = 1;     // use the look-ahead kernel when la_ring > 0
    int spike_ok = 0;      // ring of the SPIKE kernels (6, 4 or 3; 0 if none fits)
    int spike_cap[2] = {0, 0};  // clusters of 2 / of 4 co-resident with that ring
};
// re2 = 0: real factors, Re and Im of the complex vector solved as two columns; re2 = 1: factors
// of real-equivalent systems (order 2m), the complex vector read as one real column
// Mdf (may be null): the operators as (hi, lo) FP32 pairs; given, the look-ahead kernel runs in
// double-FP32 arithmetic on the FP32 pipe (k_block_solve_la_df)
void launch_block_solve(const Task *tasks, int ntasks, const BlockFactor *shapes, const double *Mall,
                        const int *Pall, const int4 *Meta, const double2 *in, double2 *out,
                        int use_fine, const int *flag, const BlockSolveCfg &cfg, int re2, cudaStream_t s,
                        const float2 *Mdf = nullptr);
void launch_ops_to_df(long long n, const double *M, float2 *Mdf, cudaStream_t s);

// SPIKE partition of one factor's blocked solve (Polizzi & Sameh's SPIKE algorithm for banded
// systems, on the blocked operators): the block range [0, nblk) split into P parts solved at
// once by a cluster of P CTAs, each part with zero values outside it; the exact solution follows
// from the local ones through the spike matrices of the parts' couplings:
//   forward  y_p = g_p + Gf_p t_p,  t_p = y[r_p - wf, r_p)        (parts p >= 1),
//   backward x_p = l_p + Gb_p h_p,  h_p = x[r_{p+1}, r_{p+1} + wb)   (parts p <= P-2),
// with r_p = 16·B[p]; the boundary values t_p, h_p chain through the parts' boundary rows.
constexpr int SPIKE_PMAX = 4;          // most parts
constexpr int SPIKE_WMAX = 512;        // widest window the kernel stages (wf, wb)
constexpr int SPIKE_LEVELS = 2;        // P = 2 and P = 4
struct SpikeInfo {
    int P;                             // parts (0: this level is not available for the shape)
    int wf, wb;                        // forward / backward window widths (widest panels)
    int B[SPIKE_PMAX + 1];             // first block of each part; B[P] = nblk
    long long gf[SPIKE_PMAX];          // part p >= 1: offset (pairs) of Gf_p, 16·(B[p+1]-B[p]) x wf
    long long gb[SPIKE_PMAX];          // part p <= P-2: offset of Gb_p, 16·(B[p+1]-B[p]) x wb
};
// The double-FP32 look-ahead solve with a cluster of P = spikes[shape].P CTAs per chain
// (spikes: the table of the level used, one SpikeInfo per shape; G: the spike matrices as
// (hi, lo) pairs) over the chains of the ntasks tasks list[0 .. ntasks) (list null: tasks
// 0 .. ntasks).  Returns false (nothing launched) if the plan does not fit.
bool launch_block_solve_spike(int P, const Task *tasks, int ntasks, const BlockFactor *shapes,
                              const float2 *Mdf, const int *Pall, const int4 *Meta, const SpikeInfo *spikes,
                              const float2 *G, const double2 *in, double2 *out, int use_fine, const int *flag,
                              const int *list, const BlockSolveCfg &cfg, int re2, cudaStream_t s);
// list[0 .. count) = indices of the nonzero flags in order (count = number of nonzero flags)
void launch_compact_flags(int n, const int *flag, int *list, cudaStream_t s);
cudaError_t set_block_solve_smem(BlockSolveCfg &cfg);

// learned warm start (kernels_cnn.cu)
constexpr int CNN_NPARAM = 20258;          // 4 conv3x3 layers: 4->32, 32->32, 32->32, 32->2
constexpr int CNN_OFF[5] = {0, 1184, 10432, 19680, 20258};   // per layer: W (COUT x 9 x CIN), b
}  // namespace hdd
#include <cuda_bf16.h>
namespace hdd {
template <typename R> void launch_cnn_input(const Task *tasks, int ntasks, const c2<R> *f, float kh,
                                            float *sigma, float *X0, float2 *Fh, cudaStream_t s);
void launch_cnn_task_scale(const Task *tasks, int ntasks, const float2 *p3f, float *scale, cudaStream_t s);
void launch_cnn_task_loss(const Task *tasks, int ntasks, const float2 *p3r, const float2 *p3f, float *loss,
                          cudaStream_t s);
template <typename R> void launch_cnn_output(const Task *tasks, const Tile *tiles, int ntiles,
                                             const float *sigma, const float *Y4, c2<R> *x0,
                                             const int *flag, cudaStream_t s);
void launch_conv_fwd(int layer, const Task *tasks, const Tile *tiles, int ntiles, const __nv_bfloat16 *W,
                     const float *b, const float *X, float *Y, cudaStream_t s);
void launch_conv_bwd_data(int layer, const Task *tasks, const Tile *tiles, int ntiles,
                          const __nv_bfloat16 *W, const float *dY, const float *act_out, float *dX,
                          cudaStream_t s);
void launch_conv_bwd_w(int layer, const Task *tasks, const Tile *tiles, int ntiles, const float *dY,
                       const float *act_out, const float *X, float *part, cudaStream_t s);
void launch_sum_partials(const float *part, int ntiles, int nw, float scale, float *grad, cudaStream_t s);
void launch_cnn_resid(const Task *tasks, const Tile *tiles, int ntiles, const Stencil &st, const float *X0,
                      const float *Y4, float *Rr, float *lpart, cudaStream_t s);
void launch_cnn_out_grad(const Task *tasks, const Tile *tiles, int ntiles, const Stencil &st, const float *Rr,
                         const float *scale, float *dY4, cudaStream_t s);
void launch_adam(int n, float *p, const float *g, float *m, float *v, __nv_bfloat16 *pb, float lr, float b1,
                 float b2, float eps, int step, cudaStream_t s);
void launch_to_bf16(int n, const float *p, __nv_bfloat16 *pb, cudaStream_t s);

// global FP64 (outer FGMRES), batched over right-hand sides
struct OuterBatch {
    int nrhs;              // independent right-hand sides
    long long n;           // entries per global vector
    long long ld;          // stride between basis vectors of one RHS (= nrhs·n)
    int ldp;               // reduction slots per CTA and per RHS (>= R+1)
    int G;                 // CTAs per RHS of the chunked reductions
    int R;                 // Hessenberg columns (restart length)
    const int *active;     // per-RHS flag, or null for all
    long long n32 = 0;     // FP32 basis copy: entries per RHS (n rounded up to even)
    long long ld32 = 0;    // FP32 basis copy: stride between basis vectors (= nrhs·n32)
    const double *D = nullptr;  // Re v - Im v of every basis vector (layout of V)
};
int outer_grid(long long n);
void launch_gstencil(const Stencil &st, int N, const double2 *x, double2 *y, const double2 *f, int nrhs,
                     const int *active, cudaStream_t s);
void launch_build_rhs(const Stencil &st, int N, double h, int npts, const double *pts, int nb,
                      const double *bumps, double2 *f, cudaStream_t s);
void launch_odots(const OuterBatch &B, const double2 *V, int nv, const double2 *w, double2 *part,
                  cudaStream_t s);
void launch_oupdate(const OuterBatch &B, const double2 *V, int nv, const double2 *h, double2 *w,
                    double2 *part_dots, double *part_norm, cudaStream_t s);
void launch_oupdate2(const OuterBatch &B, const double2 *V, const float2 *V32, int nv, const double2 *h,
                     double2 *w, const double *npart1, int g1, double *part_norm, int allow32, int *fallbacks,
                     cudaStream_t s);
// first CGS pass update in double-FP32 from the hi/lo FP32 basis; norm partials on its own grid
int oupdate_df_grid(long long n);
// delayed CGS2: fused dots of the pending vector and w, per-RHS coefficient kernels, fused update
int oupdate_dcgs_grid(long long n);
cudaError_t launch_odots2_df(const OuterBatch &B, const float2 *Vh, const float2 *Vl, int nv, const float2 *x1h,
                             const float2 *x1l, const double2 *w, double2 *part1, double2 *part2,
                             const unsigned *vmax, int bias, cudaStream_t s);
void launch_dcgs_col(const OuterBatch &B, double2 *H, double *cs, double2 *sn, double2 *g, double2 *Wq, int j,
                     const double2 *P1, double2 *P2, const double *hn, double *invs, const double *fnorm,
                     double *hist, int hstride, int it, int *err, unsigned *vmax, cudaStream_t s);
void launch_dcgs_tent(const OuterBatch &B, double2 *H, double2 *g, double2 *Wq, int j, const double *npart, int gp,
                      const double *fnorm, double tol, double *hn_out, int *flag, double *hist, int hstride, int it,
                      cudaStream_t s);
void launch_dcgs_close(const OuterBatch &B, double2 *H, double *cs, double2 *sn, double2 *g, double2 *Wq, int j,
                       const int *close, cudaStream_t s);
void launch_oupdate_dcgs(const OuterBatch &B, const float2 *Vh, const float2 *Vl, int j, int corr, double2 *Vj,
                         double *Dj, float2 *Vjh, float2 *Vjl, const double2 *acoef, const double2 *bcoef,
                         const double *invs, double2 *w, double *part_norm, unsigned *vmax, cudaStream_t s);
void launch_oupdate_df(const OuterBatch &B, const float2 *Vh, const float2 *Vl, int nv, const double2 *h,
                       double2 *w, double *part_norm, cudaStream_t s);
void launch_fill_test(long long n, unsigned long long seed, double2 *x, cudaStream_t s);
void launch_onorm(const OuterBatch &B, const double2 *x, double *part, cudaStream_t s);
void launch_oreduce(const OuterBatch &B, const double2 *part, int nv, double2 *out, cudaStream_t s);
void launch_ogivens(const OuterBatch &B, double2 *H, double *cs, double2 *sn, double2 *g, double2 *Wq, int j,
                    const double2 *h1, const double2 *h2, const double *npart, const double *fnorm,
                    double tol, double *hn_out, int *flag, double *hist, int hstride, int it,
                    cudaStream_t s);
void launch_oscale(const OuterBatch &B, double2 *out, float2 *out32, float2 *out32L, double *outD,
                   const double2 *w, const double *hn, cudaStream_t s);
// first CGS pass in double-FP32 arithmetic from the hi/lo FP32 copies of the basis
void launch_odots_df(const OuterBatch &B, const float2 *Vh, const float2 *Vl, int nv, const double2 *w,
                     double2 *part, cudaStream_t s);
void launch_otrisolve(const OuterBatch &B, const double2 *H, const double2 *g, const int *kcols, int kmax,
                      double2 *y, cudaStream_t s);
void launch_oaxpy(const OuterBatch &B, const double2 *y, const int *kcols, int kmax, const double2 *Zb,
                  double2 *x, cudaStream_t s);
void launch_oinit(const OuterBatch &B, const double2 *rv, const double *npart, double2 *V, float2 *V32,
                  float2 *V32L, double *D, double2 *g, double2 *Wq, double *beta_out, cudaStream_t s);
void launch_orotate(const OuterBatch &B, double2 *H, const double *cs, const double2 *sn, const int *kcols,
                    int kmax, cudaStream_t s);
cudaError_t set_outer_smem_limits(size_t bytes);

// tensor-core inference of the warm-start network (kernels_cnn_tc.cu)
void launch_cnn_l1_bf16(const Task *tasks, const Tile *tiles, int ntiles, const __nv_bfloat16 *W, const float *b,
                        const float *X0, uint4 *X1, long long ptot, cudaStream_t s);
void launch_cnn_tc_weights(const __nv_bfloat16 *Wb, __nv_bfloat16 *img2, __nv_bfloat16 *img3,
                           __nv_bfloat16 *img4, cudaStream_t s);
size_t conv_tc_smem(int nco, int wmax);
cudaError_t set_conv_tc_smem(int wmax);
void launch_conv_tc(int nco, int grid, const Task *tasks, const int2 *tct, int ntct, const uint4 *X, long long ptot,
                    const uint4 *Wimg, const float *bias, uint4 *Y, float2 *A4, int wmax, int *err, cudaStream_t s);

// grid coarse space of the two-level variant (kernels_cgrid.cu): the fine mesh of N intervals,
// coarsening factor c, Nc = N / c coarse intervals, m = Nc - 1 coarse unknowns per axis
struct CGrid { int N, c, Nc, m, diag; };
template <typename T>
void launch_cg_restrict(const CGrid &g, const double2 *v, c2<T> *vH, int nrhs, long long ldv, long long ldh,
                        const int *active, cudaStream_t s);
template <typename T>
void launch_cg_prolong(const CGrid &g, const c2<T> *xH, double2 *z, int accumulate, int nrhs, long long ldv,
                       long long ldh, const int *active, cudaStream_t s);
template <typename T>
void launch_dst_pass(int m, const T *S, const T *Dinv, const c2<T> *in, c2<T> *out, int nrhs, long long ldh,
                     const int *active, cudaStream_t s);
void launch_cg_widen(long long n, const float2 *in, double2 *out, cudaStream_t s);
void launch_cg_narrow(long long n, const double2 *in, float2 *out, cudaStream_t s);

}  // namespace hdd
