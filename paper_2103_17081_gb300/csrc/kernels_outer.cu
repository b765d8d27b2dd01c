// kernels_outer.cu — FP64 kernels on global vectors: the matrix-free P1 operator (Eq. 2), the
// load vector (§3), and the outer flexible GMRES (§3): classical Gram-Schmidt applied twice,
// complex Givens rotations and the solution update, all in complex128.
//
// Reductions are two-stage and deterministic: OUTER_CTAS CTAs each own a fixed contiguous chunk
// and write one partial per basis vector; a second kernel adds the partials in CTA order.
#include "hdd_common.cuh"

namespace hdd {

constexpr int OUTER_CTAS = 2 * 152;     // two CTAs per SM of a GB300 (minimum grid)
constexpr int OT = 256;                 // threads per outer CTA
constexpr int OCH = 1536;               // largest chunk one CTA owns (staged in shared memory)
constexpr int OT2 = 512;                // threads of the memory-bound FP32 second pass (more loads in flight)
// CTAs of the chunked reductions over a vector of n entries
int outer_grid(long long n) {
    long long g = (n + OCH - 1) / OCH;
    return (int)(g > OUTER_CTAS ? g : OUTER_CTAS);
}

// y = A x (f == nullptr) or y = f - A x on the (N-1)² interior grid, zero Dirichlet values, or
// (impedance condition) on all (N+1)² nodes with the boundary rows of their node class;
// blockIdx.y selects the right-hand side (vectors of n entries, consecutive).  IMP: compiled for
// the impedance condition.
template <bool IMP>
__global__ void k_gstencil(Stencil st, int N, const double2 *__restrict__ x, double2 *__restrict__ y,
                           const double2 *__restrict__ f, const int *__restrict__ active) {
    if (active && !active[blockIdx.y]) return;
    const int w = IMP ? N + 1 : N - 1;
    const long long n = (long long)w * w;
    x += blockIdx.y * n;
    y += blockIdx.y * n;
    if (f) f += blockIdx.y * n;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int ix = (int)(i % w), iy = (int)(i / w);
        auto X = [&](int a, int b) -> double2 {
            if (a < 0 || a >= w || b < 0 || b >= w) return make_double2(0.0, 0.0);
            return x[(long long)b * w + a];
        };
        double2 c = X(ix, iy), e = X(ix + 1, iy), wv = X(ix - 1, iy), nn = X(ix, iy + 1), s = X(ix, iy - 1);
        double2 d1, d2;
        if (st.diag == 0) { d1 = X(ix + 1, iy + 1); d2 = X(ix - 1, iy - 1); }
        else { d1 = X(ix + 1, iy - 1); d2 = X(ix - 1, iy + 1); }
        double2 r;
        const int cls = IMP ? node_class(N, ix, iy) : 4;    // impedance: ix, iy are mesh indices
        if (cls != 4) {
            const double2 *cf = st.bcoef + cls * 7;
            const double2 v[7] = {c, e, wv, nn, s, d1, d2};
            r = make_double2(0.0, 0.0);
            for (int q = 0; q < 7; q++) {
                const double2 a = cf[q];
                r.x += a.x * v[q].x - a.y * v[q].y;
                r.y += a.x * v[q].y + a.y * v[q].x;
            }
        } else {
            r.x = st.c0 * c.x + st.c1 * (((e.x + wv.x) + nn.x) + s.x) + st.c2 * (d1.x + d2.x);
            r.y = st.c0 * c.y + st.c1 * (((e.y + wv.y) + nn.y) + s.y) + st.c2 * (d1.y + d2.y);
        }
        if (f) { double2 fv = f[i]; r.x = fv.x - r.x; r.y = fv.y - r.y; }
        y[i] = r;
    }
}

// Load vector F = Σ amp·e_c (point sources snapped to the nearest node that is an unknown) + Σ M g
// (Gaussian bumps, g the nodal values at the unknowns, M the P1 mass matrix: at interior nodes
// h²/12 · [6 centre; 1 at E, W, N, S and the two diagonal corners], at boundary nodes of the
// impedance problem the row of the node's class).
__global__ void k_build_rhs(Stencil st, int N, double h, int npts, const double *__restrict__ pts,
                            int nb, const double *__restrict__ bumps, double2 *__restrict__ f) {
    const int diag = st.diag;
    const int lo = st.bc ? 0 : 1, hi = st.bc ? N : N - 1;
    const int w = hi - lo + 1;
    const long long n = (long long)w * w;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int gi = (int)(i % w) + lo, gj = (int)(i / w) + lo;
        double v = 0.0;
        for (int p = 0; p < npts; p++) {
            int pi = (int)floor(pts[3 * p] * N + 0.5), pj = (int)floor(pts[3 * p + 1] * N + 0.5);
            pi = pi < lo ? lo : (pi > hi ? hi : pi);
            pj = pj < lo ? lo : (pj > hi ? hi : pj);
            if (pi == gi && pj == gj) v += pts[3 * p + 2];
        }
        const int cls = st.bc ? node_class(N, gi, gj) : 4;
        for (int b = 0; b < nb; b++) {
            const double cx = bumps[4 * b], cy = bumps[4 * b + 1], sg = bumps[4 * b + 2], amp = bumps[4 * b + 3];
            auto g = [&](int a, int c) -> double {
                if (a < lo || a > hi || c < lo || c > hi) return 0.0;
                double dx = a * h - cx, dy = c * h - cy;
                return amp * exp(-(dx * dx + dy * dy) / (2.0 * sg * sg));
            };
            if (cls != 4) {
                const double *mr = st.bmass + cls * 7;
                double s = 0.0;
                for (int q = 0; q < 7; q++) {
                    int dx, dy;
                    stencil_offset(diag, q, dx, dy);
                    s += mr[q] * g(gi + dx, gj + dy);
                }
                v += s;
                continue;
            }
            double s = 6.0 * g(gi, gj) + g(gi + 1, gj) + g(gi - 1, gj) + g(gi, gj + 1) + g(gi, gj - 1);
            if (diag == 0) s += g(gi + 1, gj + 1) + g(gi - 1, gj - 1);
            else s += g(gi + 1, gj - 1) + g(gi - 1, gj + 1);
            v += h * h / 12.0 * s;
        }
        f[i] = make_double2(v, 0.0);
    }
}

__device__ __forceinline__ void chunk_of(long long n, long long &b, long long &e) {
    long long per = (n + gridDim.x - 1) / gridDim.x;
    b = blockIdx.x * per;
    e = b + per < n ? b + per : n;
}
// the same with an even chunk length (even chunk starts)
__device__ __forceinline__ void chunk_even(long long n, long long &b, long long &e) {
    long long per = (n + gridDim.x - 1) / gridDim.x;
    per += per & 1;
    b = blockIdx.x * per;
    e = b + per < n ? b + per : n;
    if (e < b) e = b;
}

// ------------------------------------------------------------------------------------------
// Outer FGMRES kernels, batched over independent right-hand sides (blockIdx.y = r).  Layout
// (OuterBatch): basis vector l of RHS r at V + l·ld + r·n (ld = nrhs·n), per-RHS work vectors at
// w + r·n, per-RHS reduction partials at part + r·G·ldp, Hessenberg of RHS r at
// H + r·(R+1)·R (column-major, leading dimension R+1).  A RHS with active[r] == 0 is skipped.
// ------------------------------------------------------------------------------------------

// Each CTA owns one contiguous chunk of the vectors (at most OCH entries).  The chunk of w is
// staged in shared memory once (stage_w); then warp q of the CTA forms the partial dots of
// vectors l = q, q + 8, ... over the chunk with shuffle reductions only (no block barrier per
// vector).  Dot products use the three-multiplication (Gauss) form of the complex product:
// with d = Re v - Im v stored per basis vector and a = Re w, p = Re w + Im w, m = Im w - Re w
// staged once per element of w,
//   conj(v)·w = (P + Q) + i (P + S),  P = d·a,  Q = Im v·p,  S = Re v·m,
// three FP64 FMAs per vector and element instead of four (the passes are bound by the FP64
// pipe, not by the extra 8 bytes of d).  Normwise its rounding error is within a small
// constant of the four-multiplication form's.
struct WStage { double a[OCH], p[OCH], m[OCH]; };

__device__ __forceinline__ void stage_w(WStage &ws, int i, double2 x) {
    ws.a[i] = x.x; ws.p[i] = x.x + x.y; ws.m[i] = x.y - x.x;
}

__device__ __forceinline__ void warp_dots(const double2 *__restrict__ V, const double *__restrict__ D,
                                          long long ld, int nv, const WStage &ws, long long b, int len,
                                          double2 *__restrict__ part, int ldp) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int l = warp; l < nv; l += OT / 32) {
        const double2 *vl = V + (long long)l * ld + b;
        const double *dl = D + (long long)l * ld + b;
        double p0 = 0.0, q0 = 0.0, s0 = 0.0, p1 = 0.0, q1 = 0.0, s1 = 0.0;
        int i = lane;
        for (; i + 32 < len; i += 64) {
            const double2 v0 = vl[i], v1 = vl[i + 32];
            const double d0 = dl[i], d1 = dl[i + 32];
            p0 = fma(d0, ws.a[i], p0); q0 = fma(v0.y, ws.p[i], q0); s0 = fma(v0.x, ws.m[i], s0);
            p1 = fma(d1, ws.a[i + 32], p1); q1 = fma(v1.y, ws.p[i + 32], q1); s1 = fma(v1.x, ws.m[i + 32], s1);
        }
        if (i < len) {
            const double2 v0 = vl[i];
            p0 = fma(dl[i], ws.a[i], p0); q0 = fma(v0.y, ws.p[i], q0); s0 = fma(v0.x, ws.m[i], s0);
        }
        const double P = p0 + p1;
        double re = P + (q0 + q1), im = P + (s0 + s1);
        for (int o = 16; o > 0; o >>= 1) { re += shfl_xor(re, o); im += shfl_xor(im, o); }
        if (lane == 0) part[(long long)blockIdx.x * ldp + l] = make_double2(re, im);
    }
}

// Partial dots part[r][cta][l] = Σ_{chunk} conj(V_{r,l}) w_r, l < nv.
__global__ void __launch_bounds__(OT)
k_odots(OuterBatch B, const double2 *__restrict__ V, int nv, const double2 *__restrict__ w,
        double2 *__restrict__ part) {
    __shared__ WStage ws;
    const int r = blockIdx.y;
    if (B.active && !B.active[r]) return;
    V += r * B.n; w += r * B.n; part += (long long)r * B.G * B.ldp;
    const double *D = B.D + r * B.n;
    long long b, e;
    chunk_of(B.n, b, e);
    const int len = (int)(e > b ? e - b : 0);
    for (int i = threadIdx.x; i < len; i += OT) stage_w(ws, i, w[b + i]);
    __syncthreads();
    warp_dots(V, D, B.ld, nv, ws, b, len, part, B.ldp);
}

// ------------------------------------------------------------------------------------------
// First CGS pass in double-FP32 arithmetic.  The basis is kept as two FP32 copies, hi = fl32(v)
// and lo = fl32(v - hi) (v = hi + lo to about 2^-48 relative), and w is split the same way per
// element.  Each real product x·y is formed as the exact product of the high parts (p, and its
// rounding error e = fma(xh, yh, -p)) plus the two cross terms xh·yl + xl·yh; p is added to the
// running sum with an error-free two-sum (Knuth) and everything small goes to a second FP32
// accumulator (the compensated dot product of Ogita, Rump & Oishi, SIAM J. Sci. Comput. 2005,
// on split inputs).  Per lane the error is at most u·|sum| + γ_m² Σ|v_i w_i| with u = 2^-24 and
// m the terms the lane adds (a few tens here: a chunk of ≤ 1536 elements over 64 accumulator
// sets); the lane results are widened to FP64 and reduced in FP64.  Checked on the CPU against
// exact rational sums: ≤ 2e-15 of Σ|v_i||w_i|, as accurate as an FP64 sum of the same terms.
// That is far below what the second CGS pass needs (it runs in FP64 and removes whatever the
// first pass left; the first-pass error only has to keep the second-pass coefficients small
// enough for the guarded FP32 correction of k_oupdate2).  These passes run
// on the FP32 pipe and read 16 bytes per basis vector and element (hi + lo), where the FP64
// Gauss form needs three FP64 FMAs and 24 bytes.  The _rn intrinsics keep the compiler from
// contracting the error-free steps into fused multiply-adds.
// ------------------------------------------------------------------------------------------
struct WStageDF { float4 w[OCH]; };        // (Re hi, Re lo, Im hi, Im lo) per element


// w (FP64) split per element into (Re hi, Re lo, Im hi, Im lo) for the double-FP32 dots
__device__ __forceinline__ void stage_w_df(WStageDF &ws, int i, double2 x) {
    const float rh = (float)x.x, ih = (float)x.y;
    ws.w[i] = make_float4(rh, (float)(x.x - (double)rh), ih, (float)(x.y - (double)ih));
}

// Warp q of the CTA forms the partial dots of vectors l = q, q + 8, ... over the chunk
// [b, b + len) from the hi/lo FP32 basis (element stride of the copies: B.ld32 between vectors).
__device__ __forceinline__ void warp_dots_df(const float2 *__restrict__ Vh, const float2 *__restrict__ Vl,
                                             long long ld32, int nv, const WStageDF &ws, long long b, int len,
                                             double2 *__restrict__ part, int ldp) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int l = warp; l < nv; l += OT / 32) {
        const float2 *hp = Vh + (long long)l * ld32 + b, *lp = Vl + (long long)l * ld32 + b;
        // four independent accumulator sets (elements i, i + 32, i + 64, i + 96), software-
        // pipelined: the eight basis loads of the next group are issued before the current
        // group's arithmetic (the pass is bound by bytes in flight, not by the FP32 pipe)
        float sh[4][2], sl[4][2];
#pragma unroll
        for (int u = 0; u < 4; u++) { sh[u][0] = sh[u][1] = sl[u][0] = sl[u][1] = 0.f; }
        const int full = len & ~127;                     // elements in whole groups of 128
        float2 vh[4], vl[4];
        int i = lane;
        if (i < full) {
#pragma unroll
            for (int u = 0; u < 4; u++) { vh[u] = hp[i + 32 * u]; vl[u] = lp[i + 32 * u]; }
        }
        for (; i < full; i += 128) {
            float2 nh[4], nl[4];
            const bool more = i + 128 < full;
#pragma unroll
            for (int u = 0; u < 4; u++) {
                nh[u] = more ? hp[i + 128 + 32 * u] : make_float2(0.f, 0.f);
                nl[u] = more ? lp[i + 128 + 32 * u] : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const float4 x = ws.w[i + 32 * u];
                // conj(v)·w = (vr wr + vi wi) + i (vr wi - vi wr)
                df_acc(sh[u][0], sl[u][0], vh[u].x, vl[u].x, x.x, x.y);
                df_acc(sh[u][1], sl[u][1], vh[u].x, vl[u].x, x.z, x.w);
                df_acc(sh[u][0], sl[u][0], vh[u].y, vl[u].y, x.z, x.w);
                df_acc(sh[u][1], sl[u][1], -vh[u].y, -vl[u].y, x.x, x.y);
            }
#pragma unroll
            for (int u = 0; u < 4; u++) { vh[u] = nh[u]; vl[u] = nl[u]; }
        }
        for (i = full + lane; i < len; i += 32) {
            const float2 h1 = hp[i], l1 = lp[i];
            const float4 x = ws.w[i];
            df_acc(sh[0][0], sl[0][0], h1.x, l1.x, x.x, x.y);
            df_acc(sh[0][1], sl[0][1], h1.x, l1.x, x.z, x.w);
            df_acc(sh[0][0], sl[0][0], h1.y, l1.y, x.z, x.w);
            df_acc(sh[0][1], sl[0][1], -h1.y, -l1.y, x.x, x.y);
        }
        // the four sets and then the 32 lanes are added as (hi, lo) pairs in FP32 (two-sum for
        // the high parts, low parts added): the epilogue stays off the FP64 pipe; lane 0 widens
        // the result to FP64
#pragma unroll
        for (int u = 1; u < 4; u++) {
            df_add(sh[0][0], sl[0][0], sh[u][0], sl[u][0]);
            df_add(sh[0][1], sl[0][1], sh[u][1], sl[u][1]);
        }
        for (int o = 16; o > 0; o >>= 1) {
            const float rh = __shfl_xor_sync(0xffffffffu, sh[0][0], o), rl = __shfl_xor_sync(0xffffffffu, sl[0][0], o);
            const float ih = __shfl_xor_sync(0xffffffffu, sh[0][1], o), il = __shfl_xor_sync(0xffffffffu, sl[0][1], o);
            df_add(sh[0][0], sl[0][0], rh, rl);
            df_add(sh[0][1], sl[0][1], ih, il);
        }
        if (lane == 0)
            part[(long long)blockIdx.x * ldp + l] = make_double2((double)sh[0][0] + (double)sl[0][0],
                                                                 (double)sh[0][1] + (double)sl[0][1]);
    }
}

// Partial dots part[r][cta][l] = Σ_{chunk} conj(V_{r,l}) w_r, l < nv, from the hi/lo FP32 basis.
__global__ void __launch_bounds__(OT, 3)
k_odots_df(OuterBatch B, const float2 *__restrict__ Vh, const float2 *__restrict__ Vl, int nv,
           const double2 *__restrict__ w, double2 *__restrict__ part) {
    __shared__ WStageDF ws;
    const int r = blockIdx.y;
    if (B.active && !B.active[r]) return;
    Vh += r * B.n32; Vl += r * B.n32; w += r * B.n; part += (long long)r * B.G * B.ldp;
    long long b, e;
    chunk_of(B.n, b, e);
    const int len = (int)(e > b ? e - b : 0);
    for (int i = threadIdx.x; i < len; i += OT) stage_w_df(ws, i, w[b + i]);
    __syncthreads();
    warp_dots_df(Vh, Vl, B.ld32, nv, ws, b, len, part, B.ldp);
}

// x -= Σ_{l<nv} hs[l] V_l(i) in FP64 with two independent accumulation chains.
__device__ __forceinline__ double2 update_fp64(double2 x0, const double2 *__restrict__ vp, long long ld,
                                               const double2 *__restrict__ hs, int nv) {
    double2 x1 = make_double2(0.0, 0.0);
    int l = 0;
    for (; l + 1 < nv; l += 2) {
        caxpy_neg<double>(x0, hs[l], vp[(long long)l * ld]);
        caxpy_neg<double>(x1, hs[l + 1], vp[(long long)(l + 1) * ld]);
    }
    if (l < nv) caxpy_neg<double>(x0, hs[l], vp[(long long)l * ld]);
    return make_double2(x0.x + x1.x, x0.y + x1.y);
}

// x -= Σ_{l<nv} h_l V_l(i) in the three-multiplication form: with d = Re v - Im v (stored per
// basis vector) and c0 = Re h, c1 = Re h - Im h, c2 = Re h + Im h (staged per vector),
//   h·v = (A + B) + i (C - A),  A = c0·d,  B = c1·Im v,  C = c2·Re v;
// A, B and C are summed over l (two chains each) and combined once per element.
__device__ __forceinline__ double2 update_gauss(double2 x, const double2 *__restrict__ vp,
                                                const double *__restrict__ dp, long long ld,
                                                const double *__restrict__ c0, const double *__restrict__ c1,
                                                const double *__restrict__ c2, int nv) {
    double a0 = 0.0, b0 = 0.0, k0 = 0.0, a1 = 0.0, b1 = 0.0, k1 = 0.0;
    int l = 0;
    for (; l + 1 < nv; l += 2) {
        const double2 v0 = vp[(long long)l * ld], v1 = vp[(long long)(l + 1) * ld];
        const double d0 = dp[(long long)l * ld], d1 = dp[(long long)(l + 1) * ld];
        a0 = fma(c0[l], d0, a0); b0 = fma(c1[l], v0.y, b0); k0 = fma(c2[l], v0.x, k0);
        a1 = fma(c0[l + 1], d1, a1); b1 = fma(c1[l + 1], v1.y, b1); k1 = fma(c2[l + 1], v1.x, k1);
    }
    if (l < nv) {
        const double2 v0 = vp[(long long)l * ld];
        a0 = fma(c0[l], dp[(long long)l * ld], a0); b0 = fma(c1[l], v0.y, b0); k0 = fma(c2[l], v0.x, k0);
    }
    const double A = a0 + a1;
    x.x -= A + (b0 + b1);
    x.y -= (k0 + k1) - A;
    return x;
}

// Block sum of one double per thread; thread 0 writes it to *out.
__device__ __forceinline__ void block_sum_store(double v, double *red, double *out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v += shfl_xor(v, o);
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); q++) s += red[q];
        *out = s;
    }
}

// w_r -= Σ_l h_{r,l} V_{r,l} in FP64 (three-multiplication form, update_gauss); then, if
// part_dots != null, partial dots V_r^H w_r; if part_norm != null, the partial ||w_r||² of the
// updated vector.  Dynamic shared memory: 3·nv doubles (c0 | c1 | c2).
__global__ void __launch_bounds__(OT)
k_oupdate(OuterBatch B, const double2 *__restrict__ V, int nv, const double2 *__restrict__ h,
          double2 *__restrict__ w, double2 *__restrict__ part_dots, double *__restrict__ part_norm) {
    extern __shared__ double hc[];
    __shared__ WStage ws;
    __shared__ double red[OT / 32];
    const int r = blockIdx.y;
    if (B.active && !B.active[r]) return;
    V += r * B.n; w += r * B.n; h += (long long)r * B.ldp;
    const double *D = B.D + r * B.n;
    long long b, e;
    chunk_of(B.n, b, e);
    const int len = (int)(e > b ? e - b : 0);
    double *c0 = hc, *c1 = hc + nv, *c2 = hc + 2 * nv;
    for (int l = threadIdx.x; l < nv; l += OT) {
        const double2 v = h[l];
        c0[l] = v.x; c1[l] = v.x - v.y; c2[l] = v.x + v.y;
    }
    __syncthreads();
    double nrm = 0.0;
    for (int i = threadIdx.x; i < len; i += OT) {
        const double2 x = update_gauss(w[b + i], V + b + i, D + b + i, B.ld, c0, c1, c2, nv);
        w[b + i] = x;
        stage_w(ws, i, x);
        nrm = fma(x.x, x.x, fma(x.y, x.y, nrm));
    }
    if (part_norm) block_sum_store(nrm, red, part_norm + (long long)r * B.G + blockIdx.x);
    if (part_dots) {
        __syncthreads();
        warp_dots(V, D, B.ld, nv, ws, b, len, part_dots + (long long)r * B.G * B.ldp, B.ldp);
    }
}

// Second CGS pass, w_r -= V_r h2_r, then the partial ||w_r||².  After the first pass (FP64 or
// double-FP32) the coefficients h2 = V^H w' are rounding-error sized, so the correction V h2 is
// tiny next to w'.  When Σ_l (|Re h2_l| + |Im h2_l|) <= 2^-34 ||w'_r|| (||w'_r||² = the sum of
// the g1 partials npart1 of RHS r) the correction is
// formed in FP32 from the FP32 copy V32 of the basis: products and partial sums over 32 vectors
// in FP32 (one chain per element), widened to FP64 between partial sums, subtracted from w' in
// FP64.  Its error is then at most about 2^-19 Σ|h2| <= 2^-53 ||w'_r|| in the 2-norm
// (||V_l|| = 1), under the FP64 unit roundoff of w' itself.  Otherwise (or with allow32 == 0) the FP64 update runs from V; every
// such RHS-iteration adds one to *fallbacks.  The guard is evaluated identically in every CTA
// (fixed-order sums), so all chunks of one RHS take the same path.
__global__ void __launch_bounds__(OT2)
k_oupdate2(OuterBatch B, const double2 *__restrict__ V, const float2 *__restrict__ V32, int nv,
           const double2 *__restrict__ h, double2 *__restrict__ w, const double *__restrict__ npart1, int g1,
           double *__restrict__ part_norm, int allow32, int *__restrict__ fallbacks) {
    extern __shared__ double2 hs[];
    __shared__ double red[OT2 / 32];
    __shared__ int use32_s;
    const int r = blockIdx.y;
    if (B.active && !B.active[r]) return;
    V += r * B.n; w += r * B.n; h += (long long)r * B.ldp; npart1 += (long long)r * g1;
    if (V32) V32 += r * B.n32;
    const int lane = threadIdx.x & 31;
    if (threadIdx.x < 32) {
        double a = 0.0, q2 = 0.0;
        for (int l = lane; l < nv; l += 32) a += fabs(h[l].x) + fabs(h[l].y);
        for (int q = lane; q < g1; q += 32) q2 += npart1[q];
        for (int o = 16; o > 0; o >>= 1) { a += shfl_xor(a, o); q2 += shfl_xor(q2, o); }
        if (lane == 0) {
            const int u = allow32 && V32 && a <= ldexp(sqrt(q2), -34);
            use32_s = u;
            if (!u && blockIdx.x == 0 && fallbacks) atomicAdd(fallbacks, 1);
        }
    }
    __syncthreads();
    const bool use32 = use32_s != 0;
    long long b, e;
    chunk_even(B.n, b, e);
    const int len = (int)(e - b);
    float2 *hf = reinterpret_cast<float2 *>(hs);
    for (int l = threadIdx.x; l < nv; l += OT2) {
        const double2 v = h[l];
        if (use32) hf[l] = make_float2((float)v.x, (float)v.y);
        else hs[l] = v;
    }
    __syncthreads();
    double nrm = 0.0;
    if (use32) {
        // element pairs (b + 2p, b + 2p + 1) as one 16-byte load per basis vector: b, n32 and
        // ld32 are even; an odd last pair reads the padding entry of its RHS and drops it
        const float4 *vp4 = reinterpret_cast<const float4 *>(V32 + b);
        const long long ld4 = B.ld32 / 2;
        for (int p = threadIdx.x; 2 * p < len; p += OT2) {
            const int i = 2 * p;
            const bool two = i + 1 < len;
            double2 xa = w[b + i], xb = two ? w[b + i + 1] : make_double2(0.0, 0.0);
            double ax = 0.0, ay = 0.0, bx = 0.0, by = 0.0;
            for (int l0 = 0; l0 < nv; l0 += 32) {
                const int l1 = l0 + 32 < nv ? l0 + 32 : nv;
                float pax = 0.f, pay = 0.f, pbx = 0.f, pby = 0.f;
#pragma unroll 8
                for (int l = l0; l < l1; l++) {
                    const float4 v = vp4[(long long)l * ld4 + p];
                    const float2 hh = hf[l];
                    pax = fmaf(hh.x, v.x, pax); pax = fmaf(-hh.y, v.y, pax);
                    pay = fmaf(hh.x, v.y, pay); pay = fmaf(hh.y, v.x, pay);
                    pbx = fmaf(hh.x, v.z, pbx); pbx = fmaf(-hh.y, v.w, pbx);
                    pby = fmaf(hh.x, v.w, pby); pby = fmaf(hh.y, v.z, pby);
                }
                ax += (double)pax; ay += (double)pay; bx += (double)pbx; by += (double)pby;
            }
            xa.x -= ax; xa.y -= ay;
            w[b + i] = xa;
            nrm = fma(xa.x, xa.x, fma(xa.y, xa.y, nrm));
            if (two) {
                xb.x -= bx; xb.y -= by;
                w[b + i + 1] = xb;
                nrm = fma(xb.x, xb.x, fma(xb.y, xb.y, nrm));
            }
        }
    } else {
        for (int i = threadIdx.x; i < len; i += OT2) {
            const double2 x = update_fp64(w[b + i], V + b + i, B.ld, hs, nv);
            w[b + i] = x;
            nrm = fma(x.x, x.x, fma(x.y, x.y, nrm));
        }
    }
    block_sum_store(nrm, red, part_norm + (long long)r * B.G + blockIdx.x);
}

// First CGS pass update w_r -= Σ_l h_{r,l} V_{r,l} in double-FP32 arithmetic from the hi/lo FP32
// copies of the basis (V = Vh + Vl to 2^-48 relative), then the partial ||w_r||² of the updated
// vector (one partial per CTA of this kernel's own grid).  Each coefficient is split once per
// CTA into (hi, lo) FP32 pairs; every real product v·h is formed as in the dot products (df_acc:
// exact product of the high parts, the two cross terms, a two-sum into a (hi, lo) FP32
// accumulator); the accumulators are widened to FP64 after every block of 32 basis vectors and
// the FP64 total is subtracted from w.  Per block the sum carries at most 2^-48 |S_b| +
// (32·2^-24)² Σ_b |v_l h_l| (Ogita, Rump & Oishi's bound for the compensated sum, the final
// rounding to FP32 replaced by the widening), i.e. 3.6e-12 Σ|v_l h_l| in the worst case and
// about 32·2^-48 typically, against nv·2^-53 Σ|v_l h_l| for the FP64 Gauss-form update
// (1.4e-13 at nv = 1270).  The second CGS pass removes the basis components of that error;
// what is left perturbs the next basis vector far below the outer tolerance.  The pass reads 16 B
// per basis vector and element and runs on the FP32 pipe (≈ 48 instructions per vector and
// element), where the FP64 update is bound by the FP64 pipe.  Thread q of the grid takes the
// element pair (2q, 2q + 1) with 16-byte loads; an odd last pair reads the padding entry of
// its RHS (n32 = n + (n & 1)) and drops it.  The CTA size (≤ OTU) is chosen so that the grid
// fills whole waves of resident CTAs (oupdate_df_plan).
constexpr int OTU = 256;
__global__ void __launch_bounds__(OTU, 3)
k_oupdate_df(OuterBatch B, const float2 *__restrict__ Vh, const float2 *__restrict__ Vl, int nv,
             const double2 *__restrict__ h, double2 *__restrict__ w, double *__restrict__ part_norm) {
    extern __shared__ float4 hq[];              // (Re hi, Re lo, Im hi, Im lo) of h_l
    __shared__ double red[OTU / 32];
    const int r = blockIdx.y;
    if (B.active && !B.active[r]) return;
    Vh += r * B.n32; Vl += r * B.n32; w += r * B.n; h += (long long)r * B.ldp;
    for (int l = threadIdx.x; l < nv; l += blockDim.x) {
        const double2 v = h[l];
        const float rh = (float)v.x, ih = (float)v.y;
        hq[l] = make_float4(rh, (float)(v.x - (double)rh), ih, (float)(v.y - (double)ih));
    }
    __syncthreads();
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x, i = 2 * p;
    double nrm = 0.0;
    if (i < B.n) {
        const bool two = i + 1 < B.n;
        const float4 *hp = reinterpret_cast<const float4 *>(Vh) + p;
        const float4 *lp = reinterpret_cast<const float4 *>(Vl) + p;
        const long long ld4 = B.ld32 / 2;
        double ax = 0.0, ay = 0.0, bx = 0.0, by = 0.0;
        float axh = 0.f, axl = 0.f, ayh = 0.f, ayl = 0.f, bxh = 0.f, bxl = 0.f, byh = 0.f, byl = 0.f;
        // v·h = (vr hr - vi hi) + i (vr hi + vi hr) for elements a = (x, y) and b = (z, w)
        auto acc = [&](const float4 vh, const float4 vl, const float4 c) {
            df_acc(axh, axl, vh.x, vl.x, c.x, c.y);
            df_acc(axh, axl, -vh.y, -vl.y, c.z, c.w);
            df_acc(ayh, ayl, vh.x, vl.x, c.z, c.w);
            df_acc(ayh, ayl, vh.y, vl.y, c.x, c.y);
            df_acc(bxh, bxl, vh.z, vl.z, c.x, c.y);
            df_acc(bxh, bxl, -vh.w, -vl.w, c.z, c.w);
            df_acc(byh, byl, vh.z, vl.z, c.z, c.w);
            df_acc(byh, byl, vh.w, vl.w, c.x, c.y);
        };
        for (int l0 = 0; l0 < nv; l0 += 32) {
            const int l1 = l0 + 32 < nv ? l0 + 32 : nv;
            int l = l0;
            // groups of four vectors: the eight 16-byte loads of a group are issued before its
            // arithmetic (the pass is bound by bytes in flight)
            for (; l + 4 <= l1; l += 4) {
                float4 vh[4], vl[4];
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    vh[u] = hp[(long long)(l + u) * ld4];
                    vl[u] = lp[(long long)(l + u) * ld4];
                }
#pragma unroll
                for (int u = 0; u < 4; u++) acc(vh[u], vl[u], hq[l + u]);
            }
            for (; l < l1; l++) acc(hp[(long long)l * ld4], lp[(long long)l * ld4], hq[l]);
            ax += (double)axh + (double)axl; ay += (double)ayh + (double)ayl;
            bx += (double)bxh + (double)bxl; by += (double)byh + (double)byl;
            axh = axl = ayh = ayl = bxh = bxl = byh = byl = 0.f;
        }
        double2 xa = w[i];
        xa.x -= ax; xa.y -= ay;
        w[i] = xa;
        nrm = fma(xa.x, xa.x, xa.y * xa.y);
        if (two) {
            double2 xb = w[i + 1];
            xb.x -= bx; xb.y -= by;
            w[i + 1] = xb;
            nrm = fma(xb.x, xb.x, fma(xb.y, xb.y, nrm));
        }
    }
    block_sum_store(nrm, red, part_norm + (long long)r * gridDim.x + blockIdx.x);
}

// Partial ||x_r||² per CTA: part[r][cta].
__global__ void __launch_bounds__(OT) k_onorm(OuterBatch B, const double2 *__restrict__ x, double *__restrict__ part) {
    __shared__ double red[OT / 32];
    const int r = blockIdx.y;
    if (B.active && !B.active[r]) return;
    x += r * B.n;
    long long b, e;
    chunk_of(B.n, b, e);
    double s = 0.0;
    for (long long i = b + threadIdx.x; i < e; i += OT) s = fma(x[i].x, x[i].x, fma(x[i].y, x[i].y, s));
    for (int o = 16; o > 0; o >>= 1) s += shfl_xor(s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < OT / 32; q++) t += red[q];
        part[(long long)r * B.G + blockIdx.x] = t;
    }
}

// out[r][l] = Σ_q part[r][q][l]: one warp per l, lane i adds q = i, i+32, ... in order, then a
// fixed shuffle tree (deterministic).
__global__ void k_oreduce(OuterBatch B, const double2 *__restrict__ part, int nv, double2 *__restrict__ out) {
    const int r = blockIdx.y;
    if (B.active && !B.active[r]) return;
    const int l = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (l >= nv) return;
    part += (long long)r * B.G * B.ldp;
    double2 s = make_double2(0.0, 0.0);
    for (int q = lane; q < B.G; q += 32) { double2 v = part[(long long)q * B.ldp + l]; s.x += v.x; s.y += v.y; }
    for (int o = 16; o > 0; o >>= 1) { s.x += shfl_xor(s.x, o); s.y += shfl_xor(s.y, o); }
    if (lane == 0) out[(long long)r * B.ldp + l] = s;
}

__device__ void zgivens(double2 a, double2 b, double &c, double2 &s, double2 &r) {
    double aa = hypot(a.x, a.y), bb = hypot(b.x, b.y);
    if (bb == 0.0) { c = 1.0; s = make_double2(0.0, 0.0); r = a; return; }
    if (aa == 0.0) { c = 0.0; s = make_double2(b.x / bb, -b.y / bb); r = make_double2(bb, 0.0); return; }
    double t = hypot(aa, bb);
    double2 ph = make_double2(a.x / aa, a.y / aa);
    c = aa / t;
    double2 cb = make_double2(b.x / t, -b.y / t);
    s = cmul<double>(ph, cb);
    r = make_double2(ph.x * t, ph.y * t);
}

// Outer Arnoldi column j of every active RHS (one CTA of OG threads each).  H keeps the
// unrotated columns h = h1 + h2 (CGS2) with h_{j+1,j} = sqrt(Σ norm partials) below them; the
// rotated entry that rotation j needs is formed without the sequential chain of the j earlier
// rotations: with Q_jᵀ = G_{j-1}⋯G_0 and W_j its row j, (Q_jᵀ h)_j = W_j · h (a parallel dot
// product), and G_j gives W_{j+1} = [-conj(s_j) W_j, c_j] (Wq, updated in place).  k_orotate
// forms the triangular factor at the end of a cycle.  Then the g update; flag[r] = 1 while
// |g_{j+1}| > tol·||f_r|| and h_{j+1,j} > 0; hist[r·hstride + it] records |g_{j+1}|/||f_r||.
constexpr int OG = 128;
__global__ void __launch_bounds__(OG)
k_ogivens(OuterBatch B, double2 *__restrict__ H, double *__restrict__ cs, double2 *__restrict__ sn,
          double2 *__restrict__ g, double2 *__restrict__ Wq, int j, const double2 *__restrict__ h1,
          const double2 *__restrict__ h2, const double *__restrict__ npart, const double *__restrict__ fnorm,
          double tol, double *__restrict__ hn_out, int *__restrict__ flag, double *__restrict__ hist,
          int hstride, int it) {
    __shared__ double red[OG / 32], redx[OG / 32], redy[OG / 32];
    __shared__ double c_s;
    __shared__ double2 s_s;
    const int r = blockIdx.x;
    if (B.active && !B.active[r]) return;
    const int R = B.R, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    H += (long long)r * (R + 1) * R; cs += (long long)r * R; sn += (long long)r * R;
    g += (long long)r * (R + 1); Wq += (long long)r * (R + 1);
    h1 += (long long)r * B.ldp; h2 += (long long)r * B.ldp; npart += (long long)r * B.G;
    double2 *hc = H + (long long)j * (R + 1);
    double s2 = 0.0;
    for (int q = tid; q < B.G; q += OG) s2 += npart[q];
    double dx = 0.0, dy = 0.0;
    for (int l = tid; l <= j; l += OG) {
        const double2 hv = make_double2(h1[l].x + h2[l].x, h1[l].y + h2[l].y);
        hc[l] = hv;
        const double2 wl = Wq[l];
        dx = fma(wl.x, hv.x, fma(-wl.y, hv.y, dx));
        dy = fma(wl.x, hv.y, fma(wl.y, hv.x, dy));
    }
    for (int o = 16; o > 0; o >>= 1) {
        s2 += shfl_xor(s2, o); dx += shfl_xor(dx, o); dy += shfl_xor(dy, o);
    }
    if (lane == 0) { red[warp] = s2; redx[warp] = dx; redy[warp] = dy; }
    __syncthreads();
    if (tid == 0) {
        double a = 0.0, bx = 0.0, by = 0.0;
        for (int q = 0; q < OG / 32; q++) { a += red[q]; bx += redx[q]; by += redy[q]; }
        const double hn = sqrt(a);
        hc[j + 1] = make_double2(hn, 0.0);
        double c; double2 sr, rr;
        zgivens(make_double2(bx, by), make_double2(hn, 0.0), c, sr, rr);
        cs[j] = c; sn[j] = sr;
        c_s = c; s_s = sr;
        const double2 gj = g[j];
        g[j + 1] = make_double2(-(sr.x * gj.x + sr.y * gj.y), -(sr.x * gj.y - sr.y * gj.x));
        g[j] = make_double2(c * gj.x, c * gj.y);
        const double res = hypot(g[j + 1].x, g[j + 1].y);
        hn_out[r] = hn;
        hist[(long long)r * hstride + it] = res / fnorm[r];
        flag[r] = (res > tol * fnorm[r] && hn > 0.0) ? 1 : 0;
    }
    __syncthreads();
    const double c = c_s;
    const double2 sr = s_s;
    for (int l = tid; l <= j; l += OG) {             // W_{j+1} = [-conj(s_j) W_j, c_j]
        const double2 wl = Wq[l];
        Wq[l] = make_double2(-(sr.x * wl.x + sr.y * wl.y), -(sr.x * wl.y - sr.y * wl.x));
    }
    if (tid == 0) Wq[j + 1] = make_double2(c, 0.0);
}

// ------------------------------------------------------------------------------------------
// Delayed CGS2 (the low-synchronisation classical Gram-Schmidt of Świrydowicz, Langou, Ananthan,
// Yang & Thomas, Numer. Linear Algebra Appl. 2021, applied to the flexible Arnoldi process).  At
// outer step j the basis slot j holds the pending vector ṽ_j = w'_{j-1}/ν_j: the previous step's
// first-pass result, normalised but not yet reorthogonalised, and column j-1 of H holds that
// step's first-pass coefficients with the tentative subdiagonal ν_j.  The preconditioner is
// applied to ṽ_j (FGMRES allows any z_j: the Arnoldi relation A Z = V H only needs the final
// orthonormal V), and one pass over the basis then forms both
//   a = V_{<j}^H ṽ_j, d = ṽ_j^H ṽ_j     (the second pass of vector j, delayed by one step)
//   b = V_{<j}^H w,   c = ṽ_j^H w       (the first pass of the new vector w = A z_j).
// With σ = sqrt(d - |a|²) the final v_j = (ṽ_j - V_{<j} a)/σ, column j-1 becomes
// h + ν_j a with subdiagonal ν_j σ, and v_j^H w = (c - a^H b)/σ; one more pass over the basis
// writes v_j and w' = w - V_{<j} b - v_j (v_j^H w) together.  Two passes per step instead of
// four; the stopping test runs on the tentative column j (its rotation is committed a step later,
// or at once when the cycle ends, the column then keeping its first-pass coefficients).
// ------------------------------------------------------------------------------------------

// Warp q forms the partial dots of vectors l = q, q + 8, ... with the two staged vectors s1, s2
// (double-FP32, as warp_dots_df; four element groups per pass, the next group's basis loads
// issued before the current group's arithmetic).  BIAS: the dots with w (s2, the first pass of
// the new vector) take the biased sums of df_acc_biased (6 FP32 instructions per product instead
// of 12).  Their error (a few 1e-12 of Σ|v w| instead of about 1e-15) needs no care: the first
// pass only has to leave w' nearly orthogonal to V, and the delayed second pass measures what it
// left, V^H ṽ, exactly and adds it to the column (the Arnoldi relation w = V h + ν σ v holds
// whatever the first-pass coefficients were).  The dots with s1 (that second pass, which sets
// the orthogonality of the basis) keep the two-sum.  The bias of vector l is the power of two
// M >= 4·T·vm_l·xm, T = 2·(len/128 + 4) the products one accumulator takes (len/128 whole
// groups plus at most four tail elements, two products each per component), vm_l >= |hi part|
// of every entry of V_l (vms[l] for the final slots, recorded by the update that wrote them; the
// chunk maximum of s1 for the last slot, which is s1) and xm the chunk maximum of w's hi parts.
template <bool BIAS>
__device__ __forceinline__ void warp_dots2_df(const float2 *__restrict__ Vh, const float2 *__restrict__ Vl,
                                              long long ld32, int nv, const float4 *__restrict__ s1,
                                              const float4 *__restrict__ s2, long long b, int len,
                                              double2 *__restrict__ part1, double2 *__restrict__ part2, int ldp,
                                              const float *__restrict__ vms, float xm1, float xm2) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float Tb = 4.001f * (float)(2 * ((len >> 7) + 4));
    for (int l = warp; l < nv; l += OT / 32) {
        const float2 *hp = Vh + (long long)l * ld32 + b, *lp = Vl + (long long)l * ld32 + b;
        const float M2 = BIAS ? pow2_ceil(Tb * (l < nv - 1 ? vms[l] : xm1) * xm2) : 0.f;
        float ah[4][2], al[4][2], bh[4][2], bl[4][2];
#pragma unroll
        for (int u = 0; u < 4; u++)
#pragma unroll
            for (int c = 0; c < 2; c++) { ah[u][c] = al[u][c] = bl[u][c] = 0.f; bh[u][c] = M2; }
        auto acc1 = [](float &sh, float &sl, float xh, float xl, float yh, float yl) {
            df_acc(sh, sl, xh, xl, yh, yl);
        };
        auto acc2 = [](float &sh, float &sl, float xh, float xl, float yh, float yl) {
            if (BIAS) df_acc_biased(sh, sl, xh, xl, yh, yl);
            else df_acc(sh, sl, xh, xl, yh, yl);
        };
        auto step = [&](int u, float2 h, float2 q, float4 x, float4 y) {
            // conj(v)·x = (vr xr + vi xi) + i (vr xi - vi xr), the same for y
            acc1(ah[u][0], al[u][0], h.x, q.x, x.x, x.y);
            acc1(ah[u][1], al[u][1], h.x, q.x, x.z, x.w);
            acc1(ah[u][0], al[u][0], h.y, q.y, x.z, x.w);
            acc1(ah[u][1], al[u][1], -h.y, -q.y, x.x, x.y);
            acc2(bh[u][0], bl[u][0], h.x, q.x, y.x, y.y);
            acc2(bh[u][1], bl[u][1], h.x, q.x, y.z, y.w);
            acc2(bh[u][0], bl[u][0], h.y, q.y, y.z, y.w);
            acc2(bh[u][1], bl[u][1], -h.y, -q.y, y.x, y.y);
        };
        const int full = len & ~127;
        float2 vh[4], vl[4];
        int i = lane;
        if (i < full) {
#pragma unroll
            for (int u = 0; u < 4; u++) { vh[u] = hp[i + 32 * u]; vl[u] = lp[i + 32 * u]; }
        }
        for (; i < full; i += 128) {
            float2 nh[4], nl[4];
            const bool more = i + 128 < full;
#pragma unroll
            for (int u = 0; u < 4; u++) {
                nh[u] = more ? hp[i + 128 + 32 * u] : make_float2(0.f, 0.f);
                nl[u] = more ? lp[i + 128 + 32 * u] : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < 4; u++) step(u, vh[u], vl[u], s1[i + 32 * u], s2[i + 32 * u]);
#pragma unroll
            for (int u = 0; u < 4; u++) { vh[u] = nh[u]; vl[u] = nl[u]; }
        }
        for (i = full + lane; i < len; i += 32) step(0, hp[i], lp[i], s1[i], s2[i]);
        if (BIAS) {            // remove the bias: sh in [3M/4, 5M/4], so sh - M is exact
#pragma unroll
            for (int u = 0; u < 4; u++)
#pragma unroll
                for (int c = 0; c < 2; c++) bh[u][c] = __fsub_rn(bh[u][c], M2);
        }
#pragma unroll
        for (int u = 1; u < 4; u++)
#pragma unroll
            for (int c = 0; c < 2; c++) {
                df_add(ah[0][c], al[0][c], ah[u][c], al[u][c]);
                df_add(bh[0][c], bl[0][c], bh[u][c], bl[u][c]);
            }
        for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
            for (int c = 0; c < 2; c++) {
                const float x1 = __shfl_xor_sync(0xffffffffu, ah[0][c], o), x2 = __shfl_xor_sync(0xffffffffu, al[0][c], o);
                const float y1 = __shfl_xor_sync(0xffffffffu, bh[0][c], o), y2 = __shfl_xor_sync(0xffffffffu, bl[0][c], o);
                df_add(ah[0][c], al[0][c], x1, x2);
                df_add(bh[0][c], bl[0][c], y1, y2);
            }
        }
        if (lane == 0) {
            part1[(long long)blockIdx.x * ldp + l] = make_double2((double)ah[0][0] + (double)al[0][0],
                                                                  (double)ah[0][1] + (double)al[0][1]);
            part2[(long long)blockIdx.x * ldp + l] = make_double2((double)bh[0][0] + (double)bl[0][0],
                                                                  (double)bh[0][1] + (double)bl[0][1]);
        }
    }
}

// Partials part1[r][cta][l] = Σ conj(V_l) x1 and part2[r][cta][l] = Σ conj(V_l) w for l < nv
// (x1: hi/lo copies of basis slot nv-1; w: FP64).  vmax[r·ldp + l], l < nv-1: max |hi part| of
// slot l as float bits (BIAS only).  Dynamic shared memory: 2 · chunk float4, then nv - 1 floats
// (BIAS).
template <bool BIAS>
__global__ void __launch_bounds__(OT, 2)
k_odots2_df(OuterBatch B, const float2 *__restrict__ Vh, const float2 *__restrict__ Vl, int nv,
            const float2 *__restrict__ x1h, const float2 *__restrict__ x1l, const double2 *__restrict__ w,
            double2 *__restrict__ part1, double2 *__restrict__ part2, const unsigned *__restrict__ vmax) {
    extern __shared__ float4 st2[];
    __shared__ float mx[2][OT / 32];
    const int r = blockIdx.y;
    if (B.active && !B.active[r]) return;
    Vh += r * B.n32; Vl += r * B.n32; x1h += r * B.n32; x1l += r * B.n32; w += r * B.n;
    part1 += (long long)r * B.G * B.ldp; part2 += (long long)r * B.G * B.ldp;
    long long b, e;
    chunk_of(B.n, b, e);
    const int len = (int)(e > b ? e - b : 0);
    const long long chunk = (B.n + gridDim.x - 1) / gridDim.x;
    float4 *s1 = st2, *s2 = st2 + len;
    float *vms = reinterpret_cast<float *>(st2 + 2 * chunk);
    float m1 = 0.f, m2 = 0.f;
    for (int i = threadIdx.x; i < len; i += OT) {
        const float2 h = x1h[b + i], q = x1l[b + i];
        s1[i] = make_float4(h.x, q.x, h.y, q.y);
        const double2 x = w[b + i];
        const float rh = (float)x.x, ih = (float)x.y;
        s2[i] = make_float4(rh, (float)(x.x - (double)rh), ih, (float)(x.y - (double)ih));
        m1 = fmaxf(m1, fmaxf(fabsf(h.x), fabsf(h.y)));
        m2 = fmaxf(m2, fmaxf(fabsf(rh), fabsf(ih)));
    }
    float xm1 = 0.f, xm2 = 0.f;
    if (BIAS) {
        vmax += (long long)r * B.ldp;
        for (int l = threadIdx.x; l < nv - 1; l += OT) vms[l] = __uint_as_float(vmax[l]);
        for (int o = 16; o > 0; o >>= 1) {
            m1 = fmaxf(m1, __shfl_xor_sync(0xffffffffu, m1, o));
            m2 = fmaxf(m2, __shfl_xor_sync(0xffffffffu, m2, o));
        }
        if ((threadIdx.x & 31) == 0) { mx[0][threadIdx.x >> 5] = m1; mx[1][threadIdx.x >> 5] = m2; }
    }
    __syncthreads();
    if (BIAS) {
#pragma unroll
        for (int q = 0; q < OT / 32; q++) { xm1 = fmaxf(xm1, mx[0][q]); xm2 = fmaxf(xm2, mx[1][q]); }
    }
    warp_dots2_df<BIAS>(Vh, Vl, B.ld32, nv, s1, s2, b, len, part1, part2, B.ldp, vms, xm1, xm2);
}

// Block reductions of the small per-RHS kernels (OG threads)
__device__ __forceinline__ double og_sum(double v, double *red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v += shfl_xor(v, o);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0.0;
    for (int q = 0; q < OG / 32; q++) s += red[q];
    return s;
}

// Rotation j of one RHS from the unrotated column hc (rows 0..j) and its subdiagonal hn: the
// rotated entry (Q_jᵀ h)_j = W_j · h, then cs, sn, g and W_{j+1} (commit) or only the residual
// estimate |g_{j+1}| (commit == false).  Returns |g_{j+1}| to every thread.
__device__ double givens_step(const double2 *__restrict__ hc, double hn, int j, double *cs, double2 *sn,
                              double2 *g, double2 *Wq, bool commit, double *red) {
    __shared__ double c_s, res_s;
    __shared__ double2 s_s;
    double dx = 0.0, dy = 0.0;
    for (int l = threadIdx.x; l <= j; l += OG) {
        const double2 hv = hc[l], wl = Wq[l];
        dx = fma(wl.x, hv.x, fma(-wl.y, hv.y, dx));
        dy = fma(wl.x, hv.y, fma(wl.y, hv.x, dy));
    }
    const double bx = og_sum(dx, red), by = og_sum(dy, red);
    if (threadIdx.x == 0) {
        double c; double2 sr, rr;
        zgivens(make_double2(bx, by), make_double2(hn, 0.0), c, sr, rr);
        const double2 gj = g[j];
        const double2 g1 = make_double2(-(sr.x * gj.x + sr.y * gj.y), -(sr.x * gj.y - sr.y * gj.x));
        res_s = hypot(g1.x, g1.y);
        c_s = c; s_s = sr;
        if (commit) {
            cs[j] = c; sn[j] = sr;
            g[j + 1] = g1;
            g[j] = make_double2(c * gj.x, c * gj.y);
        }
    }
    __syncthreads();
    const double res = res_s;
    if (commit) {
        const double c = c_s;
        const double2 sr = s_s;
        for (int l = threadIdx.x; l <= j; l += OG) {             // W_{j+1} = [-conj(s_j) W_j, c_j]
            const double2 wl = Wq[l];
            Wq[l] = make_double2(-(sr.x * wl.x + sr.y * wl.y), -(sr.x * wl.y - sr.y * wl.x));
        }
        if (threadIdx.x == 0) Wq[j + 1] = make_double2(c, 0.0);
        __syncthreads();
    }
    return res;
}

// Delayed CGS2 coefficients of step j for every active RHS (one CTA each).  P1 = V^H ṽ_j and
// P2 = V^H w over slots 0..j (reduced).  For j >= 1: column j-1 is completed (h += ν_j a,
// subdiagonal ν_j σ) and its rotation committed (hist[it-1], the final residual estimate after
// column j-1); invs = 1/σ; P2[j] becomes v_j^H w.  Then P2[0..j] is the first-pass column j,
// stored in H.  err[0] is set if σ² <= d/4 (the pending vector lost more than half of its norm
// to the basis, or is not finite): the delayed form then does not hold.  vmax[r·ldp + j] (the
// largest |hi part| of slot j, recorded by the update of this step) is cleared.
__global__ void __launch_bounds__(OG)
k_dcgs_col(OuterBatch B, double2 *__restrict__ H, double *__restrict__ cs, double2 *__restrict__ sn,
           double2 *__restrict__ g, double2 *__restrict__ Wq, int j, const double2 *__restrict__ P1,
           double2 *__restrict__ P2, const double *__restrict__ hn, double *__restrict__ invs,
           const double *__restrict__ fnorm, double *__restrict__ hist, int hstride, int it, int *__restrict__ err,
           unsigned *__restrict__ vmax) {
    __shared__ double red[OG / 32];
    __shared__ double2 hj_s;
    const int r = blockIdx.x;
    if (B.active && !B.active[r]) return;
    if (threadIdx.x == 0) vmax[(long long)r * B.ldp + j] = 0u;
    const int R = B.R;
    H += (long long)r * (R + 1) * R; cs += (long long)r * R; sn += (long long)r * R;
    g += (long long)r * (R + 1); Wq += (long long)r * (R + 1);
    P1 += (long long)r * B.ldp; P2 += (long long)r * B.ldp;
    double2 *hcol = H + (long long)j * (R + 1);
    if (j >= 1) {
        double q2 = 0.0, abx = 0.0, aby = 0.0;
        for (int l = threadIdx.x; l < j; l += OG) {
            const double2 a = P1[l], bb = P2[l];
            q2 = fma(a.x, a.x, fma(a.y, a.y, q2));
            abx = fma(a.x, bb.x, fma(a.y, bb.y, abx));          // conj(a)·b
            aby = fma(a.x, bb.y, fma(-a.y, bb.x, aby));
        }
        const double aa = og_sum(q2, red), sx = og_sum(abx, red), sy = og_sum(aby, red);
        const double d = P1[j].x, s2 = d - aa;
        const bool ok = s2 > 0.25 * d && isfinite(s2);
        const double sig = ok ? sqrt(s2) : 1.0;
        const double nu = hn[r];
        double2 *hp = H + (long long)(j - 1) * (R + 1);
        for (int l = threadIdx.x; l < j; l += OG) {
            const double2 a = P1[l];
            hp[l] = make_double2(fma(nu, a.x, hp[l].x), fma(nu, a.y, hp[l].y));
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            hp[j] = make_double2(nu * sig, 0.0);
            const double2 c = P2[j];
            hj_s = make_double2((c.x - sx) / sig, (c.y - sy) / sig);
            invs[r] = 1.0 / sig;
            if (!ok) atomicExch(err, 1);
        }
        __syncthreads();
        const double res = givens_step(hp, nu * sig, j - 1, cs, sn, g, Wq, true, red);
        if (threadIdx.x == 0) {
            hist[(long long)r * hstride + it - 1] = res / fnorm[r];
            P2[j] = hj_s;
        }
        __syncthreads();
    }
    for (int l = threadIdx.x; l <= j; l += OG) hcol[l] = P2[l];
}

// Tentative stopping test of step j: ν_{j+1} = ||w'|| (gp partials per RHS) as the subdiagonal
// of the first-pass column j, the residual estimate |g_{j+1}| that rotation j would give
// (nothing committed); flag[r] = 1 while it exceeds tol·||f_r|| and ν_{j+1} > 0.
__global__ void __launch_bounds__(OG)
k_dcgs_tent(OuterBatch B, double2 *__restrict__ H, double2 *__restrict__ g, double2 *__restrict__ Wq, int j,
            const double *__restrict__ npart, int gp, const double *__restrict__ fnorm, double tol,
            double *__restrict__ hn_out, int *__restrict__ flag, double *__restrict__ hist, int hstride, int it) {
    __shared__ double red[OG / 32];
    const int r = blockIdx.x;
    if (B.active && !B.active[r]) return;
    const int R = B.R;
    H += (long long)r * (R + 1) * R; g += (long long)r * (R + 1); Wq += (long long)r * (R + 1);
    npart += (long long)r * gp;
    double s = 0.0;
    for (int q = threadIdx.x; q < gp; q += OG) s += npart[q];
    const double nu = sqrt(og_sum(s, red));
    double2 *hcol = H + (long long)j * (R + 1);
    const double res = givens_step(hcol, nu, j, nullptr, nullptr, g, Wq, false, red);
    if (threadIdx.x == 0) {
        hcol[j + 1] = make_double2(nu, 0.0);
        hn_out[r] = nu;
        hist[(long long)r * hstride + it] = res / fnorm[r];
        flag[r] = (res > tol * fnorm[r] && nu > 0.0) ? 1 : 0;
    }
}

// End of a cycle for the RHS with close[r] = 1: rotation j of the first-pass column j (its
// subdiagonal ν_{j+1} in H) committed; the column keeps its first-pass coefficients.
__global__ void __launch_bounds__(OG)
k_dcgs_close(OuterBatch B, double2 *__restrict__ H, double *__restrict__ cs, double2 *__restrict__ sn,
             double2 *__restrict__ g, double2 *__restrict__ Wq, int j, const int *__restrict__ close) {
    __shared__ double red[OG / 32];
    const int r = blockIdx.x;
    if (!close[r]) return;
    const int R = B.R;
    H += (long long)r * (R + 1) * R; cs += (long long)r * R; sn += (long long)r * R;
    g += (long long)r * (R + 1); Wq += (long long)r * (R + 1);
    const double2 *hcol = H + (long long)j * (R + 1);
    givens_step(hcol, hcol[j + 1].x, j, cs, sn, g, Wq, true, red);
}

// Delayed CGS2 update of step j, one element pair per thread (as k_oupdate_df):
//   v_j = (ṽ_j - Σ_{l<j} V_l a_l)·invs   (corr = 1; slot j rewritten in FP64, Re - Im and hi/lo)
//   w'  = w - Σ_{l<j} V_l b_l - v_j b_j   (b_j = v_j^H w)
// The sums run over the hi/lo copies of slots 0..j-1: Σ V_l b_l in double-FP32 widened to FP64
// every 32 vectors (as k_oupdate_df); Σ V_l a_l in FP32 from the high parts (the coefficients a
// are rounding-error sized, so its error is far below the FP64 rounding of ṽ_j), widened every 32
// vectors.  corr = 0 (step 0): v_0 is final and only read.  Then the partial ||w'||², and the
// largest |hi part| of the final v_j (an atomic maximum on float bits into vmax[r·ldp + j],
// which k_dcgs_col cleared) for the biased dot products of the later steps.
// Dynamic shared memory: j · (float4 + float2).
__global__ void __launch_bounds__(OTU, 3)
k_oupdate_dcgs(OuterBatch B, const float2 *__restrict__ Vh, const float2 *__restrict__ Vl, int j, int corr,
               double2 *__restrict__ Vj, double *__restrict__ Dj, float2 *__restrict__ Vjh, float2 *__restrict__ Vjl,
               const double2 *__restrict__ acoef, const double2 *__restrict__ bcoef, const double *__restrict__ invs,
               double2 *__restrict__ w, double *__restrict__ part_norm, unsigned *__restrict__ vmax) {
    extern __shared__ float4 dq[];
    float4 *bq = dq;                                      // (Re hi, Re lo, Im hi, Im lo) of b_l
    float2 *aq = reinterpret_cast<float2 *>(dq + j);      // a_l in FP32
    __shared__ double red[OTU / 32];
    __shared__ float redm[OTU / 32];
    const int r = blockIdx.y;
    if (B.active && !B.active[r]) return;
    Vh += r * B.n32; Vl += r * B.n32; w += r * B.n; Vj += r * B.n; Dj += r * B.n;
    Vjh += r * B.n32; Vjl += r * B.n32;
    acoef += (long long)r * B.ldp; bcoef += (long long)r * B.ldp;
    for (int l = threadIdx.x; l < j; l += blockDim.x) {
        const double2 v = bcoef[l];
        const float rh = (float)v.x, ih = (float)v.y;
        bq[l] = make_float4(rh, (float)(v.x - (double)rh), ih, (float)(v.y - (double)ih));
        aq[l] = corr ? make_float2((float)acoef[l].x, (float)acoef[l].y) : make_float2(0.f, 0.f);
    }
    __syncthreads();
    const double2 hj = bcoef[j];
    const double is = corr ? invs[r] : 1.0;
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x, i = 2 * p;
    double nrm = 0.0;
    float vm = 0.f;
    if (i < B.n) {
        const bool two = i + 1 < B.n;
        const float4 *hp = reinterpret_cast<const float4 *>(Vh) + p;
        const float4 *lp = reinterpret_cast<const float4 *>(Vl) + p;
        const long long ld4 = B.ld32 / 2;
        double ax = 0.0, ay = 0.0, bx = 0.0, by = 0.0;        // Σ V b (elements a, b of the pair)
        double cx = 0.0, cy = 0.0, ex = 0.0, ey = 0.0;        // Σ V a
        float axh = 0.f, axl = 0.f, ayh = 0.f, ayl = 0.f, bxh = 0.f, bxl = 0.f, byh = 0.f, byl = 0.f;
        float cxf = 0.f, cyf = 0.f, exf = 0.f, eyf = 0.f;
        auto acc = [&](const float4 vh, const float4 vl, const float4 c, const float2 a) {
            df_acc(axh, axl, vh.x, vl.x, c.x, c.y);
            df_acc(axh, axl, -vh.y, -vl.y, c.z, c.w);
            df_acc(ayh, ayl, vh.x, vl.x, c.z, c.w);
            df_acc(ayh, ayl, vh.y, vl.y, c.x, c.y);
            df_acc(bxh, bxl, vh.z, vl.z, c.x, c.y);
            df_acc(bxh, bxl, -vh.w, -vl.w, c.z, c.w);
            df_acc(byh, byl, vh.z, vl.z, c.z, c.w);
            df_acc(byh, byl, vh.w, vl.w, c.x, c.y);
            cxf = fmaf(vh.x, a.x, fmaf(-vh.y, a.y, cxf));
            cyf = fmaf(vh.x, a.y, fmaf(vh.y, a.x, cyf));
            exf = fmaf(vh.z, a.x, fmaf(-vh.w, a.y, exf));
            eyf = fmaf(vh.z, a.y, fmaf(vh.w, a.x, eyf));
        };
        for (int l0 = 0; l0 < j; l0 += 32) {
            const int l1 = l0 + 32 < j ? l0 + 32 : j;
            int l = l0;
            for (; l + 4 <= l1; l += 4) {
                float4 vh[4], vl[4];
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    vh[u] = hp[(long long)(l + u) * ld4];
                    vl[u] = lp[(long long)(l + u) * ld4];
                }
#pragma unroll
                for (int u = 0; u < 4; u++) acc(vh[u], vl[u], bq[l + u], aq[l + u]);
            }
            for (; l < l1; l++) acc(hp[(long long)l * ld4], lp[(long long)l * ld4], bq[l], aq[l]);
            ax += (double)axh + (double)axl; ay += (double)ayh + (double)ayl;
            bx += (double)bxh + (double)bxl; by += (double)byh + (double)byl;
            cx += (double)cxf; cy += (double)cyf; ex += (double)exf; ey += (double)eyf;
            axh = axl = ayh = ayl = bxh = bxl = byh = byl = 0.f;
            cxf = cyf = exf = eyf = 0.f;
        }
        auto finish = [&](long long k, double sbx, double sby, double sax, double say) {
            double2 v = Vj[k];
            float2 hi;
            if (corr) {
                v = make_double2((v.x - sax) * is, (v.y - say) * is);
                Vj[k] = v;
                Dj[k] = v.x - v.y;
                hi = make_float2((float)v.x, (float)v.y);
                Vjh[k] = hi;
                Vjl[k] = make_float2((float)(v.x - (double)hi.x), (float)(v.y - (double)hi.y));
            } else {
                hi = Vjh[k];
            }
            vm = fmaxf(vm, fmaxf(fabsf(hi.x), fabsf(hi.y)));
            double2 x = w[k];
            x.x -= sbx + (v.x * hj.x - v.y * hj.y);
            x.y -= sby + (v.x * hj.y + v.y * hj.x);
            w[k] = x;
            return fma(x.x, x.x, x.y * x.y);
        };
        nrm = finish(i, ax, ay, cx, cy);
        if (two) nrm += finish(i + 1, bx, by, ex, ey);
    }
    for (int o = 16; o > 0; o >>= 1) vm = fmaxf(vm, __shfl_xor_sync(0xffffffffu, vm, o));
    if ((threadIdx.x & 31) == 0) redm[threadIdx.x >> 5] = vm;
    block_sum_store(nrm, red, part_norm + (long long)r * gridDim.x + blockIdx.x);   // syncs before its sum
    if (threadIdx.x == 0) {
        for (int q = 1; q < (int)(blockDim.x >> 5); q++) vm = fmaxf(vm, redm[q]);
        atomicMax(vmax + (long long)r * B.ldp + j, __float_as_uint(vm));
    }
}

// End of a cycle: the triangular factor of every RHS's Hessenberg matrix, column k < kcols[r]
// per thread: rotations 0..k-1 applied in order to the stored column, then rotation k to its
// last two entries (x, h_{k+1,k}), leaving R(0:k, k) in place.
__global__ void k_orotate(OuterBatch B, double2 *__restrict__ H, const double *__restrict__ cs,
                          const double2 *__restrict__ sn, const int *__restrict__ kcols) {
    const int r = blockIdx.y, k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= kcols[r]) return;
    const int R = B.R;
    double2 *col = H + (long long)r * (R + 1) * R + (long long)k * (R + 1);
    cs += (long long)r * R; sn += (long long)r * R;
    double2 x = col[0];
    for (int l = 0; l <= k; l++) {
        const double2 y = col[l + 1], sv = sn[l];
        const double c = cs[l];
        const double2 a = cmul<double>(sv, y);
        const double2 bq = cmul<double>(make_double2(sv.x, -sv.y), x);
        col[l] = make_double2(c * x.x + a.x, c * x.y + a.y);
        x = make_double2(c * y.x - bq.x, c * y.y - bq.y);
    }
}

// V_{r,j+1} = w_r / hn_r, its FP32 copy out32 and Re - Im into outD (each if not null)
// (and, if out32L is not null, the FP32 remainder v - fl32(v) of the double-FP32 first pass)
__global__ void k_oscale(OuterBatch B, double2 *__restrict__ out, float2 *__restrict__ out32,
                         float2 *__restrict__ out32L, double *__restrict__ outD, const double2 *__restrict__ w,
                         const double *__restrict__ hn) {
    const int r = blockIdx.y;
    if (B.active && !B.active[r]) return;
    const double h = hn[r];
    if (!(h > 0.0)) return;
    out += r * B.n; w += r * B.n;
    if (out32) out32 += r * B.n32;
    if (out32L) out32L += r * B.n32;
    if (outD) outD += r * B.n;
    const double inv = 1.0 / h;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < B.n; i += (long long)gridDim.x * blockDim.x) {
        const double2 v = make_double2(w[i].x * inv, w[i].y * inv);
        out[i] = v;
        const float2 hi = make_float2((float)v.x, (float)v.y);
        if (out32) out32[i] = hi;
        if (out32L) out32L[i] = make_float2((float)(v.x - (double)hi.x), (float)(v.y - (double)hi.y));
        if (outD) outD[i] = v.x - v.y;
    }
}

// y_r = H_r(0:k_r,0:k_r)⁻¹ g_r by column-oriented back substitution (one CTA per RHS).
__global__ void k_otrisolve(OuterBatch B, const double2 *__restrict__ H, const double2 *__restrict__ g,
                            const int *__restrict__ kcols, double2 *__restrict__ y) {
    extern __shared__ double2 rhs[];
    const int r = blockIdx.x;
    const int k = kcols[r];
    if (k <= 0) return;
    const long long ldh = B.R + 1;
    H += (long long)r * (B.R + 1) * B.R; g += (long long)r * (B.R + 1); y += (long long)r * B.ldp;
    for (int i = threadIdx.x; i < k; i += blockDim.x) rhs[i] = g[i];
    __syncthreads();
    for (int i = k - 1; i >= 0; i--) {
        const double2 d = H[(long long)i * ldh + i];
        const double2 si = rhs[i];
        const double den = d.x * d.x + d.y * d.y;
        const double2 yi = make_double2((si.x * d.x + si.y * d.y) / den, (si.y * d.x - si.x * d.y) / den);
        __syncthreads();
        for (int q = threadIdx.x; q < i; q += blockDim.x) caxpy_neg<double>(rhs[q], yi, H[(long long)i * ldh + q]);
        if (threadIdx.x == 0) y[i] = yi;
        __syncthreads();
    }
}

// x_r += Σ_{l<k_r} y_{r,l} Z_{r,l}
__global__ void k_oaxpy(OuterBatch B, const double2 *__restrict__ y, const int *__restrict__ kcols,
                        const double2 *__restrict__ Zb, double2 *__restrict__ x) {
    extern __shared__ double2 ys[];
    const int r = blockIdx.y;
    const int k = kcols[r];
    if (k <= 0) return;
    y += (long long)r * B.ldp; Zb += r * B.n; x += r * B.n;
    for (int l = threadIdx.x; l < k; l += blockDim.x) ys[l] = y[l];
    __syncthreads();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < B.n; i += (long long)gridDim.x * blockDim.x) {
        double2 acc = x[i];
        for (int l = 0; l < k; l++) caxpy<double>(acc, ys[l], Zb[(long long)l * B.ld + i]);
        x[i] = acc;
    }
}

// Cycle start for every active RHS: β_r = sqrt(Σ partials), v_{r,0} = r_r/β_r,
// g_r = [β_r, 0, ..., 0] (R+1 entries); FP32 copy of v_{r,0} in V32 (if not null); row 0 of the
// (empty) rotation product, Wq_r = [1].
__global__ void k_oinit(OuterBatch B, const double2 *__restrict__ rv, const double *__restrict__ npart,
                        double2 *__restrict__ V, float2 *__restrict__ V32, float2 *__restrict__ V32L,
                        double *__restrict__ D, double2 *__restrict__ g, double2 *__restrict__ Wq,
                        double *__restrict__ beta_out) {
    __shared__ double beta_s;
    const int r = blockIdx.y;
    if (B.active && !B.active[r]) return;
    rv += r * B.n; npart += (long long)r * B.G; double2 *v0 = V + r * B.n; g += (long long)r * (B.R + 1);
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int q = 0; q < B.G; q++) s += npart[q];
        beta_s = sqrt(s);
        if (blockIdx.x == 0) beta_out[r] = beta_s;
    }
    __syncthreads();
    const double beta = beta_s;
    if (blockIdx.x == 0) {
        for (int l = threadIdx.x; l <= B.R; l += blockDim.x) g[l] = make_double2(l == 0 ? beta : 0.0, 0.0);
        if (threadIdx.x == 0) Wq[(long long)r * (B.R + 1)] = make_double2(1.0, 0.0);
    }
    if (!(beta > 0.0)) return;
    const double inv = 1.0 / beta;
    float2 *v32 = V32 ? V32 + r * B.n32 : nullptr;
    float2 *v32l = V32L ? V32L + r * B.n32 : nullptr;
    double *d0 = D ? D + r * B.n : nullptr;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < B.n; i += (long long)gridDim.x * blockDim.x) {
        const double2 v = make_double2(rv[i].x * inv, rv[i].y * inv);
        v0[i] = v;
        const float2 hi = make_float2((float)v.x, (float)v.y);
        if (v32) v32[i] = hi;
        if (v32l) v32l[i] = make_float2((float)(v.x - (double)hi.x), (float)(v.y - (double)hi.y));
        if (d0) d0[i] = v.x - v.y;
    }
}

// Deterministic dense test vector x_i = (u_{2i} - 1/2) + i (u_{2i+1} - 1/2), u_j the SplitMix64
// output mix (Steele, Lea & Flood 2014) of seed + j scaled to [0, 1); for timing runs.
__device__ __forceinline__ double mix_unit(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    z ^= z >> 31;
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}
__global__ void k_fill_test(long long n, unsigned long long seed, double2 *__restrict__ x) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        x[i] = make_double2(mix_unit(seed + 2 * (unsigned long long)i) - 0.5,
                            mix_unit(seed + 2 * (unsigned long long)i + 1) - 0.5);
}

static int grid_for(long long n, int threads) {
    long long g = (n + threads - 1) / threads;
    if (g > 8 * 152) g = 8 * 152;
    return g < 1 ? 1 : (int)g;
}

void launch_fill_test(long long n, unsigned long long seed, double2 *x, cudaStream_t s) {
    k_fill_test<<<grid_for(n, 256), 256, 0, s>>>(n, seed, x);
}
void launch_gstencil(const Stencil &st, int N, const double2 *x, double2 *y, const double2 *f, int nrhs,
                     const int *active, cudaStream_t s) {
    const long long w = st.bc ? N + 1 : N - 1, n = w * w;
    if (st.bc) k_gstencil<true><<<dim3(grid_for(n, 256), nrhs), 256, 0, s>>>(st, N, x, y, f, active);
    else k_gstencil<false><<<dim3(grid_for(n, 256), nrhs), 256, 0, s>>>(st, N, x, y, f, active);
}
void launch_build_rhs(const Stencil &st, int N, double h, int npts, const double *pts, int nb, const double *bumps,
                      double2 *f, cudaStream_t s) {
    const long long w = st.bc ? N + 1 : N - 1, n = w * w;
    k_build_rhs<<<grid_for(n, 256), 256, 0, s>>>(st, N, h, npts, pts, nb, bumps, f);
}
void launch_odots(const OuterBatch &B, const double2 *V, int nv, const double2 *w, double2 *part, cudaStream_t s) {
    k_odots<<<dim3(B.G, B.nrhs), OT, 0, s>>>(B, V, nv, w, part);
}
void launch_odots_df(const OuterBatch &B, const float2 *Vh, const float2 *Vl, int nv, const double2 *w,
                     double2 *part, cudaStream_t s) {
    k_odots_df<<<dim3(B.G, B.nrhs), OT, 0, s>>>(B, Vh, Vl, nv, w, part);
}
void launch_oupdate(const OuterBatch &B, const double2 *V, int nv, const double2 *h, double2 *w,
                    double2 *part_dots, double *part_norm, cudaStream_t s) {
    k_oupdate<<<dim3(B.G, B.nrhs), OT, (size_t)nv * 3 * sizeof(double), s>>>(B, V, nv, h, w, part_dots, part_norm);
}
// CTA size and grid of a one-element-pair-per-thread update kernel for vectors of n entries: of
// the sizes 256, 224, ..., 128 threads the one whose grid leaves the least idle in the last wave
// of resident CTAs (occupancy from the compiled register count), the largest on ties.
struct PairPlan { long long n = -1; int threads = OTU, grid = 1; };
template <typename K>
static void pair_plan(K kern, PairPlan &c, long long n, int &threads, int &grid) {
    if (n != c.n) {
        const long long P = (n + 1) / 2;
        int dev = 0, nsm = 152;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            nsm = 152;
        double best = -1.0;
        c.threads = OTU;
        c.grid = (int)((P + OTU - 1) / OTU);
        for (int t = OTU; t >= 128; t -= 32) {
            int occ = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, t, 32 * 1024) != cudaSuccess || occ < 1)
                continue;
            const long long R = (long long)occ * nsm, g = (P + t - 1) / t, waves = (g + R - 1) / R;
            const double eff = (double)P / ((double)waves * (double)R * t);
            if (eff > best + 1e-9) { best = eff; c.threads = t; c.grid = (int)(g > 0 ? g : 1); }
        }
        c.n = n;
    }
    threads = c.threads;
    grid = c.grid;
}
static PairPlan plan_udf, plan_dcgs;
int oupdate_df_grid(long long n) {
    int t = 0, g = 0;
    pair_plan(k_oupdate_df, plan_udf, n, t, g);
    return g;
}
int oupdate_dcgs_grid(long long n) {
    int t = 0, g = 0;
    pair_plan(k_oupdate_dcgs, plan_dcgs, n, t, g);
    return g;
}
void launch_oupdate_df(const OuterBatch &B, const float2 *Vh, const float2 *Vl, int nv, const double2 *h,
                       double2 *w, double *part_norm, cudaStream_t s) {
    int t = 0, g = 0;
    pair_plan(k_oupdate_df, plan_udf, B.n, t, g);
    k_oupdate_df<<<dim3(g, B.nrhs), t, (size_t)nv * sizeof(float4), s>>>(B, Vh, Vl, nv, h, w, part_norm);
}
cudaError_t launch_odots2_df(const OuterBatch &B, const float2 *Vh, const float2 *Vl, int nv, const float2 *x1h,
                             const float2 *x1l, const double2 *w, double2 *part1, double2 *part2,
                             const unsigned *vmax, int bias, cudaStream_t s) {
    const long long chunk = (B.n + B.G - 1) / B.G;
    const size_t smem = (size_t)(2 * chunk) * sizeof(float4) + (bias ? (size_t)nv * sizeof(float) : 0);
    // the largest dynamic shared memory requested so far, per device and variant (the attribute
    // is set on the current device)
    constexpr int MAXDEV = 64;
    static size_t set[MAXDEV][2];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= MAXDEV) return cudaErrorInvalidDevice;
    bias = bias ? 1 : 0;
    void (*const kern[2])(OuterBatch, const float2 *, const float2 *, int, const float2 *, const float2 *,
                          const double2 *, double2 *, double2 *, const unsigned *) = {k_odots2_df<false>,
                                                                                      k_odots2_df<true>};
    if (smem > 48 * 1024 && smem > set[dev][bias]) {
        e = cudaFuncSetAttribute(kern[bias], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        set[dev][bias] = smem;
    }
    kern[bias]<<<dim3(B.G, B.nrhs), OT, smem, s>>>(B, Vh, Vl, nv, x1h, x1l, w, part1, part2, vmax);
    return cudaSuccess;
}
void launch_dcgs_col(const OuterBatch &B, double2 *H, double *cs, double2 *sn, double2 *g, double2 *Wq, int j,
                     const double2 *P1, double2 *P2, const double *hn, double *invs, const double *fnorm,
                     double *hist, int hstride, int it, int *err, unsigned *vmax, cudaStream_t s) {
    k_dcgs_col<<<B.nrhs, OG, 0, s>>>(B, H, cs, sn, g, Wq, j, P1, P2, hn, invs, fnorm, hist, hstride, it, err, vmax);
}
void launch_dcgs_tent(const OuterBatch &B, double2 *H, double2 *g, double2 *Wq, int j, const double *npart, int gp,
                      const double *fnorm, double tol, double *hn_out, int *flag, double *hist, int hstride, int it,
                      cudaStream_t s) {
    k_dcgs_tent<<<B.nrhs, OG, 0, s>>>(B, H, g, Wq, j, npart, gp, fnorm, tol, hn_out, flag, hist, hstride, it);
}
void launch_dcgs_close(const OuterBatch &B, double2 *H, double *cs, double2 *sn, double2 *g, double2 *Wq, int j,
                       const int *close, cudaStream_t s) {
    k_dcgs_close<<<B.nrhs, OG, 0, s>>>(B, H, cs, sn, g, Wq, j, close);
}
void launch_oupdate_dcgs(const OuterBatch &B, const float2 *Vh, const float2 *Vl, int j, int corr, double2 *Vj,
                         double *Dj, float2 *Vjh, float2 *Vjl, const double2 *acoef, const double2 *bcoef,
                         const double *invs, double2 *w, double *part_norm, unsigned *vmax, cudaStream_t s) {
    int t = 0, g = 0;
    pair_plan(k_oupdate_dcgs, plan_dcgs, B.n, t, g);
    k_oupdate_dcgs<<<dim3(g, B.nrhs), t, (size_t)j * (sizeof(float4) + sizeof(float2)), s>>>(
        B, Vh, Vl, j, corr, Vj, Dj, Vjh, Vjl, acoef, bcoef, invs, w, part_norm, vmax);
}
void launch_oupdate2(const OuterBatch &B, const double2 *V, const float2 *V32, int nv, const double2 *h,
                     double2 *w, const double *npart1, int g1, double *part_norm, int allow32, int *fallbacks,
                     cudaStream_t s) {
    k_oupdate2<<<dim3(B.G, B.nrhs), OT2, (size_t)nv * sizeof(double2), s>>>(B, V, V32, nv, h, w, npart1, g1,
                                                                           part_norm, allow32, fallbacks);
}
void launch_onorm(const OuterBatch &B, const double2 *x, double *part, cudaStream_t s) {
    k_onorm<<<dim3(B.G, B.nrhs), OT, 0, s>>>(B, x, part);
}
void launch_oreduce(const OuterBatch &B, const double2 *part, int nv, double2 *out, cudaStream_t s) {
    k_oreduce<<<dim3((nv + 7) / 8, B.nrhs), 256, 0, s>>>(B, part, nv, out);
}
void launch_ogivens(const OuterBatch &B, double2 *H, double *cs, double2 *sn, double2 *g, double2 *Wq, int j,
                    const double2 *h1, const double2 *h2, const double *npart, const double *fnorm,
                    double tol, double *hn_out, int *flag, double *hist, int hstride, int it,
                    cudaStream_t s) {
    k_ogivens<<<B.nrhs, OG, 0, s>>>(B, H, cs, sn, g, Wq, j, h1, h2, npart, fnorm, tol, hn_out, flag, hist,
                                    hstride, it);
}
void launch_orotate(const OuterBatch &B, double2 *H, const double *cs, const double2 *sn, const int *kcols,
                    int kmax, cudaStream_t s) {
    k_orotate<<<dim3((kmax + 63) / 64, B.nrhs), 64, 0, s>>>(B, H, cs, sn, kcols);
}
void launch_oscale(const OuterBatch &B, double2 *out, float2 *out32, float2 *out32L, double *outD,
                   const double2 *w, const double *hn, cudaStream_t s) {
    k_oscale<<<dim3(grid_for(B.n, 256), B.nrhs), 256, 0, s>>>(B, out, out32, out32L, outD, w, hn);
}
void launch_otrisolve(const OuterBatch &B, const double2 *H, const double2 *g, const int *kcols, int kmax,
                      double2 *y, cudaStream_t s) {
    k_otrisolve<<<B.nrhs, 256, (size_t)kmax * sizeof(double2), s>>>(B, H, g, kcols, y);
}
void launch_oaxpy(const OuterBatch &B, const double2 *y, const int *kcols, int kmax, const double2 *Zb,
                  double2 *x, cudaStream_t s) {
    k_oaxpy<<<dim3(grid_for(B.n, 256), B.nrhs), 256, (size_t)kmax * sizeof(double2), s>>>(B, y, kcols, Zb, x);
}
void launch_oinit(const OuterBatch &B, const double2 *rv, const double *npart, double2 *V, float2 *V32,
                  float2 *V32L, double *D, double2 *g, double2 *Wq, double *beta_out, cudaStream_t s) {
    k_oinit<<<dim3(grid_for(B.n, 256), B.nrhs), 256, 0, s>>>(B, rv, npart, V, V32, V32L, D, g, Wq, beta_out);
}
cudaError_t set_outer_smem_limits(size_t bytes) {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_oupdate, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_oupdate2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_oupdate_df, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_oupdate_dcgs, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_otrisolve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_oaxpy, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes)) != cudaSuccess) return e;
    return cudaSuccess;
}

}  // namespace hdd
