// kernels_coarse.cu — FP64 coarse-space kernels of the two-level deflation (Eq. 4): assembly of
// E = Zᵀ A Z on the device, banded LU with partial pivoting, and the batched banded solve
// E⁻¹ y for every task (real factor, real and imaginary parts as two chains).
// The same factor/solve serves the direct local solve A_j⁻¹ (§3.1 benchmark).
#include <algorithm>

#include "hdd_common.cuh"

namespace hdd {

__device__ __forceinline__ double zwd(int t) {
    return t == 0 || t == 4 ? 0.125 : (t == 2 ? 0.75 : 0.5);
}
// 1D weight of fine node f in coarse column c (0-based), zero outside the Bézier support
__device__ __forceinline__ double z1(int f, int c) {
    int t = f - 2 * c + 1;
    return (t >= 0 && t <= 4) ? zwd(t) : 0.0;
}

// Stencil coefficient coupling fine node (x,y) to (x+dx, y+dy); 0 if not a stencil neighbour.
__device__ __forceinline__ double acoef(const Stencil &st, int dx, int dy) {
    if (dx == 0 && dy == 0) return st.c0;
    if ((dx == 0 && (dy == 1 || dy == -1)) || (dy == 0 && (dx == 1 || dx == -1))) return st.c1;
    if (st.diag == 0 && ((dx == 1 && dy == 1) || (dx == -1 && dy == -1))) return st.c2;
    if (st.diag == 1 && ((dx == 1 && dy == -1) || (dx == -1 && dy == 1))) return st.c2;
    return 0.0;
}

// E[c][c'] = Σ_f Z[f,c] Σ_{f'} A[f,f'] Z[f',c'] for the box nx x ny, written into row-band
// storage (row r, column c at ab[r·W + c - r + kl], W = 2kl+ku+1); entries outside the 5x5
// coarse neighbourhood are zero and were cleared by the caller.
__global__ void k_assemble_E(Stencil st, int nx, int ny, int kl, int ku, double *__restrict__ ab) {
    const int mx = nx / 2, my = ny / 2, m = mx * my;
    const int W = 2 * kl + ku + 1;
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= (long long)m * 25) return;
    const int c = (int)(idx / 25), d = (int)(idx % 25);
    const int cx = c % mx, cy = c / mx;
    const int ex = cx + d % 5 - 2, ey = cy + d / 5 - 2;
    if (ex < 0 || ex >= mx || ey < 0 || ey >= my) return;
    double acc = 0.0;
    for (int fy = 2 * cy - 1; fy <= 2 * cy + 3; fy++) {
        if (fy < 0 || fy >= ny) continue;
        const double wy = z1(fy, cy);
        for (int fx = 2 * cx - 1; fx <= 2 * cx + 3; fx++) {
            if (fx < 0 || fx >= nx) continue;
            const double wf = wy * z1(fx, cx);
            double inner = 0.0;
            for (int dy = -1; dy <= 1; dy++)
                for (int dx = -1; dx <= 1; dx++) {
                    const int gx = fx + dx, gy = fy + dy;
                    if (gx < 0 || gx >= nx || gy < 0 || gy >= ny) continue;
                    const double a = acoef(st, dx, dy);
                    if (a == 0.0) continue;
                    inner += a * z1(gx, ex) * z1(gy, ey);
                }
            acc += wf * inner;
        }
    }
    const int e = ex + ey * mx;
    ab[(long long)c * W + (e - c + kl)] = acc;
}

// A_j itself in row-band storage (kl = ku = nx + 1).
__global__ void k_assemble_Aloc(Stencil st, int nx, int ny, int kl, int ku, double *__restrict__ ab) {
    const int n = nx * ny, W = 2 * kl + ku + 1;
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= (long long)n * 9) return;
    const int r = (int)(idx / 9), d = (int)(idx % 9);
    const int x = r % nx, y = r / nx, dx = d % 3 - 1, dy = d / 3 - 1;
    const int gx = x + dx, gy = y + dy;
    if (gx < 0 || gx >= nx || gy < 0 || gy >= ny) return;
    const double a = acoef(st, dx, dy);
    if (a == 0.0) return;
    const int c = gx + gy * nx;
    ab[(long long)r * W + (c - r + kl)] = a;
}

// Coefficient of A coupling mesh node (gx, gy) to (gx+dx, gy+dy): the interior stencil, or under
// the impedance condition the complex row of a boundary node's class.
__device__ __forceinline__ double2 acoef_z(const Stencil &st, int gx, int gy, int dx, int dy) {
    const int cls = st.bc ? node_class(st.N, gx, gy) : 4;
    if (cls == 4) return make_double2(acoef(st, dx, dy), 0.0);
    const int q = stencil_slot(st.diag, dx, dy);
    return q < 0 ? make_double2(0.0, 0.0) : st.bcoef[cls * 7 + q];
}

// Complex value v at (row r, column c) of a complex band matrix, written as its real equivalent:
// rows/columns 2r, 2r+1 (2c, 2c+1) carry the real and imaginary parts, block [Re v, -Im v;
// Im v, Re v], in row-band storage of half-bandwidth kl2 and row width W.
__device__ __forceinline__ void put_re2(double *ab, int W, int kl2, long long r, long long c, double2 v) {
    const long long r0 = 2 * r, r1 = r0 + 1, c0 = 2 * c, c1 = c0 + 1;
    ab[r0 * W + (c0 - r0 + kl2)] = v.x;
    ab[r0 * W + (c1 - r0 + kl2)] = -v.y;
    ab[r1 * W + (c0 - r1 + kl2)] = v.y;
    ab[r1 * W + (c1 - r1 + kl2)] = v.x;
}

// E = Zᵀ A Z of the box nx x ny with origin (gx0, gy0) (impedance condition: complex), as its
// real equivalent of order 2m with kl2 = ku2 = 2·(2mx+2)+1; entries outside the 5x5 coarse
// neighbourhood are zero and were cleared by the caller.
__global__ void k_assemble_E_re2(Stencil st, int nx, int ny, int gx0, int gy0, int kl2, int ku2,
                                 double *__restrict__ ab) {
    const int mx = nx / 2, my = ny / 2, m = mx * my;
    const int W = 2 * kl2 + ku2 + 1;
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= (long long)m * 25) return;
    const int c = (int)(idx / 25), d = (int)(idx % 25);
    const int cx = c % mx, cy = c / mx;
    const int ex = cx + d % 5 - 2, ey = cy + d / 5 - 2;
    if (ex < 0 || ex >= mx || ey < 0 || ey >= my) return;
    double ar = 0.0, ai = 0.0;
    for (int fy = 2 * cy - 1; fy <= 2 * cy + 3; fy++) {
        if (fy < 0 || fy >= ny) continue;
        const double wy = z1(fy, cy);
        for (int fx = 2 * cx - 1; fx <= 2 * cx + 3; fx++) {
            if (fx < 0 || fx >= nx) continue;
            const double wf = wy * z1(fx, cx);
            double ir = 0.0, ii = 0.0;
            for (int dy = -1; dy <= 1; dy++)
                for (int dx = -1; dx <= 1; dx++) {
                    const int gx = fx + dx, gy = fy + dy;
                    if (gx < 0 || gx >= nx || gy < 0 || gy >= ny) continue;
                    const double2 a = acoef_z(st, gx0 + fx, gy0 + fy, dx, dy);
                    if (a.x == 0.0 && a.y == 0.0) continue;
                    const double z = z1(gx, ex) * z1(gy, ey);
                    ir += a.x * z;
                    ii += a.y * z;
                }
            ar += wf * ir;
            ai += wf * ii;
        }
    }
    put_re2(ab, W, kl2, c, ex + ey * mx, make_double2(ar, ai));
}

// A_j of the box with origin (gx0, gy0) (impedance condition) as its real equivalent of order
// 2n, kl2 = ku2 = 2·(nx+1)+1.
__global__ void k_assemble_Aloc_re2(Stencil st, int nx, int ny, int gx0, int gy0, int kl2, int ku2,
                                    double *__restrict__ ab) {
    const int n = nx * ny, W = 2 * kl2 + ku2 + 1;
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= (long long)n * 9) return;
    const int r = (int)(idx / 9), d = (int)(idx % 9);
    const int x = r % nx, y = r / nx, dx = d % 3 - 1, dy = d / 3 - 1;
    const int gx = x + dx, gy = y + dy;
    if (gx < 0 || gx >= nx || gy < 0 || gy >= ny) return;
    const double2 a = acoef_z(st, gx0 + x, gy0 + y, dx, dy);
    if (a.x == 0.0 && a.y == 0.0) return;
    put_re2(ab, W, kl2, r, gx + gy * nx, a);
}

// Banded LU with partial pivoting of one matrix per CTA (row-band storage, in place).  The
// pivot is the first row of largest magnitude (ties → lowest index), as in textbook Gaussian
// elimination; the interchanges widen U to kl+ku superdiagonals.  info[b] = j+1 if column j
// had no non-zero pivot candidate (or a non-finite one), else 0.
__global__ void __launch_bounds__(512)
k_band_lu(const int *__restrict__ mv, const int *__restrict__ klv, const int *__restrict__ kuv,
          double *const *__restrict__ abv, int *const *__restrict__ pivv, int *__restrict__ info) {
    __shared__ double rv[512];
    __shared__ int ri[512];
    __shared__ int piv_s;
    __shared__ double inv_s;
    const int b = blockIdx.x;
    const int m = mv[b], kl = klv[b], ku = kuv[b];
    const int W = 2 * kl + ku + 1;
    double *ab = abv[b];
    int *piv = pivv[b];
    if (threadIdx.x == 0) info[b] = 0;
#define ABX(r, c) ab[(long long)(r) * W + ((c) - (r) + kl)]
    for (int j = 0; j < m; j++) {
        const int rlast = min(j + kl, m - 1), clast = min(j + kl + ku, m - 1);
        // pivot search
        double best = -1.0;
        int bi = 0x7fffffff;
        for (int r = j + (int)threadIdx.x; r <= rlast; r += blockDim.x) {
            double v = fabs(ABX(r, j));
            if (v > best || (v == best && r < bi)) { best = v; bi = r; }
        }
        rv[threadIdx.x] = best; ri[threadIdx.x] = bi;
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if ((int)threadIdx.x < o) {
                double v2 = rv[threadIdx.x + o]; int i2 = ri[threadIdx.x + o];
                if (v2 > rv[threadIdx.x] || (v2 == rv[threadIdx.x] && i2 < ri[threadIdx.x])) {
                    rv[threadIdx.x] = v2; ri[threadIdx.x] = i2;
                }
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            piv_s = ri[0];
            piv[j] = ri[0];
            if (!(rv[0] > 0.0) || !isfinite(rv[0])) info[b] = j + 1;
        }
        __syncthreads();
        if (info[b] != 0) return;
        const int p = piv_s;
        if (p != j)
            for (int c = j + (int)threadIdx.x; c <= clast; c += blockDim.x) {
                double t = ABX(j, c); ABX(j, c) = ABX(p, c); ABX(p, c) = t;
            }
        __syncthreads();
        if (threadIdx.x == 0) inv_s = ABX(j, j);
        __syncthreads();
        const double piv_v = inv_s;
        for (int r = j + 1 + (int)threadIdx.x; r <= rlast; r += blockDim.x) ABX(r, j) = ABX(r, j) / piv_v;
        __syncthreads();
        const int nr = rlast - j, nc = clast - j;
        for (int e = threadIdx.x; e < nr * nc; e += blockDim.x) {
            const int r = j + 1 + e / nc, c = j + 1 + e % nc;
            ABX(r, c) = fma(-ABX(r, j), ABX(j, c), ABX(r, c));
        }
        __syncthreads();
    }
#undef ABX
}

// ------------------------------------------------------------------------------------------
// Blocked form of the banded LU factor for the solve.
//
// The factorisation records the interchange piv[j] and the multipliers of column j at the row
// positions of step j.  Applying every later interchange to those multipliers gives the usual
// P E = L U with a fully permuted unit lower L, whose column j may then reach beyond row j+kl.
// The solve works on blocks of BNB rows: with L_JJ the diagonal block and L_J the panel of the
// WL columns to its left (U_JJ, U_J: diagonal block and the WU columns to its right),
//   y_J = L_JJ⁻¹ (Pb)_J - L_JJ⁻¹ L_J y_{J-WL..J}          (forward)
//   x_J = U_JJ⁻¹ y_J   - U_JJ⁻¹ U_J x_{J+1..J+WU}          (backward)
// so each block is one dense matrix–vector product with the precomputed operator
// M_J = [L_JJ⁻¹ | -L_JJ⁻¹ L_J] (resp. [U_JJ⁻¹ | -U_JJ⁻¹ U_J]) instead of BNB dependent rows.
// ------------------------------------------------------------------------------------------

// perm: (P b)[i] = b[perm[i]], the interchanges applied in order to the identity.
__global__ void k_perm(int m, const int *__restrict__ piv, int *__restrict__ perm) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int i = 0; i < m; i++) perm[i] = i;
    for (int j = 0; j < m; j++) {
        int p = piv[j];
        if (p != j) { int t = perm[j]; perm[j] = perm[p]; perm[p] = t; }
    }
}

// Column j of the permuted L: multipliers of step j with every later interchange applied.
// Lp[j*KLW + q] = L(j+1+q, j); lext[j] = 1 + last non-zero q.  err is set if a multiplier
// would leave the KLW window.
__global__ void k_lperm(int m, int kl, int ku, const double *__restrict__ ab, const int *__restrict__ piv,
                        int KLW, double *__restrict__ Lp, int *__restrict__ lext, int *__restrict__ err) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    const int W = 2 * kl + ku + 1;
    double *c = Lp + (long long)j * KLW;
    for (int q = 0; q < KLW; q++) {
        const int r = j + 1 + q;
        c[q] = (q < kl && r < m) ? ab[(long long)r * W + (j - r + kl)] : 0.0;
    }
    const int jmax = min(m - 1, j + KLW);
    for (int jp = j + 1; jp <= jmax; jp++) {
        const int p = piv[jp];
        if (p == jp) continue;
        const int qa = jp - j - 1, qb = p - j - 1;
        if (qb >= KLW) {
            if (c[qa] != 0.0) atomicExch(err, 1);
            c[qa] = 0.0;
            continue;
        }
        const double t = c[qa]; c[qa] = c[qb]; c[qb] = t;
    }
    int e = 0;
    for (int q = 0; q < KLW; q++) if (c[q] != 0.0) e = q + 1;
    lext[j] = e;
}

// U column extents above the diagonal (for the backward window).
__global__ void k_uext(int m, int kl, int ku, const double *__restrict__ ab, int *__restrict__ uext) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= m) return;
    const int W = 2 * kl + ku + 1;
    int e = 0;
    for (int q = 0; q < kl + ku; q++) {
        const int r = c - 1 - q;
        if (r >= 0 && ab[(long long)r * W + (c - r + kl)] != 0.0) e = q + 1;
    }
    uext[c] = e;
}

// Forward block operators: one CTA per block J, M_J row-major BNB x (BNB + w_J) at meta[J].x
// (row stride op_stride(w_J)), w_J = meta[J].y the width of block J's left panel.
__global__ void k_block_fwd(int m, int KLW, const double *__restrict__ Lp, const int4 *__restrict__ meta,
                            double *__restrict__ Mall) {
    __shared__ double Li[BNB][BNB];
    const int J = blockIdx.x, r0 = J * BNB;
    const int WL = meta[J].y, K = BNB + WL, KS = op_stride(WL);
    double *MJ = Mall + meta[J].x;
    auto Lv = [&](int r, int c) -> double {            // permuted L(r, c), r > c
        if (c < 0 || r >= m || c >= m) return 0.0;
        const int q = r - c - 1;
        return (q >= 0 && q < KLW) ? Lp[(long long)c * KLW + q] : 0.0;
    };
    // L_JJ⁻¹ column by column (unit lower triangular; rows past m are identity)
    if (threadIdx.x < BNB) {
        const int c = threadIdx.x;
        double x[BNB];
        for (int r = 0; r < BNB; r++) x[r] = (r == c) ? 1.0 : 0.0;
        for (int r = c + 1; r < BNB; r++) {
            double acc = 0.0;
            for (int k = c; k < r; k++) acc = fma(Lv(r0 + r, r0 + k), x[k], acc);
            x[r] = -acc;
        }
        for (int r = 0; r < BNB; r++) Li[r][c] = x[r];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < BNB * KS; e += blockDim.x) {
        const int r = e / KS, cc = e % KS;
        double v;
        if (cc < BNB) v = Li[r][cc];
        else if (cc >= K) v = 0.0;                         // row padding
        else {
            const int col = r0 - WL + (cc - BNB);          // global column of the panel entry
            double acc = 0.0;
            for (int k = 0; k <= r; k++) acc = fma(Li[r][k], Lv(r0 + k, col), acc);
            v = -acc;
        }
        MJ[e] = (r0 + r < m) ? v : 0.0;
    }
}

// Backward block operators from the row-band U: M_J = [U_JJ⁻¹ | -U_JJ⁻¹ U_J], BNB x (BNB + w_J)
// at meta[J].z (row stride op_stride(w_J)) with w_J = meta[J].w.
__global__ void k_block_bwd(int m, int kl, int ku, const double *__restrict__ ab,
                            const int4 *__restrict__ meta, double *__restrict__ Mall) {
    __shared__ double Ui[BNB][BNB];
    const int J = blockIdx.x, r0 = J * BNB;
    const int WU = meta[J].w, K = BNB + WU, KS = op_stride(WU);
    const int W = 2 * kl + ku + 1;
    double *MJ = Mall + meta[J].z;
    auto Uv = [&](int r, int c) -> double {            // U(r, c), c >= r
        if (r >= m || c >= m || c < r || c - r > kl + ku) return 0.0;
        return ab[(long long)r * W + (c - r + kl)];
    };
    if (threadIdx.x < BNB) {
        const int c = threadIdx.x;
        double x[BNB];
        for (int r = 0; r < BNB; r++) x[r] = 0.0;
        if (r0 + c < m) {
            for (int r = c; r >= 0; r--) {
                double acc = (r == c) ? 1.0 : 0.0;
                for (int k = r + 1; k <= c; k++) acc = fma(-Uv(r0 + r, r0 + k), x[k], acc);
                x[r] = acc / Uv(r0 + r, r0 + r);
            }
        }
        for (int r = 0; r < BNB; r++) Ui[r][c] = x[r];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < BNB * KS; e += blockDim.x) {
        const int r = e / KS, cc = e % KS;
        double v;
        if (cc < BNB) v = Ui[r][cc];
        else if (cc >= K) v = 0.0;                         // row padding
        else {
            const int col = r0 + BNB + (cc - BNB);
            double acc = 0.0;
            for (int k = r; k < BNB; k++) acc = fma(Ui[r][k], Uv(r0 + k, col), acc);
            v = -acc;
        }
        MJ[e] = (r0 + r < m) ? v : 0.0;
    }
}

__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gsrc) {
    unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

constexpr int BS_T = 128;                 // threads: BNB rows x (BS_T/BNB) lanes per row
constexpr int BS_LPR = BS_T / BNB;        // lanes per row (8)

// y = M_J [a ; window] for the BNB rows of block J: lane `part` of row r sums the columns
// part, part + BS_LPR, ... of the row with four independent accumulators (operands loaded
// ahead of the FMAs), then the row's lanes reduce by shuffles.  The window is read from a
// circular buffer: column c of the panel is win[(base + c) & mask].
__device__ __forceinline__ double block_row_dot(const double *__restrict__ Mrow, int K,
                                                const double *__restrict__ a,
                                                const double *__restrict__ win, int base, int mask,
                                                int part) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
#pragma unroll
    for (int c = part; c < BNB; c += 2 * BS_LPR) {
        s0 = fma(Mrow[c], a[c], s0);
        if (c + BS_LPR < BNB) s1 = fma(Mrow[c + BS_LPR], a[c + BS_LPR], s1);
    }
    const int WL = K - BNB;
    int c = part;
    for (; c + 3 * BS_LPR < WL; c += 4 * BS_LPR) {
        const double m0 = Mrow[BNB + c], m1 = Mrow[BNB + c + BS_LPR];
        const double m2 = Mrow[BNB + c + 2 * BS_LPR], m3 = Mrow[BNB + c + 3 * BS_LPR];
        const double w0 = win[(base + c) & mask], w1 = win[(base + c + BS_LPR) & mask];
        const double w2 = win[(base + c + 2 * BS_LPR) & mask], w3 = win[(base + c + 3 * BS_LPR) & mask];
        s0 = fma(m0, w0, s0); s1 = fma(m1, w1, s1); s2 = fma(m2, w2, s2); s3 = fma(m3, w3, s3);
    }
    for (; c < WL; c += BS_LPR) s0 = fma(Mrow[BNB + c], win[(base + c) & mask], s0);
    s0 = (s0 + s1) + (s2 + s3);
#pragma unroll
    for (int o = BS_LPR / 2; o > 0; o >>= 1) s0 += __shfl_xor_sync(0xffffffffu, s0, o);
    return s0;
}

template <int N> __device__ __forceinline__ void cp_async_wait_n() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
// 8-byte asynchronous copy; src_size 0 fills the destination with zeros without reading.
__device__ __forceinline__ void cp_async8_zfill(void *smem_dst, const void *gsrc, int src_size) {
    unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(gsrc), "r"(src_size) : "memory");
}

// x = F⁻¹ b with the blocked operators, one CTA per (task, component); with RE2 the factor is that
// of a real-equivalent system and one CTA per task solves the complex vector read as doubles.  Shared memory holds only
// a ring of RING slots — the operator of one block plus that block's BNB input values, streamed
// by cp.async RING-1 blocks ahead of the block being applied — and two circular windows (cwy,
// cwx entries, powers of two >= BNB + panel width) of the latest y and x values; so the order of
// the factor is not limited by shared memory.  The output vector carries the rest: it first
// receives P b (gathered), the forward sweep overwrites block J with y_J after reading it, and the
// backward sweep overwrites block J with x_J after reading y_J.  One barrier per block.
template <int RING, bool RE2>
__global__ void __launch_bounds__(BS_T, 2)
k_block_solve(const Task *__restrict__ tasks, const BlockFactor *__restrict__ shapes,
              const double *__restrict__ Mall, const int *__restrict__ Pall,
              const int4 *__restrict__ Meta, const double2 *__restrict__ in,
              double2 *__restrict__ out, int use_fine, const int *__restrict__ flag, int maxK,
              int cwy, int cwx) {
    extern __shared__ double sm[];
    constexpr int STR = RE2 ? 1 : 2;        // stride (doubles) of the solved real column
    const int t = RE2 ? (int)blockIdx.x : (int)(blockIdx.x >> 1), comp = RE2 ? 0 : (int)(blockIdx.x & 1);
    if (flag && !flag[t]) return;
    const Task T = tasks[t];
    const BlockFactor F = shapes[T.shape];
    const long long off = use_fine ? T.foff : T.coff;
    const int m = F.m, nbk = F.nblk;
    const int slot = BNB * maxK + BNB;
    double *CY = sm + RING * slot, *CX = CY + cwy;
    const int *perm = Pall + F.perm_off;
    const int4 *meta = Meta + F.meta_off;
    const double *inr = reinterpret_cast<const double *>(in + off) + comp;
    double *outr = reinterpret_cast<double *>(out + off) + comp;
    const int tid = threadIdx.x, row = tid / BS_LPR, part = tid % BS_LPR;
    // operator of block J (src_off, K = BNB + panel) and its BNB inputs from outr into slot buf
    auto load_block = [&](long long src_off, int K, int buf, int J) {
        double *dst = sm + buf * slot;
        const double *src = Mall + src_off;
        const int nchunk = BNB * K / 2;                 // 16-byte chunks
        for (int q = tid; q < nchunk; q += BS_T) cp_async16(dst + 2 * q, src + 2 * q);
        if (tid < BNB) {
            const int i = J * BNB + tid;
            cp_async8_zfill(dst + BNB * maxK + tid, i < m ? outr + STR * (long long)i : outr, i < m ? 8 : 0);
        }
    };
    // (P b) into the output; zero windows (positions before 0 / after the end read zeros)
    for (int i = tid; i < m; i += BS_T) outr[STR * (long long)i] = inr[STR * (long long)perm[i]];
    for (int i = tid; i < cwy; i += BS_T) CY[i] = 0.0;
    for (int i = tid; i < cwx; i += BS_T) CX[i] = 0.0;
    __threadfence_block();
    __syncthreads();
    // Block descriptors (operator offsets and panel widths) are global; the one a step prefetches
    // is loaded a step ahead (mnext), and the prefetching thread stores the panel width of each
    // slot in sw[], so no global load sits on a step's dependent path.
    __shared__ int sw[RING];
    // ---- forward: y_J = M_J [(Pb)_J ; y_{J-w_J..J}] ----
#pragma unroll
    for (int u = 0; u < RING - 1; u++) {
        if (u < nbk) {
            const int4 mt = meta[u];
            load_block(mt.x, op_stride(mt.y), u, u);
            if (tid == 0) sw[u] = mt.y;
        }
        cp_async_commit();
    }
    int4 mnext = RING - 1 < nbk ? meta[RING - 1] : make_int4(0, 0, 0, 0);
    for (int J = 0; J < nbk; J++) {
        cp_async_wait_n<RING - 2>();
        __syncthreads();
        if (J + RING - 1 < nbk) {
            const int buf = (J + RING - 1) % RING;
            load_block(mnext.x, op_stride(mnext.y), buf, J + RING - 1);
            if (tid == 0) sw[buf] = mnext.y;
        }
        cp_async_commit();
        if (J + RING < nbk) mnext = meta[J + RING];
        const int wJ = sw[J % RING];
        const double *Mb = sm + (J % RING) * slot;
        const double v = block_row_dot(Mb + row * op_stride(wJ), BNB + wJ, Mb + BNB * maxK, CY, J * BNB - wJ,
                                       cwy - 1, part);
        if (part == 0) {
            const int i = J * BNB + row;
            CY[i & (cwy - 1)] = v;
            if (i < m) outr[STR * (long long)i] = v;
        }
    }
    cp_async_wait_n<0>();
    __threadfence_block();
    __syncthreads();
    // ---- backward: x_J = M_J [y_J ; x_{J+1..J+w_J}] ----
#pragma unroll
    for (int u = 0; u < RING - 1; u++) {
        const int J = nbk - 1 - u;
        if (J >= 0) {
            const int4 mt = meta[J];
            load_block(mt.z, op_stride(mt.w), u, J);
            if (tid == 0) sw[u] = mt.w;
        }
        cp_async_commit();
    }
    mnext = nbk - RING >= 0 ? meta[nbk - RING] : make_int4(0, 0, 0, 0);
    for (int J = nbk - 1; J >= 0; J--) {
        const int k = nbk - 1 - J;                          // sweep position
        cp_async_wait_n<RING - 2>();
        __syncthreads();
        if (J - (RING - 1) >= 0) {
            const int buf = (k + RING - 1) % RING;
            load_block(mnext.z, op_stride(mnext.w), buf, J - (RING - 1));
            if (tid == 0) sw[buf] = mnext.w;
        }
        cp_async_commit();
        if (J - RING >= 0) mnext = meta[J - RING];
        const int wJ = sw[k % RING];
        const double *Mb = sm + (k % RING) * slot;
        const double v = block_row_dot(Mb + row * op_stride(wJ), BNB + wJ, Mb + BNB * maxK, CX, (J + 1) * BNB,
                                       cwx - 1, part);
        if (part == 0) {
            const int i = J * BNB + row;
            CX[i & (cwx - 1)] = v;
            if (i < m) outr[STR * (long long)i] = v;
        }
    }
    cp_async_wait_n<0>();
}

// ------------------------------------------------------------------------------------------
// Look-ahead form of the blocked solve.  In block J's product y_J = M_J [(Pb)_J ; panel] only the
// panel columns of the previous block (y_{J-1}; backward: x_{J+1}) depend on the step just
// finished; the diagonal part and the older panel columns are known one block earlier.  So while
// warp 0 finishes block J (its recent columns plus the partial sums below: at most 16 columns
// per row), the other LA_BW warps already sum the diagonal and older columns of block J+1 into
// per-warp partials.  The dependent chain per block shrinks to one 16-column product and a
// barrier, and the bulk of the FP64 work of consecutive blocks overlaps.  Same operators, ring
// and windows as k_block_solve; the sums are taken in a fixed order (deterministic).
// ------------------------------------------------------------------------------------------
__host__ __device__ __forceinline__ int la_slot(int maxK) { return BNB * maxK + BNB; }
constexpr int LA_T = 256;                 // threads: warp 0 (chain) + LA_BW bulk warps
constexpr int LA_BW = LA_T / 32 - 1;      // bulk warps (7)
constexpr int LA_BL = 2 * LA_BW;          // bulk lanes per row (14): (warp, half)

template <int RING, bool RE2>
__global__ void __launch_bounds__(LA_T, 2)
k_block_solve_la(const Task *__restrict__ tasks, const BlockFactor *__restrict__ shapes,
                 const double *__restrict__ Mall, const int *__restrict__ Pall,
                 const int4 *__restrict__ Meta, const double2 *__restrict__ in,
                 double2 *__restrict__ out, int use_fine, const int *__restrict__ flag, int maxK,
                 int cwy, int cwx) {
    static_assert(RING >= 3, "the look-ahead needs blocks J and J+1 resident while J+2 loads");
    static_assert(LA_BW == 7, "chain_row adds the seven bulk partials in four accumulators");
    extern __shared__ double sm[];
    __shared__ double part[2][LA_BW][BNB];   // bulk partial sums of the next block, by parity
    __shared__ int sw[RING];                  // panel width of the block in each ring slot
    constexpr int STR = RE2 ? 1 : 2;
    const int t = RE2 ? (int)blockIdx.x : (int)(blockIdx.x >> 1), comp = RE2 ? 0 : (int)(blockIdx.x & 1);
    if (flag && !flag[t]) return;
    const Task T = tasks[t];
    const BlockFactor F = shapes[T.shape];
    const long long off = use_fine ? T.foff : T.coff;
    const int m = F.m, nbk = F.nblk;
    const int slot = la_slot(maxK);
    double *CY = sm + RING * slot, *CX = CY + cwy;
    const int *perm = Pall + F.perm_off;
    const int4 *meta = Meta + F.meta_off;
    const double *inr = reinterpret_cast<const double *>(in + off) + comp;
    double *outr = reinterpret_cast<double *>(out + off) + comp;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int row = lane >> 1, half = lane & 1;          // 16 rows x 2 lanes per warp
    const int q = (warp - 1) * 2 + half;                 // bulk lane of the row (warp >= 1)
    // copies are issued by the bulk warps only (warp 0 goes straight to the dependent chain);
    // the thread of index LA_T - LA_BW·32 = 32 records each slot's panel width
    const int bt = tid - 32;                             // bulk thread index (< 0 in warp 0)
    auto load_block = [&](long long src_off, int K, int buf, int J) {
        if (bt < 0) return;
        double *dst = sm + buf * slot;
        const double *src = Mall + src_off;
        const int nchunk = BNB * K / 2;                  // 16-byte chunks
        for (int c = bt; c < nchunk; c += LA_T - 32) cp_async16(dst + 2 * c, src + 2 * c);
        if (bt < BNB) {
            const int i = J * BNB + bt;
            cp_async8_zfill(dst + BNB * maxK + bt, i < m ? outr + STR * (long long)i : outr, i < m ? 8 : 0);
        }
    };
    for (int i = tid; i < m; i += LA_T) outr[STR * (long long)i] = inr[STR * (long long)perm[i]];
    for (int i = tid; i < cwy; i += LA_T) CY[i] = 0.0;
    for (int i = tid; i < cwx; i += LA_T) CX[i] = 0.0;
    __threadfence_block();
    __syncthreads();

    // Sum over the columns [k0, k1) of block J's operator (slot Mb, row stride K) for this bulk
    // lane's row: diagonal columns k < BNB take the block's inputs, panel column p = k - BNB takes
    // win[(pbase + p) & mask].  Columns q, q + LA_BL, ... of the range; four accumulators.
    auto bulk_row = [&](const double *Mb, int K, int k0, int k1, const double *win, int pbase, int mask) {
        const double *Mr = Mb + row * K;
        const double *a = Mb + BNB * maxK;
        // one accumulator: every FP64 add here occupies the sub-partition's FP64 unit like an FMA,
        // and the bulk's FMAs are few per lane (≈ 7) and off the dependent chain of the solve, so a
        // single dependent sum beats partial sums (two: 226 µs per k=200 launch; four: 250 µs)
        double v = 0.0;
        int k = q;
        for (; k < BNB; k += LA_BL) v = fma(Mr[k], a[k], v);
        if (k < k0) k += ((k0 - k + LA_BL - 1) / LA_BL) * LA_BL;
        for (; k < k1; k += LA_BL) v = fma(Mr[k], win[(pbase + k - BNB) & mask], v);
        v += __shfl_xor_sync(0xffffffffu, v, 1);
        return v;
    };
    // Warp 0: block J from the bulk partials (parity par) and the recent panel columns [p0, p1).
    // This is the dependent chain of the solve, so its FP64 latency is kept short: the lane's
    // partials (three or four) and its products (at most eight) go round-robin into four
    // independent accumulators, combined by a two-level tree and one shuffle.
    auto chain_row = [&](const double *Mb, int K, int p0, int p1, const double *win, int pbase, int mask,
                         int par) {
        const double *Mr = Mb + row * K + BNB;
        double a0 = part[par][half][row], a1 = part[par][half + 2][row], a2 = part[par][half + 4][row];
        double a3 = half == 0 ? part[par][6][row] : 0.0;
        int p = p0 + half;
        for (; p + 6 < p1; p += 8) {
            a0 = fma(Mr[p], win[(pbase + p) & mask], a0);
            a1 = fma(Mr[p + 2], win[(pbase + p + 2) & mask], a1);
            a2 = fma(Mr[p + 4], win[(pbase + p + 4) & mask], a2);
            a3 = fma(Mr[p + 6], win[(pbase + p + 6) & mask], a3);
        }
        if (p < p1) a0 = fma(Mr[p], win[(pbase + p) & mask], a0);
        if (p + 2 < p1) a1 = fma(Mr[p + 2], win[(pbase + p + 2) & mask], a1);
        if (p + 4 < p1) a2 = fma(Mr[p + 4], win[(pbase + p + 4) & mask], a2);
        double v = (a0 + a1) + (a2 + a3);
        v += __shfl_xor_sync(0xffffffffu, v, 1);
        return v;
    };

    // ---- forward: y_J = M_J [(Pb)_J ; y_{J-w_J..J}] ----
    // metadata of the blocks three prefetches ahead, in a register queue: each global load has
    // three steps to arrive before the copy it addresses is issued
    int4 mq0 = make_int4(0, 0, 0, 0), mq1 = mq0, mq2 = mq0;
#pragma unroll
    for (int u = 0; u < RING - 1; u++) {
        if (u < nbk) {
            const int4 mt = meta[u];
            load_block(mt.x, op_stride(mt.y), u, u);
            if (tid == 32) sw[u] = mt.y;
        }
        cp_async_commit();
    }
    if (RING - 1 < nbk) mq0 = meta[RING - 1];
    if (RING < nbk) mq1 = meta[RING];
    if (RING + 1 < nbk) mq2 = meta[RING + 1];
    cp_async_wait_n<RING - 2>();                           // block 0 resident
    __syncthreads();
    if (warp > 0) {                                        // bulk part of block 0
        const int w0 = sw[0], nold = w0 > BNB ? w0 - BNB : 0;
        const double v = bulk_row(sm, op_stride(w0), BNB, BNB + nold, CY, -w0, cwy - 1);
        if (half == 0) part[0][warp - 1][row] = v;
    }
    for (int J = 0; J < nbk; J++) {
        cp_async_wait_n<RING - 3>();                       // blocks J and J+1 resident
        __syncthreads();
        if (J + RING - 1 < nbk) {                          // into the slot block J-1 used
            const int buf = (J + RING - 1) % RING;
            load_block(mq0.x, op_stride(mq0.y), buf, J + RING - 1);
            if (tid == 32) sw[buf] = mq0.y;
        }
        cp_async_commit();
        mq0 = mq1; mq1 = mq2;
        if (J + RING + 2 < nbk) mq2 = meta[J + RING + 2];
        if (warp == 0) {
            const int wJ = sw[J % RING];
            const int p0 = wJ > BNB ? wJ - BNB : 0;
            const double v = chain_row(sm + (J % RING) * slot, op_stride(wJ), p0, wJ, CY, J * BNB - wJ, cwy - 1, J & 1);
            if (half == 0) {
                const int i = J * BNB + row;
                CY[i & (cwy - 1)] = v;
                if (i < m) outr[STR * (long long)i] = v;
            }
        } else if (J + 1 < nbk) {
            const int Jn = J + 1, w1 = sw[Jn % RING], nold = w1 > BNB ? w1 - BNB : 0;
            const double v = bulk_row(sm + (Jn % RING) * slot, op_stride(w1), BNB, BNB + nold, CY, Jn * BNB - w1, cwy - 1);
            if (half == 0) part[Jn & 1][warp - 1][row] = v;
        }
    }
    cp_async_wait_n<0>();
    __threadfence_block();
    __syncthreads();

    // ---- backward: x_J = M_J [y_J ; x_{J+1..J+w_J}] ----
#pragma unroll
    for (int u = 0; u < RING - 1; u++) {
        const int J = nbk - 1 - u;
        if (J >= 0) {
            const int4 mt = meta[J];
            load_block(mt.z, op_stride(mt.w), u, J);
            if (tid == 32) sw[u] = mt.w;
        }
        cp_async_commit();
    }
    mq0 = nbk - RING >= 0 ? meta[nbk - RING] : make_int4(0, 0, 0, 0);
    mq1 = nbk - RING - 1 >= 0 ? meta[nbk - RING - 1] : make_int4(0, 0, 0, 0);
    mq2 = nbk - RING - 2 >= 0 ? meta[nbk - RING - 2] : make_int4(0, 0, 0, 0);
    cp_async_wait_n<RING - 2>();
    __syncthreads();
    if (warp > 0) {                                        // bulk part of block nbk-1
        const int J = nbk - 1, w0 = sw[0];
        const double v = bulk_row(sm, op_stride(w0), 2 * BNB, BNB + w0, CX, (J + 1) * BNB, cwx - 1);
        if (half == 0) part[0][warp - 1][row] = v;
    }
    for (int k = 0; k < nbk; k++) {                        // sweep position k: block J = nbk-1-k
        const int J = nbk - 1 - k;
        cp_async_wait_n<RING - 3>();
        __syncthreads();
        if (J - (RING - 1) >= 0) {
            const int buf = (k + RING - 1) % RING;
            load_block(mq0.z, op_stride(mq0.w), buf, J - (RING - 1));
            if (tid == 32) sw[buf] = mq0.w;
        }
        cp_async_commit();
        mq0 = mq1; mq1 = mq2;
        if (J - RING - 2 >= 0) mq2 = meta[J - RING - 2];
        if (warp == 0) {
            const int wJ = sw[k % RING];
            const double v = chain_row(sm + (k % RING) * slot, op_stride(wJ), 0, wJ < BNB ? wJ : BNB, CX, (J + 1) * BNB,
                                       cwx - 1, k & 1);
            if (half == 0) {
                const int i = J * BNB + row;
                CX[i & (cwx - 1)] = v;
                if (i < m) outr[STR * (long long)i] = v;
            }
        } else if (J - 1 >= 0) {
            const int kn = k + 1, Jn = J - 1, w1 = sw[kn % RING];
            const double v = bulk_row(sm + (kn % RING) * slot, op_stride(w1), 2 * BNB, BNB + w1, CX, (Jn + 1) * BNB,
                                      cwx - 1);
            if (half == 0) part[kn & 1][warp - 1][row] = v;
        }
    }
    cp_async_wait_n<0>();
}

// ------------------------------------------------------------------------------------------
// Double-FP32 form of the look-ahead blocked solve, for the coarse solves of the complex64 inner
// iteration.  GB300's FP64 pipe issues two FMAs per clock per SM, so k_block_solve_la is bound by
// it (the chain warp's eight FMAs per lane occupy one sub-partition's FP64 unit for ~512 cycles
// per block).  Here the same block operators, converted once to (hi, lo) FP32 pairs (Mdf, the
// offsets of Mall in 8-byte entries), are applied with df_acc on the FP32 pipe: every product
// exact in its high parts, sums by two-sum, windows, partial sums and the working vector kept as
// pairs (the input split once at the start, the result widened to FP64 once at the end: on GB300
// an FP64 conversion of a warp costs as much as an FP64 FMA, so none stays inside the sweeps).  The operators carry 2^-48 relative error instead
// of 2^-53, so the solve's forward error grows to about κ(E)·2^-48 (4e-10 at κ = 1e5), far
// below what inner solves to a relative tolerance of 1e-2 in complex64 arithmetic need; the
// complex128 inner solves and the direct local solve keep k_block_solve_la.  Schedule, ring,
// windows and shared-memory layout are those of k_block_solve_la (a pair takes the 8 bytes of a
// double).
// ------------------------------------------------------------------------------------------
// 16 warps: warp 0 runs the chain alone on its sub-partition (warps are issued by the
// sub-partition of index warp mod 4); warps 4, 8 and 12 share that sub-partition and only issue
// the block copies; the other 12 warps sum the bulk of the next block.
constexpr int LAD_T = 512;
constexpr int LAD_BW = 12;                 // bulk warps
constexpr int LAD_BL = 2 * LAD_BW;         // bulk lanes per row (24)
template <int RING, bool RE2>
__global__ void __launch_bounds__(LAD_T, 1)
k_block_solve_la_df(const Task *__restrict__ tasks, const BlockFactor *__restrict__ shapes,
                    const float2 *__restrict__ Mdf, const int *__restrict__ Pall,
                    const int4 *__restrict__ Meta, const double2 *__restrict__ in,
                    double2 *__restrict__ out, int use_fine, const int *__restrict__ flag, int maxK,
                    int cwy, int cwx) {
    static_assert(RING >= 3, "the look-ahead needs blocks J and J+1 resident while J+2 loads");
    extern __shared__ double smd[];
    __shared__ float2 part[2][LAD_BW][BNB];
    __shared__ int sw[RING];
    constexpr int STR = RE2 ? 1 : 2;
    const int t = RE2 ? (int)blockIdx.x : (int)(blockIdx.x >> 1), comp = RE2 ? 0 : (int)(blockIdx.x & 1);
    if (flag && !flag[t]) return;
    const Task T = tasks[t];
    const BlockFactor F = shapes[T.shape];
    const long long off = use_fine ? T.foff : T.coff;
    const int m = F.m, nbk = F.nblk;
    const int slot = la_slot(maxK);
    float2 *CY = reinterpret_cast<float2 *>(smd + RING * slot), *CX = CY + cwy;
    const int *perm = Pall + F.perm_off;
    const int4 *meta = Meta + F.meta_off;
    const double *inr = reinterpret_cast<const double *>(in + off) + comp;
    double *outr = reinterpret_cast<double *>(out + off) + comp;
    // during the solve every 8-byte slot of the output holds the entry as a (hi, lo) pair: the
    // inputs are split once here, the block inputs travel as pairs, the outputs are widened to
    // FP64 once at the end (no FP64-pipe conversion inside the sweeps)
    float2 *od = reinterpret_cast<float2 *>(outr);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int row = lane >> 1, half = lane & 1;
    const bool bulkw = warp > 0 && (warp & 3) != 0;
    const int wb = warp - 1 - (warp >> 2);                 // bulk warp index 0..11 (if bulkw)
    const int q = wb * 2 + half;
    const int bt = tid - 32;
    auto load_block = [&](long long src_off, int K, int buf, int J) {
        if (bt < 0) return;
        double *dst = smd + buf * slot;
        const float2 *src = Mdf + src_off;
        const int nchunk = BNB * K / 2;                  // 16-byte chunks (two pairs each)
        for (int c = bt; c < nchunk; c += LAD_T - 32) cp_async16(dst + 2 * c, src + 2 * c);
        if (bt < BNB) {
            const int i = J * BNB + bt;
            cp_async8_zfill(dst + BNB * maxK + bt, i < m ? outr + STR * (long long)i : outr, i < m ? 8 : 0);
        }
    };
    for (int i = tid; i < m; i += LAD_T) od[STR * (long long)i] = df_split(inr[STR * (long long)perm[i]]);
    for (int i = tid; i < cwy; i += LAD_T) CY[i] = make_float2(0.f, 0.f);
    for (int i = tid; i < cwx; i += LAD_T) CX[i] = make_float2(0.f, 0.f);
    __threadfence_block();
    __syncthreads();

    // columns [k0, k1) of the block in slot sp (row stride K) for this bulk lane's row: diagonal
    // columns k < BNB take the block's inputs (pairs), panel column p = k - BNB the window
    auto bulk_row = [&](const double *sp, int K, int k0, int k1, const float2 *win, int pbase, int mask) {
        const float2 *Mr = reinterpret_cast<const float2 *>(sp) + row * K;
        const float2 *a = reinterpret_cast<const float2 *>(sp + BNB * maxK);
        float sh = 0.f, sl = 0.f;
        int k = q;
        for (; k < BNB; k += LAD_BL) {
            const float2 mk = Mr[k], x = a[k];
            df_acc(sh, sl, mk.x, mk.y, x.x, x.y);
        }
        if (k < k0) k += ((k0 - k + LAD_BL - 1) / LAD_BL) * LAD_BL;
        for (; k < k1; k += LAD_BL) {
            const float2 mk = Mr[k], x = win[(pbase + k - BNB) & mask];
            df_acc(sh, sl, mk.x, mk.y, x.x, x.y);
        }
        const float oh = __shfl_xor_sync(0xffffffffu, sh, 1), ol = __shfl_xor_sync(0xffffffffu, sl, 1);
        df_add(sh, sl, oh, ol);
        return make_float2(sh, sl);
    };
    // warp 0: block J from the bulk partials (parity par) and the recent panel columns [p0, p1),
    // four pair accumulators seeded by the lane's partials, combined by a two-level tree
    auto chain_row = [&](const double *sp, int K, int p0, int p1, const float2 *win, int pbase, int mask,
                         int par) {
        const float2 *Mr = reinterpret_cast<const float2 *>(sp) + row * K + BNB;
        // lane half h seeds the four accumulators with the partials h, h + 2, ... round-robin
        float2 a0 = make_float2(0.f, 0.f), a1 = a0, a2 = a0, a3 = a0;
#pragma unroll
        for (int w = 0; 2 * w < LAD_BW; w++) {
            const int src = 2 * w + half;
            if (src >= LAD_BW) break;
            const float2 pv = part[par][src][row];
            float2 &acc = (w & 3) == 0 ? a0 : (w & 3) == 1 ? a1 : (w & 3) == 2 ? a2 : a3;
            df_add(acc.x, acc.y, pv.x, pv.y);
        }
        auto madd = [&](float2 &acc, int p) {
            const float2 mk = Mr[p], x = win[(pbase + p) & mask];
            df_acc(acc.x, acc.y, mk.x, mk.y, x.x, x.y);
        };
        int p = p0 + half;
        for (; p + 6 < p1; p += 8) { madd(a0, p); madd(a1, p + 2); madd(a2, p + 4); madd(a3, p + 6); }
        if (p < p1) madd(a0, p);
        if (p + 2 < p1) madd(a1, p + 2);
        if (p + 4 < p1) madd(a2, p + 4);
        df_add(a0.x, a0.y, a1.x, a1.y);
        df_add(a2.x, a2.y, a3.x, a3.y);
        df_add(a0.x, a0.y, a2.x, a2.y);
        const float oh = __shfl_xor_sync(0xffffffffu, a0.x, 1), ol = __shfl_xor_sync(0xffffffffu, a0.y, 1);
        df_add(a0.x, a0.y, oh, ol);
        return a0;
    };

    // ---- forward: y_J = M_J [(Pb)_J ; y_{J-w_J..J}] ----
    // metadata of the blocks three prefetches ahead, in a register queue: each global load has
    // three steps to arrive before the copy it addresses is issued
    int4 mq0 = make_int4(0, 0, 0, 0), mq1 = mq0, mq2 = mq0;
#pragma unroll
    for (int u = 0; u < RING - 1; u++) {
        if (u < nbk) {
            const int4 mt = meta[u];
            load_block(mt.x, op_stride(mt.y), u, u);
            if (tid == 32) sw[u] = mt.y;
        }
        cp_async_commit();
    }
    if (RING - 1 < nbk) mq0 = meta[RING - 1];
    if (RING < nbk) mq1 = meta[RING];
    if (RING + 1 < nbk) mq2 = meta[RING + 1];
    cp_async_wait_n<RING - 2>();
    __syncthreads();
    if (bulkw) {
        const int w0 = sw[0], nold = w0 > BNB ? w0 - BNB : 0;
        const float2 v = bulk_row(smd, op_stride(w0), BNB, BNB + nold, CY, -w0, cwy - 1);
        if (half == 0) part[0][wb][row] = v;
    }
    for (int J = 0; J < nbk; J++) {
        cp_async_wait_n<RING - 3>();
        __syncthreads();
        if (J + RING - 1 < nbk) {
            const int buf = (J + RING - 1) % RING;
            load_block(mq0.x, op_stride(mq0.y), buf, J + RING - 1);
            if (tid == 32) sw[buf] = mq0.y;
        }
        cp_async_commit();
        mq0 = mq1; mq1 = mq2;
        if (J + RING + 2 < nbk) mq2 = meta[J + RING + 2];
        if (warp == 0) {
            const int wJ = sw[J % RING];
            const int p0 = wJ > BNB ? wJ - BNB : 0;
            const float2 v = chain_row(smd + (J % RING) * slot, op_stride(wJ), p0, wJ, CY, J * BNB - wJ, cwy - 1, J & 1);
            if (half == 0) {
                const int i = J * BNB + row;
                CY[i & (cwy - 1)] = v;
                if (i < m) od[STR * (long long)i] = v;
            }
        } else if (bulkw && J + 1 < nbk) {
            const int Jn = J + 1, w1 = sw[Jn % RING], nold = w1 > BNB ? w1 - BNB : 0;
            const float2 v = bulk_row(smd + (Jn % RING) * slot, op_stride(w1), BNB, BNB + nold, CY, Jn * BNB - w1, cwy - 1);
            if (half == 0) part[Jn & 1][wb][row] = v;
        }
    }
    cp_async_wait_n<0>();
    __threadfence_block();
    __syncthreads();

    // ---- backward: x_J = M_J [y_J ; x_{J+1..J+w_J}] ----
#pragma unroll
    for (int u = 0; u < RING - 1; u++) {
        const int J = nbk - 1 - u;
        if (J >= 0) {
            const int4 mt = meta[J];
            load_block(mt.z, op_stride(mt.w), u, J);
            if (tid == 32) sw[u] = mt.w;
        }
        cp_async_commit();
    }
    mq0 = nbk - RING >= 0 ? meta[nbk - RING] : make_int4(0, 0, 0, 0);
    mq1 = nbk - RING - 1 >= 0 ? meta[nbk - RING - 1] : make_int4(0, 0, 0, 0);
    mq2 = nbk - RING - 2 >= 0 ? meta[nbk - RING - 2] : make_int4(0, 0, 0, 0);
    cp_async_wait_n<RING - 2>();
    __syncthreads();
    if (bulkw) {
        const int J = nbk - 1, w0 = sw[0];
        const float2 v = bulk_row(smd, op_stride(w0), 2 * BNB, BNB + w0, CX, (J + 1) * BNB, cwx - 1);
        if (half == 0) part[0][wb][row] = v;
    }
    for (int k = 0; k < nbk; k++) {
        const int J = nbk - 1 - k;
        cp_async_wait_n<RING - 3>();
        __syncthreads();
        if (J - (RING - 1) >= 0) {
            const int buf = (k + RING - 1) % RING;
            load_block(mq0.z, op_stride(mq0.w), buf, J - (RING - 1));
            if (tid == 32) sw[buf] = mq0.w;
        }
        cp_async_commit();
        mq0 = mq1; mq1 = mq2;
        if (J - RING - 2 >= 0) mq2 = meta[J - RING - 2];
        if (warp == 0) {
            const int wJ = sw[k % RING];
            const float2 v = chain_row(smd + (k % RING) * slot, op_stride(wJ), 0, wJ < BNB ? wJ : BNB, CX, (J + 1) * BNB,
                                       cwx - 1, k & 1);
            if (half == 0) {
                const int i = J * BNB + row;
                CX[i & (cwx - 1)] = v;
                if (i < m) od[STR * (long long)i] = v;
            }
        } else if (bulkw && J - 1 >= 0) {
            const int kn = k + 1, Jn = J - 1, w1 = sw[kn % RING];
            const float2 v = bulk_row(smd + (kn % RING) * slot, op_stride(w1), 2 * BNB, BNB + w1, CX, (Jn + 1) * BNB,
                                      cwx - 1);
            if (half == 0) part[kn & 1][wb][row] = v;
        }
    }
    cp_async_wait_n<0>();
    __syncthreads();
    for (int i = tid; i < m; i += LAD_T) {
        const float2 v = od[STR * (long long)i];
        outr[STR * (long long)i] = (double)v.x + (double)v.y;
    }
}

// ------------------------------------------------------------------------------------------
// SPIKE form of the double-FP32 look-ahead solve (SpikeInfo, hdd_common.cuh).  One cluster of P
// CTAs per chain; CTA p sweeps the blocks [B[p], B[p+1]) of both triangular solves with the
// schedule of k_block_solve_la_df (8 warps: the chain in warp 0, the next block's bulk in warps
// 1-7) and zero window values outside its part.  The parts then exchange boundary values through
// the output vector (written before a cluster barrier) and correct:
//   forward:  t_1 = g_0[tail], t_{q+1} = g_q[tail] + Gf_q[tail rows] t_q,  y_p = g_p + Gf_p t_p;
//   backward: h_{P-2} = l_{P-1}[head], h_{q-1} = l_q[head] + Gb_q[head rows] h_q,  x_p = l_p + Gb_p h_p.
// Each CTA forms the boundary chain up to its own part itself (a few small dense products), so
// the phases need four cluster barriers.  Spike matrices are column-major per part (rows of the
// part contiguous), so that threads over rows read them coalesced.  All arithmetic in pairs.
// ------------------------------------------------------------------------------------------
constexpr int SPK_T = 256;
constexpr int SPK_BW = SPK_T / 32 - 1;    // bulk warps (7)
constexpr int SPK_BL = 2 * SPK_BW;        // bulk lanes per row (14)

__device__ __forceinline__ void spk_cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
    asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

template <int RING, bool RE2>
__global__ void __launch_bounds__(SPK_T, 1)
k_block_solve_spike_df(const Task *__restrict__ tasks, const BlockFactor *__restrict__ shapes,
                       const float2 *__restrict__ Mdf, const int *__restrict__ Pall,
                       const int4 *__restrict__ Meta, const SpikeInfo *__restrict__ spikes,
                       const float2 *__restrict__ G, const double2 *__restrict__ in,
                       double2 *__restrict__ out, int use_fine, const int *__restrict__ flag,
                       const int *__restrict__ list, int maxK, int cwy, int cwx, int P) {
    static_assert(RING >= 3, "the look-ahead needs blocks J and J+1 resident while J+2 loads");
    extern __shared__ double smd[];
    __shared__ float2 part[2][SPK_BW][BNB];
    __shared__ int sw[RING];
    __shared__ float2 tb[2][SPIKE_WMAX];
    constexpr int STR = RE2 ? 1 : 2;
    // clusters over the active chains only (list: the active tasks in order, or null = every task)
    const int chain = (int)blockIdx.x / P, rank = (int)blockIdx.x % P;
    const int tl = RE2 ? chain : chain >> 1, comp = RE2 ? 0 : (chain & 1);
    const int t = list ? list[tl] : tl;
    if (t < 0) return;                               // past the compacted count (every CTA of the cluster)
    if (flag && !flag[t]) return;                    // every CTA of the cluster shares the chain
    const Task T = tasks[t];
    const BlockFactor F = shapes[T.shape];
    const SpikeInfo SP = spikes[T.shape];
    const long long off = use_fine ? T.foff : T.coff;
    const int m = F.m;
    const int J0 = SP.B[rank], J1 = SP.B[rank + 1], nb = J1 - J0;
    const int r0 = J0 * BNB, r1 = J1 * BNB, rend = r1 < m ? r1 : m;
    const int slot = la_slot(maxK);
    float2 *CY = reinterpret_cast<float2 *>(smd + RING * slot), *CX = CY + cwy;
    const int *perm = Pall + F.perm_off;
    const int4 *meta = Meta + F.meta_off;
    const double *inr = reinterpret_cast<const double *>(in + off) + comp;
    double *outr = reinterpret_cast<double *>(out + off) + comp;
    float2 *od = reinterpret_cast<float2 *>(outr);   // entries as (hi, lo) pairs during the solve
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int row = lane >> 1, half = lane & 1;
    const int q = (warp - 1) * 2 + half;
    const int bt = tid - 32;
    auto load_block = [&](long long src_off, int K, int buf, int J) {
        if (bt < 0) return;
        double *dst = smd + buf * slot;
        const float2 *src = Mdf + src_off;
        const int nchunk = BNB * K / 2;
        for (int c = bt; c < nchunk; c += SPK_T - 32) cp_async16(dst + 2 * c, src + 2 * c);
        if (bt < BNB) {
            const int i = J * BNB + bt;
            cp_async8_zfill(dst + BNB * maxK + bt, i < m ? outr + STR * (long long)i : outr, i < m ? 8 : 0);
        }
    };
    for (int i = r0 + tid; i < rend; i += SPK_T) od[STR * (long long)i] = df_split(inr[STR * (long long)perm[i]]);
    for (int i = tid; i < cwy; i += SPK_T) CY[i] = make_float2(0.f, 0.f);
    for (int i = tid; i < cwx; i += SPK_T) CX[i] = make_float2(0.f, 0.f);
    __threadfence_block();
    __syncthreads();

    auto bulk_row = [&](const double *sp, int K, int k0, int k1, const float2 *win, int pbase, int mask) {
        const float2 *Mr = reinterpret_cast<const float2 *>(sp) + row * K;
        const float2 *a = reinterpret_cast<const float2 *>(sp + BNB * maxK);
        float sh = 0.f, sl = 0.f;
        int k = q;
        for (; k < BNB; k += SPK_BL) {
            const float2 mk = Mr[k], x = a[k];
            df_acc(sh, sl, mk.x, mk.y, x.x, x.y);
        }
        if (k < k0) k += ((k0 - k + SPK_BL - 1) / SPK_BL) * SPK_BL;
        for (; k < k1; k += SPK_BL) {
            const float2 mk = Mr[k], x = win[(pbase + k - BNB) & mask];
            df_acc(sh, sl, mk.x, mk.y, x.x, x.y);
        }
        const float oh = __shfl_xor_sync(0xffffffffu, sh, 1), ol = __shfl_xor_sync(0xffffffffu, sl, 1);
        df_add(sh, sl, oh, ol);
        return make_float2(sh, sl);
    };
    auto chain_row = [&](const double *sp, int K, int p0, int p1, const float2 *win, int pbase, int mask,
                         int par) {
        const float2 *Mr = reinterpret_cast<const float2 *>(sp) + row * K + BNB;
        // lane half 0 seeds with the partials of bulk warps 0, 2, 4, 6; half 1 with 1, 3, 5
        float2 a0 = part[par][half][row], a1 = part[par][half + 2][row], a2 = part[par][half + 4][row];
        float2 a3 = half == 0 ? part[par][6][row] : make_float2(0.f, 0.f);
        auto madd = [&](float2 &acc, int p) {
            const float2 mk = Mr[p], x = win[(pbase + p) & mask];
            df_acc(acc.x, acc.y, mk.x, mk.y, x.x, x.y);
        };
        int p = p0 + half;
        for (; p + 6 < p1; p += 8) { madd(a0, p); madd(a1, p + 2); madd(a2, p + 4); madd(a3, p + 6); }
        if (p < p1) madd(a0, p);
        if (p + 2 < p1) madd(a1, p + 2);
        if (p + 4 < p1) madd(a2, p + 4);
        df_add(a0.x, a0.y, a1.x, a1.y);
        df_add(a2.x, a2.y, a3.x, a3.y);
        df_add(a0.x, a0.y, a2.x, a2.y);
        const float oh = __shfl_xor_sync(0xffffffffu, a0.x, 1), ol = __shfl_xor_sync(0xffffffffu, a0.y, 1);
        df_add(a0.x, a0.y, oh, ol);
        return a0;
    };

    // acc += Σ_{k<n} g[k·ld] x[k] in pairs, the spike entries loaded eight at a time ahead of
    // their arithmetic (they come from L2; one dependent sum would wait on every load)
    auto gdot = [&](float2 acc, const float2 *g, long long ld, const float2 *x, int n) {
        int k = 0;
        for (; k + 8 <= n; k += 8) {
            float2 gv[8];
#pragma unroll
            for (int u = 0; u < 8; u++) gv[u] = g[(long long)(k + u) * ld];
#pragma unroll
            for (int u = 0; u < 8; u++) df_acc(acc.x, acc.y, gv[u].x, gv[u].y, x[k + u].x, x[k + u].y);
        }
        for (; k < n; k++) {
            const float2 gv = g[(long long)k * ld];
            df_acc(acc.x, acc.y, gv.x, gv.y, x[k].x, x[k].y);
        }
        return acc;
    };

    // ---- forward local sweep over the part's blocks: g_p (window values below r0 are zero) ----
    int4 mq0 = make_int4(0, 0, 0, 0), mq1 = mq0, mq2 = mq0;
#pragma unroll
    for (int u = 0; u < RING - 1; u++) {
        if (u < nb) {
            const int4 mt = meta[J0 + u];
            load_block(mt.x, op_stride(mt.y), u, J0 + u);
            if (tid == 32) sw[u] = mt.y;
        }
        cp_async_commit();
    }
    if (RING - 1 < nb) mq0 = meta[J0 + RING - 1];
    if (RING < nb) mq1 = meta[J0 + RING];
    if (RING + 1 < nb) mq2 = meta[J0 + RING + 1];
    cp_async_wait_n<RING - 2>();
    __syncthreads();
    if (warp > 0) {
        const int w0 = sw[0], nold = w0 > BNB ? w0 - BNB : 0;
        const float2 v = bulk_row(smd, op_stride(w0), BNB, BNB + nold, CY, r0 - w0, cwy - 1);
        if (half == 0) part[0][warp - 1][row] = v;
    }
    for (int k = 0; k < nb; k++) {
        const int J = J0 + k;
        cp_async_wait_n<RING - 3>();
        __syncthreads();
        if (k + RING - 1 < nb) {
            const int buf = (k + RING - 1) % RING;
            load_block(mq0.x, op_stride(mq0.y), buf, J + RING - 1);
            if (tid == 32) sw[buf] = mq0.y;
        }
        cp_async_commit();
        mq0 = mq1; mq1 = mq2;
        if (k + RING + 2 < nb) mq2 = meta[J + RING + 2];
        if (warp == 0) {
            const int wJ = sw[k % RING];
            const int p0 = wJ > BNB ? wJ - BNB : 0;
            const float2 v = chain_row(smd + (k % RING) * slot, op_stride(wJ), p0, wJ, CY, J * BNB - wJ, cwy - 1, k & 1);
            if (half == 0) {
                const int i = J * BNB + row;
                CY[i & (cwy - 1)] = v;
                if (i < m) od[STR * (long long)i] = v;
            }
        } else if (k + 1 < nb) {
            const int kn = k + 1, Jn = J + 1, w1 = sw[kn % RING], nold = w1 > BNB ? w1 - BNB : 0;
            const float2 v = bulk_row(smd + (kn % RING) * slot, op_stride(w1), BNB, BNB + nold, CY, Jn * BNB - w1, cwy - 1);
            if (half == 0) part[kn & 1][warp - 1][row] = v;
        }
    }
    cp_async_wait_n<0>();
    __threadfence();
    __syncthreads();
    spk_cluster_sync();                              // (1) every part's g is written

    // ---- forward boundary values t_rank (parts >= 1) from the parts' local solutions ----
    const int wf = SP.wf, wb = SP.wb;
    float2 *tcur = tb[0], *tnext = tb[1];
    if (rank >= 1) {
        const int ra = SP.B[1] * BNB - wf;            // tail rows of part 0: [r_1 - wf, r_1)
        for (int k = tid; k < wf; k += SPK_T) tcur[k] = od[STR * (long long)(ra + k)];
        __syncthreads();
        for (int qq = 1; qq < rank; qq++) {           // t_{qq+1} = g_qq[tail] + Gf_qq[tail rows] t_qq
            const int rq = SP.B[qq] * BNB, nq = (SP.B[qq + 1] - SP.B[qq]) * BNB;
            const float2 *Gq = G + SP.gf[qq];
            for (int kk = tid; kk < wf; kk += SPK_T) {
                const int il = nq - wf + kk;          // local row of the tail entry
                tnext[kk] = gdot(od[STR * (long long)(rq + il)], Gq + il, nq, tcur, wf);
            }
            __syncthreads();
            float2 *sx = tcur; tcur = tnext; tnext = sx;
        }
    }
    spk_cluster_sync();                              // (2) every part has read the g it needs
    if (rank >= 1) {                                 // y_p = g_p + Gf_p t_p
        const int np = r1 - r0;
        const float2 *Gp = G + SP.gf[rank];
        for (int i = r0 + tid; i < rend; i += SPK_T)
            od[STR * (long long)i] = gdot(od[STR * (long long)i], Gp + (i - r0), np, tcur, wf);
    }
    __threadfence_block();
    __syncthreads();

    // ---- backward local sweep: l_p (window values from r1 on are zero) ----
#pragma unroll
    for (int u = 0; u < RING - 1; u++) {
        const int J = J1 - 1 - u;
        if (J >= J0) {
            const int4 mt = meta[J];
            load_block(mt.z, op_stride(mt.w), u, J);
            if (tid == 32) sw[u] = mt.w;
        }
        cp_async_commit();
    }
    mq0 = J1 - RING >= J0 ? meta[J1 - RING] : make_int4(0, 0, 0, 0);
    mq1 = J1 - RING - 1 >= J0 ? meta[J1 - RING - 1] : make_int4(0, 0, 0, 0);
    mq2 = J1 - RING - 2 >= J0 ? meta[J1 - RING - 2] : make_int4(0, 0, 0, 0);
    cp_async_wait_n<RING - 2>();
    __syncthreads();
    if (warp > 0) {
        const int w0 = sw[0];
        const float2 v = bulk_row(smd, op_stride(w0), 2 * BNB, BNB + w0, CX, r1, cwx - 1);
        if (half == 0) part[0][warp - 1][row] = v;
    }
    for (int k = 0; k < nb; k++) {
        const int J = J1 - 1 - k;
        cp_async_wait_n<RING - 3>();
        __syncthreads();
        if (J - (RING - 1) >= J0) {
            const int buf = (k + RING - 1) % RING;
            load_block(mq0.z, op_stride(mq0.w), buf, J - (RING - 1));
            if (tid == 32) sw[buf] = mq0.w;
        }
        cp_async_commit();
        mq0 = mq1; mq1 = mq2;
        if (J - RING - 2 >= J0) mq2 = meta[J - RING - 2];
        if (warp == 0) {
            const int wJ = sw[k % RING];
            const float2 v = chain_row(smd + (k % RING) * slot, op_stride(wJ), 0, wJ < BNB ? wJ : BNB, CX,
                                       (J + 1) * BNB, cwx - 1, k & 1);
            if (half == 0) {
                const int i = J * BNB + row;
                CX[i & (cwx - 1)] = v;
                if (i < m) od[STR * (long long)i] = v;
            }
        } else if (J - 1 >= J0) {
            const int kn = k + 1, Jn = J - 1, w1 = sw[kn % RING];
            const float2 v = bulk_row(smd + (kn % RING) * slot, op_stride(w1), 2 * BNB, BNB + w1, CX, (Jn + 1) * BNB,
                                      cwx - 1);
            if (half == 0) part[kn & 1][warp - 1][row] = v;
        }
    }
    cp_async_wait_n<0>();
    __threadfence();
    __syncthreads();
    spk_cluster_sync();                              // (3) every part's l is written

    // ---- backward boundary values h_rank (parts <= P-2) ----
    if (rank <= P - 2) {
        const int ra = SP.B[P - 1] * BNB;             // head rows of the last part (final as solved)
        for (int k = tid; k < wb; k += SPK_T)
            tcur[k] = ra + k < m ? od[STR * (long long)(ra + k)] : make_float2(0.f, 0.f);
        __syncthreads();
        for (int qq = P - 2; qq > rank; qq--) {       // h_{qq-1} = l_qq[head] + Gb_qq[head rows] h_qq
            const int rq = SP.B[qq] * BNB, nq = (SP.B[qq + 1] - SP.B[qq]) * BNB;
            const float2 *Gq = G + SP.gb[qq];
            for (int kk = tid; kk < wb; kk += SPK_T) {
                tnext[kk] = gdot(od[STR * (long long)(rq + kk)], Gq + kk, nq, tcur, wb);
            }
            __syncthreads();
            float2 *sx = tcur; tcur = tnext; tnext = sx;
        }
    }
    spk_cluster_sync();                              // (4) every part has read the l it needs
    if (rank <= P - 2) {                             // x_p = l_p + Gb_p h_p
        const int np = r1 - r0;
        const float2 *Gp = G + SP.gb[rank];
        for (int i = r0 + tid; i < rend; i += SPK_T)
            od[STR * (long long)i] = gdot(od[STR * (long long)i], Gp + (i - r0), np, tcur, wb);
    }
    __syncthreads();
    for (int i = r0 + tid; i < rend; i += SPK_T) {
        const float2 v = od[STR * (long long)i];
        outr[STR * (long long)i] = (double)v.x + (double)v.y;
    }
}

// list[0 .. count) = the indices i < n with flag[i] != 0, in increasing order, list[count .. n) =
// -1 (one CTA of 1024 threads: ballots within warps, a scan of the warp counts per chunk)
__global__ void __launch_bounds__(1024) k_compact_flags(int n, const int *__restrict__ flag, int *__restrict__ list) {
    __shared__ int wc[32];
    __shared__ int base_s;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) base_s = 0;
    __syncthreads();
    for (int c0 = 0; c0 < n; c0 += 1024) {
        const int i = c0 + tid;
        const bool on = i < n && flag[i] != 0;
        const unsigned b = __ballot_sync(0xffffffffu, on);
        if (lane == 0) wc[warp] = __popc(b);
        __syncthreads();
        int before = 0, total = 0;
        for (int w = 0; w < 32; w++) {
            if (w < warp) before += wc[w];
            total += wc[w];
        }
        const int base = base_s;
        if (on) list[base + before + __popc(b & ((1u << lane) - 1u))] = i;
        __syncthreads();
        if (tid == 0) base_s = base + total;
        __syncthreads();
    }
    for (int i = base_s + tid; i < n; i += 1024) list[i] = -1;      // past the count: no task
}
void launch_compact_flags(int n, const int *flag, int *list, cudaStream_t s) {
    k_compact_flags<<<1, 1024, 0, s>>>(n, flag, list);
}

__global__ void k_ops_to_df(long long n, const double *__restrict__ M, float2 *__restrict__ Mdf) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        Mdf[i] = df_split(M[i]);
}

void launch_assemble_E(const Stencil &st, int nx, int ny, int kl, int ku, double *ab, cudaStream_t s) {
    long long tot = (long long)(nx / 2) * (ny / 2) * 25;
    k_assemble_E<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(st, nx, ny, kl, ku, ab);
}
void launch_assemble_Aloc(const Stencil &st, int nx, int ny, int kl, int ku, double *ab, cudaStream_t s) {
    long long tot = (long long)nx * ny * 9;
    k_assemble_Aloc<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(st, nx, ny, kl, ku, ab);
}
void launch_assemble_E_re2(const Stencil &st, int nx, int ny, int gx0, int gy0, int kl2, int ku2, double *ab,
                           cudaStream_t s) {
    long long tot = (long long)(nx / 2) * (ny / 2) * 25;
    k_assemble_E_re2<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(st, nx, ny, gx0, gy0, kl2, ku2, ab);
}
void launch_assemble_Aloc_re2(const Stencil &st, int nx, int ny, int gx0, int gy0, int kl2, int ku2, double *ab,
                              cudaStream_t s) {
    long long tot = (long long)nx * ny * 9;
    k_assemble_Aloc_re2<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(st, nx, ny, gx0, gy0, kl2, ku2, ab);
}
void launch_band_lu(int nmat, const int *m, const int *kl, const int *ku, double *const *ab,
                    int *const *piv, int *info, cudaStream_t s) {
    k_band_lu<<<nmat, 512, 0, s>>>(m, kl, ku, ab, piv, info);
}
void launch_ops_to_df(long long n, const double *M, float2 *Mdf, cudaStream_t s) {
    long long g = (n + 255) / 256;
    if (g > 8 * 152) g = 8 * 152;
    k_ops_to_df<<<(int)(g > 0 ? g : 1), 256, 0, s>>>(n, M, Mdf);
}
void launch_factor_prepare(int m, int kl, int ku, const double *ab, const int *piv, int KLW,
                           double *Lp, int *lext, int *uext, int *perm, int *err, cudaStream_t s) {
    k_perm<<<1, 32, 0, s>>>(m, piv, perm);
    k_lperm<<<(m + 127) / 128, 128, 0, s>>>(m, kl, ku, ab, piv, KLW, Lp, lext, err);
    k_uext<<<(m + 127) / 128, 128, 0, s>>>(m, kl, ku, ab, uext);
}
void launch_block_operators(int m, int kl, int ku, const double *ab, int KLW, const double *Lp,
                            const int4 *meta, double *Mall, cudaStream_t s) {
    const int nbk = (m + BNB - 1) / BNB;
    k_block_fwd<<<nbk, 128, 0, s>>>(m, KLW, Lp, meta, Mall);
    k_block_bwd<<<nbk, 128, 0, s>>>(m, kl, ku, ab, meta, Mall);
}
static size_t bs_smem(const BlockSolveCfg &c, int ring) {
    return ((size_t)ring * ((size_t)BNB * c.maxK + BNB) + (size_t)c.cwy + (size_t)c.cwx) * sizeof(double);
}
static size_t la_smem(const BlockSolveCfg &c, int ring) {
    return ((size_t)ring * la_slot(c.maxK) + (size_t)c.cwy + (size_t)c.cwx) * sizeof(double);
}

template <int RING, bool RE2>
static void la_launch(int grid, const BlockSolveCfg &c, const Task *tasks, const BlockFactor *shapes,
                      const double *Mall, const float2 *Mdf, const int *Pall, const int4 *Meta, const double2 *in,
                      double2 *out, int use_fine, const int *flag, cudaStream_t s) {
    if (Mdf)
        k_block_solve_la_df<RING, RE2><<<grid, LAD_T, la_smem(c, RING), s>>>(tasks, shapes, Mdf, Pall, Meta, in, out,
                                                                             use_fine, flag, c.maxK, c.cwy, c.cwx);
    else
        k_block_solve_la<RING, RE2><<<grid, LA_T, la_smem(c, RING), s>>>(tasks, shapes, Mall, Pall, Meta, in, out,
                                                                          use_fine, flag, c.maxK, c.cwy, c.cwx);
}

static int sm_count() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
            n = 152;
    }
    return n;
}

void launch_block_solve(const Task *tasks, int ntasks, const BlockFactor *shapes, const double *Mall,
                        const int *Pall, const int4 *Meta, const double2 *in, double2 *out,
                        int use_fine, const int *flag, const BlockSolveCfg &c, int re2, cudaStream_t s,
                        const float2 *Mdf) {
    const int chains = re2 ? ntasks : 2 * ntasks;
    if (!(c.lookahead && c.la_ring >= 3)) Mdf = nullptr;    // the double-FP32 form exists as look-ahead only
    if (c.lookahead && c.la_ring >= 3) {
        // the deepest ring that fits, unless there are more chains than SMs and a ring of 4 lets
        // two CTAs share an SM (many chains: throughput over latency)
        int ring = c.la_ring;
        if (ring > 4 && chains > sm_count() && 2 * (la_smem(c, 4) + 4096) <= 228 * 1024) ring = 4;
        if (re2) {
            if (ring == 6) la_launch<6, true>(chains, c, tasks, shapes, Mall, Mdf, Pall, Meta, in, out, use_fine, flag, s);
            else if (ring == 4) la_launch<4, true>(chains, c, tasks, shapes, Mall, Mdf, Pall, Meta, in, out, use_fine, flag, s);
            else la_launch<3, true>(chains, c, tasks, shapes, Mall, Mdf, Pall, Meta, in, out, use_fine, flag, s);
        } else {
            if (ring == 6) la_launch<6, false>(chains, c, tasks, shapes, Mall, Mdf, Pall, Meta, in, out, use_fine, flag, s);
            else if (ring == 4) la_launch<4, false>(chains, c, tasks, shapes, Mall, Mdf, Pall, Meta, in, out, use_fine, flag, s);
            else la_launch<3, false>(chains, c, tasks, shapes, Mall, Mdf, Pall, Meta, in, out, use_fine, flag, s);
        }
        return;
    }
    if (re2) {
        if (c.ring == 4)
            k_block_solve<4, true><<<ntasks, BS_T, bs_smem(c, 4), s>>>(tasks, shapes, Mall, Pall, Meta, in, out,
                                                                       use_fine, flag, c.maxK, c.cwy, c.cwx);
        else
            k_block_solve<2, true><<<ntasks, BS_T, bs_smem(c, 2), s>>>(tasks, shapes, Mall, Pall, Meta, in, out,
                                                                       use_fine, flag, c.maxK, c.cwy, c.cwx);
        return;
    }
    if (c.ring == 4)
        k_block_solve<4, false><<<2 * ntasks, BS_T, bs_smem(c, 4), s>>>(tasks, shapes, Mall, Pall, Meta, in, out,
                                                                        use_fine, flag, c.maxK, c.cwy, c.cwx);
    else
        k_block_solve<2, false><<<2 * ntasks, BS_T, bs_smem(c, 2), s>>>(tasks, shapes, Mall, Pall, Meta, in, out,
                                                                        use_fine, flag, c.maxK, c.cwy, c.cwx);
}

// SPIKE launches: clusters of P CTAs, one CTA per SM, the ring of the look-ahead kernel (6, 4 or 3)
template <int RING, bool RE2>
static cudaError_t spk_launch(int P, int grid, const BlockSolveCfg &c, const Task *tasks, const BlockFactor *shapes,
                              const float2 *Mdf, const int *Pall, const int4 *Meta, const SpikeInfo *spikes,
                              const float2 *G, const double2 *in, double2 *out, int use_fine, const int *flag,
                              const int *list, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(SPK_T);
    cfg.dynamicSmemBytes = la_smem(c, RING);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)P;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_block_solve_spike_df<RING, RE2>, tasks, shapes, Mdf, Pall, Meta, spikes, G, in,
                              out, use_fine, flag, list, c.maxK, c.cwy, c.cwx, P);
}
template <bool RE2>
static cudaError_t spk_launch_ring(int P, int grid, const BlockSolveCfg &c, const Task *tasks,
                                   const BlockFactor *shapes, const float2 *Mdf, const int *Pall, const int4 *Meta,
                                   const SpikeInfo *spikes, const float2 *G, const double2 *in, double2 *out,
                                   int use_fine, const int *flag, const int *list, cudaStream_t s) {
    if (c.spike_ok >= 6)
        return spk_launch<6, RE2>(P, grid, c, tasks, shapes, Mdf, Pall, Meta, spikes, G, in, out, use_fine, flag, list, s);
    if (c.spike_ok >= 4)
        return spk_launch<4, RE2>(P, grid, c, tasks, shapes, Mdf, Pall, Meta, spikes, G, in, out, use_fine, flag, list, s);
    return spk_launch<3, RE2>(P, grid, c, tasks, shapes, Mdf, Pall, Meta, spikes, G, in, out, use_fine, flag, list, s);
}

bool launch_block_solve_spike(int P, const Task *tasks, int ntasks, const BlockFactor *shapes,
                              const float2 *Mdf, const int *Pall, const int4 *Meta, const SpikeInfo *spikes,
                              const float2 *G, const double2 *in, double2 *out, int use_fine, const int *flag,
                              const int *list, const BlockSolveCfg &c, int re2, cudaStream_t s) {
    if (P < 2 || P > SPIKE_PMAX || !c.spike_ok || ntasks < 1) return false;
    const int chains = re2 ? ntasks : 2 * ntasks;
    const cudaError_t e = re2 ? spk_launch_ring<true>(P, chains * P, c, tasks, shapes, Mdf, Pall, Meta, spikes, G, in,
                                                      out, use_fine, flag, list, s)
                              : spk_launch_ring<false>(P, chains * P, c, tasks, shapes, Mdf, Pall, Meta, spikes, G, in,
                                                       out, use_fine, flag, list, s);
    if (e != cudaSuccess) cudaGetLastError();      // a refused launch configuration: the caller falls back
    return e == cudaSuccess;
}

template <int RING, bool RE2> static cudaError_t spk_attr(size_t lim, size_t &static_bytes) {
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, k_block_solve_spike_df<RING, RE2>);
    if (e != cudaSuccess) return e;
    static_bytes = std::max(static_bytes, a.sharedSizeBytes);
    return cudaFuncSetAttribute(k_block_solve_spike_df<RING, RE2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(lim - a.sharedSizeBytes));
}
template <int RING, bool RE2> static cudaError_t la_attr(size_t lim, size_t &static_bytes) {
    cudaFuncAttributes a, b;
    cudaError_t e = cudaFuncGetAttributes(&a, k_block_solve_la<RING, RE2>);
    if (e != cudaSuccess) return e;
    if ((e = cudaFuncGetAttributes(&b, k_block_solve_la_df<RING, RE2>)) != cudaSuccess) return e;
    static_bytes = std::max(static_bytes, std::max(a.sharedSizeBytes, b.sharedSizeBytes));
    if ((e = cudaFuncSetAttribute(k_block_solve_la<RING, RE2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)(lim - a.sharedSizeBytes))) != cudaSuccess)
        return e;
    return cudaFuncSetAttribute(k_block_solve_la_df<RING, RE2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(lim - b.sharedSizeBytes));
}

// Ring depth 4 if its shared memory fits the per-CTA limit, else 2; error if not even that fits.
// The kernels' attribute is raised to the limit itself (several factor sets with different plans
// share the kernels; each launch requests only what its plan needs).  The look-ahead kernel takes
// the deepest of rings 6, 4, 3 that fits (la_ring, 0 if none: the plain kernel then serves).
cudaError_t set_block_solve_smem(BlockSolveCfg &c) {
    cudaFuncAttributes a4, a2, b4, b2;
    cudaError_t e = cudaFuncGetAttributes(&a4, k_block_solve<4, false>);
    if (e != cudaSuccess) return e;
    if ((e = cudaFuncGetAttributes(&a2, k_block_solve<2, false>)) != cudaSuccess) return e;
    if ((e = cudaFuncGetAttributes(&b4, k_block_solve<4, true>)) != cudaSuccess) return e;
    if ((e = cudaFuncGetAttributes(&b2, k_block_solve<2, true>)) != cudaSuccess) return e;
    const size_t lim = 227 * 1024;                        // per-CTA limit, static + dynamic
    const size_t lim4 = lim - std::max(a4.sharedSizeBytes, b4.sharedSizeBytes);
    const size_t lim2 = lim - std::max(a2.sharedSizeBytes, b2.sharedSizeBytes);
    c.ring = bs_smem(c, 4) <= lim4 ? 4 : 2;
    if (bs_smem(c, c.ring) > (c.ring == 4 ? lim4 : lim2)) return cudaErrorInvalidValue;
    if ((e = cudaFuncSetAttribute(k_block_solve<4, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lim4)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_block_solve<2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lim2)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_block_solve<4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lim4)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_block_solve<2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lim2)) != cudaSuccess)
        return e;
    size_t st = 0;
    if ((e = la_attr<6, false>(lim, st)) != cudaSuccess) return e;
    if ((e = la_attr<4, false>(lim, st)) != cudaSuccess) return e;
    if ((e = la_attr<3, false>(lim, st)) != cudaSuccess) return e;
    if ((e = la_attr<6, true>(lim, st)) != cudaSuccess) return e;
    if ((e = la_attr<4, true>(lim, st)) != cudaSuccess) return e;
    if ((e = la_attr<3, true>(lim, st)) != cudaSuccess) return e;
    c.la_ring = 0;
    for (int r : {6, 4, 3})
        if (la_smem(c, r) + st <= lim) { c.la_ring = r; break; }
    // the SPIKE kernels (one CTA per SM): the deepest ring of 6, 4, 3 that fits (spike_ok = ring)
    size_t sst = 0;
    if ((e = spk_attr<6, false>(lim, sst)) != cudaSuccess) return e;
    if ((e = spk_attr<6, true>(lim, sst)) != cudaSuccess) return e;
    if ((e = spk_attr<4, false>(lim, sst)) != cudaSuccess) return e;
    if ((e = spk_attr<4, true>(lim, sst)) != cudaSuccess) return e;
    if ((e = spk_attr<3, false>(lim, sst)) != cudaSuccess) return e;
    if ((e = spk_attr<3, true>(lim, sst)) != cudaSuccess) return e;
    c.spike_ok = 0;
    for (int r : {6, 4, 3})
        if (la_smem(c, r) + sst <= lim) { c.spike_ok = r; break; }
    // clusters of 2 and of 4 the device co-schedules with that ring (a cluster lives in one GPC,
    // so this is below #SMs / P): more active chains than this would run in a second wave
    c.spike_cap[0] = c.spike_cap[1] = 0;
    if (c.spike_ok) {
        for (int L = 0; L < 2; L++) {
            cudaLaunchConfig_t cf = {};
            cf.gridDim = dim3(L == 0 ? 2u : 4u);
            cf.blockDim = dim3(SPK_T);
            cf.dynamicSmemBytes = la_smem(c, c.spike_ok);
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = L == 0 ? 2u : 4u;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            cf.attrs = at;
            cf.numAttrs = 1;
            int n = 0;
            const cudaError_t qe = c.spike_ok >= 6 ? cudaOccupancyMaxActiveClusters(&n, k_block_solve_spike_df<6, false>, &cf)
                                 : c.spike_ok >= 4 ? cudaOccupancyMaxActiveClusters(&n, k_block_solve_spike_df<4, false>, &cf)
                                                   : cudaOccupancyMaxActiveClusters(&n, k_block_solve_spike_df<3, false>, &cf);
            if (qe != cudaSuccess) { cudaGetLastError(); n = 0; }
            c.spike_cap[L] = n;
        }
    }
    return cudaSuccess;
}

}  // namespace hdd
