// kernels_coarse.cu — FP64 coarse-space kernels of the two-level deflation (Eq. 4): assembly of
// E = Zᵀ A Z on the device, banded LU with partial pivoting, and the batched banded solve
// E⁻¹ y for every task (real factor, real and imaginary parts as two chains).
// The same factor/solve serves the direct local solve A_j⁻¹ (§3.1 benchmark).
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

// Re-layout a factor for the solve: L by columns; U by columns above the diagonal, scaled to a
// unit diagonal (Û = D⁻¹U, entry Û(r,c) = U(r,c)/U(r,r)), with the true extent of each column;
// reciprocal pivots 1/U(r,r).
__global__ void k_band_convert(int m, int kl, int ku, const double *__restrict__ ab,
                               const int *__restrict__ piv, double *__restrict__ Lcol,
                               double *__restrict__ Ucol, int *__restrict__ uext,
                               double *__restrict__ rinv, int *__restrict__ pivout) {
    const int W = 2 * kl + ku + 1, KU = kl + ku;
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    for (int q = 0; q < kl; q++) {
        int r = j + 1 + q;
        Lcol[(long long)j * kl + q] = r < m ? ab[(long long)r * W + (j - r + kl)] : 0.0;
    }
    int ext = 0;
    for (int q = 0; q < KU; q++) {
        int r = j - 1 - q;
        double v = 0.0;
        if (r >= 0) {
            double u = ab[(long long)r * W + (j - r + kl)];
            v = u / ab[(long long)r * W + kl];
        }
        Ucol[(long long)j * KU + q] = v;
        if (v != 0.0) ext = q + 1;
    }
    uext[j] = ext;
    rinv[j] = 1.0 / ab[(long long)j * W + kl];
    pivout[j] = piv[j];
}

constexpr int BS_PF = 8;        // factor columns in flight ahead of the sweep (per warp ring)
constexpr int BS_KMAX = 8;      // up to 8 x 32 = 256 band entries per column

__device__ __forceinline__ void cp_async8(void *smem_dst, const void *gsrc) {
    unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// x = F⁻¹ b for the real banded factor F of the task's shape.  One WARP per (task, component)
// chain, so a step needs only warp-level synchronisation: lane ℓ updates rows j+1+ℓ+32k.
// The warp's vector sits in shared memory; the factor columns stream through a per-warp ring
// filled by cp.async BS_PF steps ahead (each lane copies, and later reads, its own entries).
// Forward: interchange b_j ↔ b_piv(j), then b_{j+1..j+kl} -= L(:,j) b_j; backward: unit upper
// sweep on D⁻¹y with the true extent of every column of Û.
template <int K>
__global__ void __launch_bounds__(128)
k_band_solve(const Task *__restrict__ tasks, int ntasks, const BandFactor *__restrict__ shapes,
             const double *__restrict__ Lall, const double *__restrict__ Uall,
             const int *__restrict__ Iall, const double *__restrict__ Rall,
             const double2 *__restrict__ in, double2 *__restrict__ out, int use_fine,
             const int *__restrict__ flag, int max_m) {
    extern __shared__ double bsm[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int chain = blockIdx.x * (blockDim.x >> 5) + warp;
    if (chain >= 2 * ntasks) return;
    const int t = chain >> 1, comp = chain & 1;
    if (flag && !flag[t]) return;
    // per-warp shared memory: b[max_m] | piv[max_m] | uext[max_m] | ring[BS_PF][32K]
    const size_t per_warp = (size_t)max_m * 16 + (size_t)BS_PF * 32 * K * 8;
    double *b = reinterpret_cast<double *>(reinterpret_cast<unsigned char *>(bsm) + per_warp * warp);
    int *piv = reinterpret_cast<int *>(b + max_m);
    int *uext = piv + max_m;
    double *ring = reinterpret_cast<double *>(uext + max_m);
    const Task T = tasks[t];
    const BandFactor F = shapes[T.shape];
    const long long off = use_fine ? T.foff : T.coff;
    const int m = F.m, kl = F.kl, KU = F.kl + F.ku;
    const double *L = Lall + F.l_off;
    const double *U = Uall + F.u_off;
    const int *piv_g = Iall + 2 * F.p_off;
    const int *uext_g = piv_g + m;
    const double *rinv = Rall + F.p_off;
    const double *inr = reinterpret_cast<const double *>(in + off) + comp;
    double *outr = reinterpret_cast<double *>(out + off) + comp;
    for (int i = lane; i < m; i += 32) {
        b[i] = inr[2 * (long long)i];
        piv[i] = piv_g[i];
        uext[i] = uext_g[i];
    }
    // ---- forward ----
    auto issue_L = [&](int j) {          // column min(j, m-1) of L, entries lane + 32k (clamped)
        const double *col = L + (long long)min(j, m - 1) * kl;
        double *slot = ring + (j % BS_PF) * 32 * K;
#pragma unroll
        for (int k = 0; k < K; k++) cp_async8(slot + k * 32 + lane, col + min(lane + 32 * k, kl - 1));
        cp_async_commit();
    };
#pragma unroll
    for (int u = 0; u < BS_PF - 1; u++) issue_L(u);
    __syncwarp();
    for (int j = 0; j < m; j++) {
        issue_L(j + BS_PF - 1);
        cp_async_wait<BS_PF - 1>();                  // column j of L is in this lane's slots
        const int p = piv[j];
        const double sj = b[j], sp = b[p];
        const int nq = min(kl, m - 1 - j);
        const double *lc = ring + (j % BS_PF) * 32 * K;
        double nv[K];
#pragma unroll
        for (int k = 0; k < K; k++) {
            const int q = lane + 32 * k, r = j + 1 + q;
            nv[k] = 0.0;
            if (q < nq) nv[k] = fma(-lc[k * 32 + lane], sp, (r == p) ? sj : b[r]);
        }
        __syncwarp();                                 // every lane has read b[j], b[p]
#pragma unroll
        for (int k = 0; k < K; k++) {
            const int q = lane + 32 * k;
            if (q < nq) b[j + 1 + q] = nv[k];
        }
        if (lane == 0) b[j] = sp;                     // y_j
        __syncwarp();
    }
    cp_async_wait<0>();
    // ---- D⁻¹ y ----
    for (int i = lane; i < m; i += 32) b[i] *= rinv[i];
    __syncwarp();
    // ---- backward ----
    auto issue_U = [&](int c) {          // column max(c, 0) of Û, entries lane + 32k (clamped)
        const double *col = U + (long long)max(c, 0) * KU;
        double *slot = ring + (((c % BS_PF) + BS_PF) % BS_PF) * 32 * K;
#pragma unroll
        for (int k = 0; k < K; k++) cp_async8(slot + k * 32 + lane, col + min(lane + 32 * k, KU - 1));
        cp_async_commit();
    };
#pragma unroll
    for (int u = 0; u < BS_PF - 1; u++) issue_U(m - 1 - u);
    for (int c = m - 1; c >= 0; c--) {
        issue_U(c - (BS_PF - 1));
        cp_async_wait<BS_PF - 1>();
        const double xc = b[c];
        const int ne = uext[c];
        const double *uc = ring + (c % BS_PF) * 32 * K;
        double nv[K];
#pragma unroll
        for (int k = 0; k < K; k++) {
            const int q = lane + 32 * k;
            nv[k] = 0.0;
            if (q < ne) nv[k] = fma(-uc[k * 32 + lane], xc, b[c - 1 - q]);
        }
        __syncwarp();
#pragma unroll
        for (int k = 0; k < K; k++) {
            const int q = lane + 32 * k;
            if (q < ne) b[c - 1 - q] = nv[k];
        }
        if (lane == 0) outr[2 * (long long)c] = xc;
        __syncwarp();
    }
    cp_async_wait<0>();
}

void launch_assemble_E(const Stencil &st, int nx, int ny, int kl, int ku, double *ab, cudaStream_t s) {
    long long tot = (long long)(nx / 2) * (ny / 2) * 25;
    k_assemble_E<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(st, nx, ny, kl, ku, ab);
}
void launch_assemble_Aloc(const Stencil &st, int nx, int ny, int kl, int ku, double *ab, cudaStream_t s) {
    long long tot = (long long)nx * ny * 9;
    k_assemble_Aloc<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(st, nx, ny, kl, ku, ab);
}
void launch_band_lu(int nmat, const int *m, const int *kl, const int *ku, double *const *ab,
                    int *const *piv, int *info, cudaStream_t s) {
    k_band_lu<<<nmat, 512, 0, s>>>(m, kl, ku, ab, piv, info);
}
void launch_band_convert(int m, int kl, int ku, const double *ab, const int *piv, double *Lcol,
                         double *Ucol, int *uext, double *rinv, int *pivout, cudaStream_t s) {
    k_band_convert<<<(m + 127) / 128, 128, 0, s>>>(m, kl, ku, ab, piv, Lcol, Ucol, uext, rinv, pivout);
}
// warps per CTA and dynamic shared memory of the banded solve for factors up to order max_m
// whose columns hold at most kmax_entries band entries
static int bs_k(int kmax_entries) { return (kmax_entries + 31) / 32; }
static size_t bs_per_warp(int max_m, int K) { return (size_t)max_m * 16 + (size_t)BS_PF * 32 * K * 8; }
static int bs_wpc(int max_m, int K) {
    size_t pw = bs_per_warp(max_m, K);
    int w = (int)((200 * 1024) / pw);
    return w < 1 ? 1 : (w > 4 ? 4 : w);
}

template <int K>
static void bs_launch(const Task *tasks, int ntasks, const BandFactor *shapes, const double *Lall,
                      const double *Uall, const int *Iall, const double *Rall, const double2 *in,
                      double2 *out, int use_fine, const int *flag, int max_m, cudaStream_t s) {
    const int wpc = bs_wpc(max_m, K);
    const int grid = (2 * ntasks + wpc - 1) / wpc;
    k_band_solve<K><<<grid, 32 * wpc, bs_per_warp(max_m, K) * wpc, s>>>(
        tasks, ntasks, shapes, Lall, Uall, Iall, Rall, in, out, use_fine, flag, max_m);
}

void launch_band_solve(const Task *tasks, int ntasks, const BandFactor *shapes, const double *Lall,
                       const double *Uall, const int *Iall, const double *Rall, const double2 *in,
                       double2 *out, int use_fine_offsets, const int *flag, int max_m,
                       int kmax_entries, cudaStream_t s) {
    switch (bs_k(kmax_entries)) {
        case 1: bs_launch<1>(tasks, ntasks, shapes, Lall, Uall, Iall, Rall, in, out, use_fine_offsets, flag, max_m, s); break;
        case 2: bs_launch<2>(tasks, ntasks, shapes, Lall, Uall, Iall, Rall, in, out, use_fine_offsets, flag, max_m, s); break;
        case 3: bs_launch<3>(tasks, ntasks, shapes, Lall, Uall, Iall, Rall, in, out, use_fine_offsets, flag, max_m, s); break;
        case 4: bs_launch<4>(tasks, ntasks, shapes, Lall, Uall, Iall, Rall, in, out, use_fine_offsets, flag, max_m, s); break;
        case 5: case 6: bs_launch<6>(tasks, ntasks, shapes, Lall, Uall, Iall, Rall, in, out, use_fine_offsets, flag, max_m, s); break;
        default: bs_launch<8>(tasks, ntasks, shapes, Lall, Uall, Iall, Rall, in, out, use_fine_offsets, flag, max_m, s); break;
    }
}
// Opt the solve kernels into the shared memory they need; returns an error if one warp's
// share does not fit.
cudaError_t set_band_solve_smem(int max_m, int kmax_entries) {
    const int K = bs_k(kmax_entries);
    if (K > BS_KMAX) return cudaErrorInvalidValue;
    const size_t bytes = bs_per_warp(max_m, K) * bs_wpc(max_m, K);
    if (bytes > 227 * 1024) return cudaErrorInvalidValue;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_band_solve<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_band_solve<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_band_solve<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_band_solve<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_band_solve<6>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes)) != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_band_solve<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace hdd
