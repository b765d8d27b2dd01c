// kernels_cgrid.cu — the grid coarse space of the two-level RAS variant (the conclusions, §4,
// name a coarse space as the next step): restriction Pᵀ and interpolation P between the fine
// interior nodes and the P1 nodes of the mesh of spacing H = c·h (same diagonal direction), and
// A_H⁻¹ for the lumped coarse operator A_H = K_H - k²H² I through the 2D sine transform.
//
// Layouts: fine vectors complex128, (N-1)² interior nodes, x fastest, nrhs consecutive vectors
// (stride ldv); coarse vectors m² entries (m = N/c - 1), x fastest, stride ldh.
#include "hdd_common.cuh"

namespace hdd {

// Numerator of the coarse hat function at a fine offset (dx, dy) in fine cells from its node:
// φ = num / c with num = max(0, c - max(|dx|, |dy|, |dx ∓ dy|)) (diag 0: dx - dy, the mesh's
// diagonals run along (1, 1); diag 1: dx + dy, along (1, -1)).
__device__ __forceinline__ int hat_num(int dx, int dy, int c, int diag) {
    const int ad = diag ? abs(dx + dy) : abs(dx - dy);
    const int mx = max(max(abs(dx), abs(dy)), ad);
    return mx < c ? c - mx : 0;
}

// vH = Pᵀ v: a coarse node gathers its (2c-1)² fine neighbours weighted by its hat function
// (all interior nodes for 1 <= I, J <= m), rows of the stencil in increasing fine index.
template <typename T>
__global__ void k_cg_restrict(CGrid g, const double2 *__restrict__ v, c2<T> *__restrict__ vH,
                              long long ldv, long long ldh, const int *__restrict__ active) {
    if (active && !active[blockIdx.y]) return;
    v += blockIdx.y * ldv;
    vH += blockIdx.y * ldh;
    const int m = g.m, c = g.c, w = g.N - 1;
    const long long mm = (long long)m * m;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < mm;
         e += (long long)gridDim.x * blockDim.x) {
        const int I = (int)(e % m) + 1, J = (int)(e / m) + 1;
        double sx = 0.0, sy = 0.0;
        for (int dy = 1 - c; dy < c; dy++) {
            const double2 *row = v + (long long)(c * J + dy - 1) * w + (c * I - 1);
            for (int dx = 1 - c; dx < c; dx++) {
                const int num = hat_num(dx, dy, c, g.diag);
                if (num == 0) continue;
                const double wt = (double)num / c;
                const double2 a = row[dx];
                sx = fma(wt, a.x, sx);
                sy = fma(wt, a.y, sy);
            }
        }
        vH[e] = mk<T>((T)sx, (T)sy);
    }
}

// z = P xH (accumulate = 0) or z += P xH (1): a fine node interpolates the corners of the coarse
// cell that contains it (the corner off its triangle has weight 0; boundary corners hold 0).
template <typename T>
__global__ void k_cg_prolong(CGrid g, const c2<T> *__restrict__ xH, double2 *__restrict__ z, int accumulate,
                             long long ldv, long long ldh, const int *__restrict__ active) {
    if (active && !active[blockIdx.y]) return;
    z += blockIdx.y * ldv;
    xH += blockIdx.y * ldh;
    const int m = g.m, c = g.c, w = g.N - 1;
    const long long n = (long long)w * w;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e % w) + 1, j = (int)(e / w) + 1;
        const int cx0 = i / c, cy0 = j / c;
        double sx = 0.0, sy = 0.0;
        for (int b = 0; b < 2; b++) {
            const int J = cy0 + b;
            if (J < 1 || J > m) continue;
            for (int a = 0; a < 2; a++) {
                const int I = cx0 + a;
                if (I < 1 || I > m) continue;
                const int num = hat_num(i - c * I, j - c * J, c, g.diag);
                if (num == 0) continue;
                const double wt = (double)num / c;
                const c2<T> u = xH[(I - 1) + (long long)(J - 1) * m];
                sx = fma(wt, (double)u.x, sx);
                sy = fma(wt, (double)u.y, sy);
            }
        }
        if (accumulate) {
            double2 o = z[e];
            o.x += sx;
            o.y += sy;
            z[e] = o;
        } else {
            z[e] = make_double2(sx, sy);
        }
    }
}

// One pass of the separable sine transform: out = (S · in)ᵀ, optionally scaled entrywise by
// Dinv, for an m x m complex matrix `in` (row j, column x) and the real symmetric S:
// out[x][i] = Dinv[x][i] · Σ_j S[i][j] in[j][x].  Two passes give S X S; the solve is
// A_H⁻¹ Y = S (D⁻¹ ∘ (S Y S)) S (S orthonormal and symmetric, D symmetric), four passes.
// CTA: a DT x DT output tile, the j range in chunks of DKC staged in shared memory (coalesced
// along x for `in` and along i for S, which is read as S[j][i] = S[i][j]); each of the 128
// threads accumulates 2 rows x 4 columns (i = i0 + ti + 8q, x = x0 + tx + 16p).
constexpr int DT = 32, DKC = 32, DTHREADS = 128;
template <typename T>
__global__ void __launch_bounds__(DTHREADS)
k_dst_pass(int m, long long ldh, const T *__restrict__ S, const T *__restrict__ Dinv,
           const c2<T> *__restrict__ in, c2<T> *__restrict__ out, const int *__restrict__ active) {
    if (active && !active[blockIdx.z]) return;
    in += blockIdx.z * ldh;
    out += blockIdx.z * ldh;
    __shared__ c2<T> Xs[DKC][DT];
    __shared__ T Ss[DKC][DT];
    const int tid = threadIdx.x, ti = tid & 7, tx = tid >> 3;
    const int i0 = blockIdx.x * DT, x0 = blockIdx.y * DT;
    c2<T> acc[2][4];
#pragma unroll
    for (int p = 0; p < 2; p++)
#pragma unroll
        for (int q = 0; q < 4; q++) acc[p][q] = mk<T>((T)0, (T)0);
    for (int j0 = 0; j0 < m; j0 += DKC) {
        for (int e = tid; e < DKC * DT; e += DTHREADS) {
            const int kk = e / DT, cc = e % DT, j = j0 + kk;
            const bool okj = j < m;
            Xs[kk][cc] = (okj && x0 + cc < m) ? in[(long long)j * m + x0 + cc] : mk<T>((T)0, (T)0);
            Ss[kk][cc] = (okj && i0 + cc < m) ? S[(long long)j * m + i0 + cc] : (T)0;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < DKC; kk++) {
            T sv[4];
            c2<T> xv[2];
#pragma unroll
            for (int q = 0; q < 4; q++) sv[q] = Ss[kk][ti + 8 * q];
#pragma unroll
            for (int p = 0; p < 2; p++) xv[p] = Xs[kk][tx + 16 * p];
#pragma unroll
            for (int p = 0; p < 2; p++)
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    acc[p][q].x = fma(sv[q], xv[p].x, acc[p][q].x);
                    acc[p][q].y = fma(sv[q], xv[p].y, acc[p][q].y);
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int p = 0; p < 2; p++) {
        const int x = x0 + tx + 16 * p;
        if (x >= m) continue;
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int i = i0 + ti + 8 * q;
            if (i >= m) continue;
            c2<T> r = acc[p][q];
            if (Dinv) {
                const T d = Dinv[(long long)x * m + i];
                r.x *= d;
                r.y *= d;
            }
            out[(long long)x * m + i] = r;
        }
    }
}

template <typename TI, typename TO>
__global__ void k_cg_convert(long long n, const TI *__restrict__ in, TO *__restrict__ out) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        const TI a = in[e];
        TO b;
        b.x = a.x;
        b.y = a.y;
        out[e] = b;
    }
}

static int cg_grid(long long n) {
    long long g = (n + 255) / 256;
    if (g > 8 * 152) g = 8 * 152;
    return g < 1 ? 1 : (int)g;
}

template <typename T>
void launch_cg_restrict(const CGrid &g, const double2 *v, c2<T> *vH, int nrhs, long long ldv, long long ldh,
                        const int *active, cudaStream_t s) {
    k_cg_restrict<T><<<dim3(cg_grid((long long)g.m * g.m), nrhs), 256, 0, s>>>(g, v, vH, ldv, ldh, active);
}
template <typename T>
void launch_cg_prolong(const CGrid &g, const c2<T> *xH, double2 *z, int accumulate, int nrhs, long long ldv,
                       long long ldh, const int *active, cudaStream_t s) {
    const long long n = (long long)(g.N - 1) * (g.N - 1);
    k_cg_prolong<T><<<dim3(cg_grid(n), nrhs), 256, 0, s>>>(g, xH, z, accumulate, ldv, ldh, active);
}
template <typename T>
void launch_dst_pass(int m, const T *S, const T *Dinv, const c2<T> *in, c2<T> *out, int nrhs, long long ldh,
                     const int *active, cudaStream_t s) {
    const int t = (m + DT - 1) / DT;
    k_dst_pass<T><<<dim3(t, t, nrhs), DTHREADS, 0, s>>>(m, ldh, S, Dinv, in, out, active);
}
void launch_cg_widen(long long n, const float2 *in, double2 *out, cudaStream_t s) {
    k_cg_convert<float2, double2><<<cg_grid(n), 256, 0, s>>>(n, in, out);
}
void launch_cg_narrow(long long n, const double2 *in, float2 *out, cudaStream_t s) {
    k_cg_convert<double2, float2><<<cg_grid(n), 256, 0, s>>>(n, in, out);
}

template void launch_cg_restrict<float>(const CGrid &, const double2 *, float2 *, int, long long, long long,
                                        const int *, cudaStream_t);
template void launch_cg_restrict<double>(const CGrid &, const double2 *, double2 *, int, long long, long long,
                                         const int *, cudaStream_t);
template void launch_cg_prolong<float>(const CGrid &, const float2 *, double2 *, int, int, long long, long long,
                                       const int *, cudaStream_t);
template void launch_cg_prolong<double>(const CGrid &, const double2 *, double2 *, int, int, long long, long long,
                                        const int *, cudaStream_t);
template void launch_dst_pass<float>(int, const float *, const float *, const float2 *, float2 *, int, long long,
                                     const int *, cudaStream_t);
template void launch_dst_pass<double>(int, const double *, const double *, const double2 *, double2 *, int,
                                      long long, const int *, cudaStream_t);

}  // namespace hdd
