// kernels_cnn.cu — the learned warm start: a 4-layer 3x3 convolutional network (32 channels,
// BF16 weights, FP32 accumulation) mapping a restricted subdomain right-hand side to an initial
// guess for its deflated GMRES, with its training kernels (backward passes and Adam).
//
// Images are the solver's tasks: task t is an nx x ny image stored channels-last at pixel
// offsets Task::foff (activation index (foff + y·nx + x)·C + c).  Zero padding at the box edge
// matches the zero Dirichlet values around a subdomain.
#include "hdd_common.cuh"

#include <cuda_bf16.h>

namespace hdd {

constexpr int CT = 256;                    // threads per conv CTA

__device__ __forceinline__ float bf2f(__nv_bfloat16 v) { return __bfloat162float(v); }

// Per-task scale σ_t = sqrt(mean |f̃|²) (one CTA per task) and the input image
// (Re f̃/σ, Im f̃/σ, k·h, 0).
template <typename R>
__global__ void __launch_bounds__(CT)
k_cnn_input(const Task *__restrict__ tasks, const c2<R> *__restrict__ f, float kh,
            float *__restrict__ sigma, float *__restrict__ X0, float2 *__restrict__ Fh) {
    __shared__ float red[CT / 32];
    __shared__ float sig_s;
    const Task T = tasks[blockIdx.x];
    const int n = T.nx * T.ny;
    float s = 0.f;
    for (int i = threadIdx.x; i < n; i += CT) {
        const c2<R> v = f[T.foff + i];
        s = fmaf((float)v.x, (float)v.x, fmaf((float)v.y, (float)v.y, s));
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int q = 0; q < CT / 32; q++) t += red[q];
        float sg = sqrtf(t / (float)n);
        sig_s = sg > 0.f ? sg : 1.f;
        sigma[blockIdx.x] = sig_s;
    }
    __syncthreads();
    const float inv = 1.f / sig_s;
    for (int i = threadIdx.x; i < n; i += CT) {
        const c2<R> v = f[T.foff + i];
        float4 o = make_float4((float)v.x * inv, (float)v.y * inv, kh, 0.f);
        reinterpret_cast<float4 *>(X0)[T.foff + i] = o;
        if (Fh) Fh[T.foff + i] = make_float2(o.x, o.y);
    }
}

// Y = conv3x3(X) + b, optionally ReLU; one fine tile per CTA, one output pixel per thread step,
// all COUT channels accumulated in registers; weights (BF16 → FP32) staged in shared memory.
template <int CIN, int COUT, bool RELU>
__global__ void __launch_bounds__(CT)
k_conv_fwd(const Task *__restrict__ tasks, const Tile *__restrict__ tiles,
           const __nv_bfloat16 *__restrict__ Wb, const float *__restrict__ bias,
           const float *__restrict__ X, float *__restrict__ Y) {
    __shared__ float Ws[COUT * 9 * CIN];
    __shared__ float Bs[COUT];
    for (int i = threadIdx.x; i < COUT * 9 * CIN; i += CT) Ws[i] = bf2f(Wb[i]);
    for (int i = threadIdx.x; i < COUT; i += CT) Bs[i] = bias[i];
    __syncthreads();
    const Tile tl = tiles[blockIdx.x];
    const Task T = tasks[tl.task];
    const int nx = T.nx, ny = T.ny;
    for (int e = threadIdx.x; e < tl.nr * nx; e += CT) {
        const int y = tl.r0 + e / nx, x = e % nx;
        float acc[COUT];
#pragma unroll
        for (int c = 0; c < COUT; c++) acc[c] = Bs[c];
#pragma unroll
        for (int k = 0; k < 9; k++) {
            const int yy = y + k / 3 - 1, xx = x + k % 3 - 1;
            if (yy < 0 || yy >= ny || xx < 0 || xx >= nx) continue;
            const float4 *xp = reinterpret_cast<const float4 *>(X + (T.foff + (long long)yy * nx + xx) * CIN);
#pragma unroll
            for (int c4 = 0; c4 < CIN / 4; c4++) {
                const float4 v = __ldg(xp + c4);
#pragma unroll
                for (int co = 0; co < COUT; co++) {
                    const float *w = Ws + (co * 9 + k) * CIN + 4 * c4;
                    acc[co] = fmaf(w[0], v.x, fmaf(w[1], v.y, fmaf(w[2], v.z, fmaf(w[3], v.w, acc[co]))));
                }
            }
        }
        float *yp = Y + (T.foff + (long long)y * nx + x) * COUT;
#pragma unroll
        for (int co = 0; co < COUT; co++) yp[co] = RELU ? fmaxf(acc[co], 0.f) : acc[co];
    }
}

// dX[p][ci] = Σ_k Σ_co W[co][k][ci] dY'[p - d_k][co], dY' = dY masked by the ReLU of the
// layer's output (act_out > 0) when act_out is given.
template <int CIN, int COUT>
__global__ void __launch_bounds__(CT)
k_conv_bwd_data(const Task *__restrict__ tasks, const Tile *__restrict__ tiles,
                const __nv_bfloat16 *__restrict__ Wb, const float *__restrict__ dY,
                const float *__restrict__ act_out, float *__restrict__ dX) {
    __shared__ float Ws[COUT * 9 * CIN];
    for (int i = threadIdx.x; i < COUT * 9 * CIN; i += CT) Ws[i] = bf2f(Wb[i]);
    __syncthreads();
    const Tile tl = tiles[blockIdx.x];
    const Task T = tasks[tl.task];
    const int nx = T.nx, ny = T.ny;
    for (int e = threadIdx.x; e < tl.nr * nx; e += CT) {
        const int y = tl.r0 + e / nx, x = e % nx;
        float acc[CIN];
#pragma unroll
        for (int c = 0; c < CIN; c++) acc[c] = 0.f;
#pragma unroll
        for (int k = 0; k < 9; k++) {
            // output pixel q with q + d_k = p
            const int yy = y - (k / 3 - 1), xx = x - (k % 3 - 1);
            if (yy < 0 || yy >= ny || xx < 0 || xx >= nx) continue;
            const long long q = T.foff + (long long)yy * nx + xx;
#pragma unroll
            for (int co = 0; co < COUT; co++) {
                float g = dY[q * COUT + co];
                if (act_out && !(act_out[q * COUT + co] > 0.f)) g = 0.f;
                const float *w = Ws + (co * 9 + k) * CIN;
#pragma unroll
                for (int ci = 0; ci < CIN; ci++) acc[ci] = fmaf(w[ci], g, acc[ci]);
            }
        }
        float *xp = dX + (T.foff + (long long)y * nx + x) * CIN;
#pragma unroll
        for (int ci = 0; ci < CIN; ci++) xp[ci] = acc[ci];
    }
}

// Partial weight gradients of one fine tile (deterministic: every weight is summed by one
// thread in pixel order):
//   part[tile][(co·9 + k)·CIN + ci] = Σ_q dY'[q][co] X[q + d_k][ci],  part[tile][W + co] = Σ_q dY'[q][co].
template <int CIN, int COUT>
__global__ void __launch_bounds__(CT)
k_conv_bwd_w(const Task *__restrict__ tasks, const Tile *__restrict__ tiles,
             const float *__restrict__ dY, const float *__restrict__ act_out,
             const float *__restrict__ X, float *__restrict__ part) {
    constexpr int NW = COUT * 9 * CIN;
    const Tile tl = tiles[blockIdx.x];
    const Task T = tasks[tl.task];
    const int nx = T.nx, ny = T.ny;
    float *mine = part + (long long)blockIdx.x * (NW + COUT);
    for (int w = threadIdx.x; w < NW + COUT; w += CT) {
        float acc = 0.f;
        if (w < NW) {
            const int co = w / (9 * CIN), k = (w / CIN) % 9, ci = w % CIN;
            const int dy = k / 3 - 1, dx = k % 3 - 1;
            for (int e = 0; e < tl.nr * nx; e++) {
                const int y = tl.r0 + e / nx, x = e % nx;
                const int yy = y + dy, xx = x + dx;
                if (yy < 0 || yy >= ny || xx < 0 || xx >= nx) continue;
                const long long q = T.foff + (long long)y * nx + x;
                if (act_out && !(act_out[q * COUT + co] > 0.f)) continue;
                acc = fmaf(dY[q * COUT + co], X[(T.foff + (long long)yy * nx + xx) * CIN + ci], acc);
            }
        } else {
            const int co = w - NW;
            for (int e = 0; e < tl.nr * nx; e++) {
                const long long q = T.foff + (long long)(tl.r0 + e / nx) * nx + e % nx;
                if (act_out && !(act_out[q * COUT + co] > 0.f)) continue;
                acc += dY[q * COUT + co];
            }
        }
        mine[w] = acc;
    }
}

// grad[w] = scale · Σ_tile part[tile][w] (fixed tile order)
__global__ void k_sum_partials(const float *__restrict__ part, int ntiles, int nw, float scale,
                               float *__restrict__ grad) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= nw) return;
    float s = 0.f;
    for (int t = 0; t < ntiles; t++) s += part[(long long)t * nw + w];
    grad[w] = s * scale;
}

// Residual of the guess in normalised units, r = f̃/σ - A (a + i b) (A real, zero outside the
// box), from the input image X0 (channels 0, 1) and the network output Y4 (2 channels); per-tile
// partial Σ|r|²/n_t.
__global__ void __launch_bounds__(CT)
k_cnn_resid(const Task *__restrict__ tasks, const Tile *__restrict__ tiles, Stencil st,
            const float *__restrict__ X0, const float *__restrict__ Y4, float *__restrict__ Rr,
            float *__restrict__ lpart) {
    __shared__ float red[CT / 32];
    const Tile tl = tiles[blockIdx.x];
    const Task T = tasks[tl.task];
    const int nx = T.nx, ny = T.ny;
    const float c0 = (float)st.c0, c1 = (float)st.c1, c2v = (float)st.c2;
    float s = 0.f;
    for (int e = threadIdx.x; e < tl.nr * nx; e += CT) {
        const int y = tl.r0 + e / nx, x = e % nx;
        auto U = [&](int xx, int yy) -> float2 {
            if (xx < 0 || xx >= nx || yy < 0 || yy >= ny) return make_float2(0.f, 0.f);
            return reinterpret_cast<const float2 *>(Y4)[T.foff + (long long)yy * nx + xx];
        };
        const float2 cc = U(x, y), ee = U(x + 1, y), ww = U(x - 1, y), nn = U(x, y + 1), ss = U(x, y - 1);
        float2 d1, d2;
        if (st.diag == 0) { d1 = U(x + 1, y + 1); d2 = U(x - 1, y - 1); }
        else { d1 = U(x + 1, y - 1); d2 = U(x - 1, y + 1); }
        const long long p = T.foff + (long long)y * nx + x;
        const float4 in = reinterpret_cast<const float4 *>(X0)[p];
        float2 r;
        r.x = in.x - (c0 * cc.x + c1 * (((ee.x + ww.x) + nn.x) + ss.x) + c2v * (d1.x + d2.x));
        r.y = in.y - (c0 * cc.y + c1 * (((ee.y + ww.y) + nn.y) + ss.y) + c2v * (d1.y + d2.y));
        reinterpret_cast<float2 *>(Rr)[p] = r;
        s = fmaf(r.x, r.x, fmaf(r.y, r.y, s));
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int q = 0; q < CT / 32; q++) t += red[q];
        lpart[blockIdx.x] = t / (float)(nx * ny);
    }
}

// dL/d(a, b) = scale_t · A v (A real symmetric, so Aᵀ = A) for the vector v of the loss.
__global__ void __launch_bounds__(CT)
k_cnn_out_grad(const Task *__restrict__ tasks, const Tile *__restrict__ tiles, Stencil st,
               const float *__restrict__ Rr, const float *__restrict__ scale, float *__restrict__ dY4) {
    const Tile tl = tiles[blockIdx.x];
    const Task T = tasks[tl.task];
    const int nx = T.nx, ny = T.ny;
    const float c0 = (float)st.c0, c1 = (float)st.c1, c2v = (float)st.c2;
    const float sc = scale[tl.task];
    for (int e = threadIdx.x; e < tl.nr * nx; e += CT) {
        const int y = tl.r0 + e / nx, x = e % nx;
        auto U = [&](int xx, int yy) -> float2 {
            if (xx < 0 || xx >= nx || yy < 0 || yy >= ny) return make_float2(0.f, 0.f);
            return reinterpret_cast<const float2 *>(Rr)[T.foff + (long long)yy * nx + xx];
        };
        const float2 cc = U(x, y), ee = U(x + 1, y), ww = U(x - 1, y), nn = U(x, y + 1), ss = U(x, y - 1);
        float2 d1, d2;
        if (st.diag == 0) { d1 = U(x + 1, y + 1); d2 = U(x - 1, y - 1); }
        else { d1 = U(x + 1, y - 1); d2 = U(x - 1, y + 1); }
        float2 g;
        g.x = sc * (c0 * cc.x + c1 * (((ee.x + ww.x) + nn.x) + ss.x) + c2v * (d1.x + d2.x));
        g.y = sc * (c0 * cc.y + c1 * (((ee.y + ww.y) + nn.y) + ss.y) + c2v * (d1.y + d2.y));
        reinterpret_cast<float2 *>(dY4)[T.foff + (long long)y * nx + x] = g;
    }
}

// Loss of the batch: L = mean_t ||P r_t||² / ||P f̂_t||², f̂ = f̃/σ, r = f̂ - A(a + i b) (the
// relative deflated residual the local GMRES starts from).  scale_t = -2 / (ntask ||P f̂_t||²)
// from the per-tile partial norms of P f̂ (slot LDP-1 of each tile's partial-sum block).
__global__ void k_cnn_task_scale(const Task *__restrict__ tasks, int ntask, const float2 *__restrict__ p3f,
                                 float *__restrict__ scale) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntask) return;
    const Task T = tasks[t];
    float s = 0.f;
    for (int q = 0; q < T.ntiles; q++) s += p3f[(long long)(T.tile0 + q) * LOCAL_LDP + LOCAL_LDP - 1].x;
    scale[t] = s > 0.f ? -2.f / ((float)ntask * s) : 0.f;
}
__global__ void k_cnn_task_loss(const Task *__restrict__ tasks, int ntask, const float2 *__restrict__ p3r,
                                const float2 *__restrict__ p3f, float *__restrict__ loss) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntask) return;
    const Task T = tasks[t];
    float a = 0.f, b = 0.f;
    for (int q = 0; q < T.ntiles; q++) {
        a += p3r[(long long)(T.tile0 + q) * LOCAL_LDP + LOCAL_LDP - 1].x;
        b += p3f[(long long)(T.tile0 + q) * LOCAL_LDP + LOCAL_LDP - 1].x;
    }
    loss[t] = b > 0.f ? a / b : 0.f;
}

// x0 = σ_t (a + i b) into the packed local iterate (precision R)
template <typename R>
__global__ void k_cnn_output(const Task *__restrict__ tasks, const Tile *__restrict__ tiles,
                             const float *__restrict__ sigma, const float *__restrict__ Y4,
                             c2<R> *__restrict__ x0, const int *__restrict__ flag) {
    const Tile tl = tiles[blockIdx.x];
    if (flag && !flag[tl.task]) return;
    const Task T = tasks[tl.task];
    const float sg = sigma[tl.task];
    for (int e = threadIdx.x; e < tl.nr * T.nx; e += blockDim.x) {
        const long long p = T.foff + (long long)tl.r0 * T.nx + e;
        const float2 v = reinterpret_cast<const float2 *>(Y4)[p];
        x0[p] = mk<R>((R)(sg * v.x), (R)(sg * v.y));
    }
}

// Adam on the FP32 master weights (Kingma & Ba 2015), then the BF16 copy used by the kernels.
__global__ void k_adam(int n, float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, __nv_bfloat16 *__restrict__ pb, float lr, float b1,
                       float b2, float eps, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi; v[i] = vi;
    const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = pi;
    pb[i] = __float2bfloat16(pi);
}

__global__ void k_to_bf16(int n, const float *__restrict__ p, __nv_bfloat16 *__restrict__ pb) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) pb[i] = __float2bfloat16(p[i]);
}

// ------------------------------------------------------------------------------------------
// launchers
// ------------------------------------------------------------------------------------------
template <typename R>
void launch_cnn_input(const Task *tasks, int ntasks, const c2<R> *f, float kh, float *sigma, float *X0,
                      float2 *Fh, cudaStream_t s) {
    k_cnn_input<R><<<ntasks, CT, 0, s>>>(tasks, f, kh, sigma, X0, Fh);
}
void launch_cnn_task_scale(const Task *tasks, int ntasks, const float2 *p3f, float *scale, cudaStream_t s) {
    k_cnn_task_scale<<<(ntasks + 127) / 128, 128, 0, s>>>(tasks, ntasks, p3f, scale);
}
void launch_cnn_task_loss(const Task *tasks, int ntasks, const float2 *p3r, const float2 *p3f, float *loss,
                          cudaStream_t s) {
    k_cnn_task_loss<<<(ntasks + 127) / 128, 128, 0, s>>>(tasks, ntasks, p3r, p3f, loss);
}
template <typename R>
void launch_cnn_output(const Task *tasks, const Tile *tiles, int ntiles, const float *sigma,
                       const float *Y4, c2<R> *x0, const int *flag, cudaStream_t s) {
    k_cnn_output<R><<<ntiles, 256, 0, s>>>(tasks, tiles, sigma, Y4, x0, flag);
}
void launch_conv_fwd(int layer, const Task *tasks, const Tile *tiles, int ntiles, const __nv_bfloat16 *W,
                     const float *b, const float *X, float *Y, cudaStream_t s) {
    switch (layer) {
        case 0: k_conv_fwd<4, 32, true><<<ntiles, CT, 0, s>>>(tasks, tiles, W, b, X, Y); break;
        case 1:
        case 2: k_conv_fwd<32, 32, true><<<ntiles, CT, 0, s>>>(tasks, tiles, W, b, X, Y); break;
        default: k_conv_fwd<32, 2, false><<<ntiles, CT, 0, s>>>(tasks, tiles, W, b, X, Y); break;
    }
}
void launch_conv_bwd_data(int layer, const Task *tasks, const Tile *tiles, int ntiles,
                          const __nv_bfloat16 *W, const float *dY, const float *act_out, float *dX,
                          cudaStream_t s) {
    switch (layer) {
        case 1:
        case 2: k_conv_bwd_data<32, 32><<<ntiles, CT, 0, s>>>(tasks, tiles, W, dY, act_out, dX); break;
        case 3: k_conv_bwd_data<32, 2><<<ntiles, CT, 0, s>>>(tasks, tiles, W, dY, act_out, dX); break;
        default: break;                       // the input image needs no gradient
    }
}
void launch_conv_bwd_w(int layer, const Task *tasks, const Tile *tiles, int ntiles, const float *dY,
                       const float *act_out, const float *X, float *part, cudaStream_t s) {
    switch (layer) {
        case 0: k_conv_bwd_w<4, 32><<<ntiles, CT, 0, s>>>(tasks, tiles, dY, act_out, X, part); break;
        case 1:
        case 2: k_conv_bwd_w<32, 32><<<ntiles, CT, 0, s>>>(tasks, tiles, dY, act_out, X, part); break;
        default: k_conv_bwd_w<32, 2><<<ntiles, CT, 0, s>>>(tasks, tiles, dY, act_out, X, part); break;
    }
}
void launch_sum_partials(const float *part, int ntiles, int nw, float scale, float *grad, cudaStream_t s) {
    k_sum_partials<<<(nw + 255) / 256, 256, 0, s>>>(part, ntiles, nw, scale, grad);
}
void launch_cnn_resid(const Task *tasks, const Tile *tiles, int ntiles, const Stencil &st, const float *X0,
                      const float *Y4, float *Rr, float *lpart, cudaStream_t s) {
    k_cnn_resid<<<ntiles, CT, 0, s>>>(tasks, tiles, st, X0, Y4, Rr, lpart);
}
void launch_cnn_out_grad(const Task *tasks, const Tile *tiles, int ntiles, const Stencil &st, const float *Rr,
                         const float *scale, float *dY4, cudaStream_t s) {
    k_cnn_out_grad<<<ntiles, CT, 0, s>>>(tasks, tiles, st, Rr, scale, dY4);
}
void launch_adam(int n, float *p, const float *g, float *m, float *v, __nv_bfloat16 *pb, float lr, float b1,
                 float b2, float eps, int step, cudaStream_t s) {
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    k_adam<<<(n + 255) / 256, 256, 0, s>>>(n, p, g, m, v, pb, lr, b1, b2, eps, c1, c2);
}
void launch_to_bf16(int n, const float *p, __nv_bfloat16 *pb, cudaStream_t s) {
    k_to_bf16<<<(n + 255) / 256, 256, 0, s>>>(n, p, pb);
}

template void launch_cnn_input<float>(const Task *, int, const float2 *, float, float *, float *, float2 *, cudaStream_t);
template void launch_cnn_input<double>(const Task *, int, const double2 *, float, float *, float *, float2 *, cudaStream_t);
template void launch_cnn_output<float>(const Task *, const Tile *, int, const float *, const float *, float2 *, const int *, cudaStream_t);
template void launch_cnn_output<double>(const Task *, const Tile *, int, const float *, const float *, double2 *, const int *, cudaStream_t);

}  // namespace hdd
