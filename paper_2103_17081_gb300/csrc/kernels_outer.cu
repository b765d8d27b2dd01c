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
constexpr int OCH = 2048;               // largest chunk one CTA owns (staged in shared memory)
// CTAs of the chunked reductions over a vector of n entries
int outer_grid(long long n) {
    long long g = (n + OCH - 1) / OCH;
    return (int)(g > OUTER_CTAS ? g : OUTER_CTAS);
}

// y = A x (f == nullptr) or y = f - A x on the (N-1)² interior grid, zero Dirichlet values.
__global__ void k_gstencil(Stencil st, int N, const double2 *__restrict__ x, double2 *__restrict__ y,
                           const double2 *__restrict__ f) {
    const int w = N - 1;
    const long long n = (long long)w * w;
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
        r.x = st.c0 * c.x + st.c1 * (((e.x + wv.x) + nn.x) + s.x) + st.c2 * (d1.x + d2.x);
        r.y = st.c0 * c.y + st.c1 * (((e.y + wv.y) + nn.y) + s.y) + st.c2 * (d1.y + d2.y);
        if (f) { double2 fv = f[i]; r.x = fv.x - r.x; r.y = fv.y - r.y; }
        y[i] = r;
    }
}

// Load vector F = Σ amp·e_c (point sources snapped to the nearest interior node) + Σ M g
// (Gaussian bumps, g the nodal values at interior nodes, M the P1 mass matrix
// h²/12 · [6 centre; 1 at E, W, N, S and the two diagonal corners]).
__global__ void k_build_rhs(int N, double h, int diag, int npts, const double *__restrict__ pts,
                            int nb, const double *__restrict__ bumps, double2 *__restrict__ f) {
    const int w = N - 1;
    const long long n = (long long)w * w;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int gi = (int)(i % w) + 1, gj = (int)(i / w) + 1;
        double v = 0.0;
        for (int p = 0; p < npts; p++) {
            int pi = (int)floor(pts[3 * p] * N + 0.5), pj = (int)floor(pts[3 * p + 1] * N + 0.5);
            pi = pi < 1 ? 1 : (pi > N - 1 ? N - 1 : pi);
            pj = pj < 1 ? 1 : (pj > N - 1 ? N - 1 : pj);
            if (pi == gi && pj == gj) v += pts[3 * p + 2];
        }
        for (int b = 0; b < nb; b++) {
            const double cx = bumps[4 * b], cy = bumps[4 * b + 1], sg = bumps[4 * b + 2], amp = bumps[4 * b + 3];
            auto g = [&](int a, int c) -> double {
                if (a < 1 || a > N - 1 || c < 1 || c > N - 1) return 0.0;
                double dx = a * h - cx, dy = c * h - cy;
                return amp * exp(-(dx * dx + dy * dy) / (2.0 * sg * sg));
            };
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

// Each CTA owns one contiguous chunk of the vectors (at most OCH entries).  The chunk of w is
// staged in shared memory once; then warp q of the CTA forms the partial dots of vectors
// l = q, q + 8, ... over the chunk with shuffle reductions only (no block barrier per vector).

__device__ __forceinline__ void warp_dots(const double2 *__restrict__ V, long long ld, int nv,
                                          const double2 *__restrict__ ws, long long b, int len,
                                          double2 *__restrict__ part, int ldp) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int l = warp; l < nv; l += OT / 32) {
        const double2 *vl = V + (long long)l * ld + b;
        double2 a0 = make_double2(0.0, 0.0), a1 = make_double2(0.0, 0.0);
        int i = lane;
        for (; i + 32 < len; i += 64) {
            cdotc_acc<double>(a0, vl[i], ws[i]);
            cdotc_acc<double>(a1, vl[i + 32], ws[i + 32]);
        }
        if (i < len) cdotc_acc<double>(a0, vl[i], ws[i]);
        a0.x += a1.x; a0.y += a1.y;
        for (int o = 16; o > 0; o >>= 1) { a0.x += shfl_xor(a0.x, o); a0.y += shfl_xor(a0.y, o); }
        if (lane == 0) part[(long long)blockIdx.x * ldp + l] = a0;
    }
}

// Partial dots part[cta][l] = Σ_{chunk} conj(V_l) w, l < nv.
__global__ void __launch_bounds__(OT)
k_odots(const double2 *__restrict__ V, long long ld, int nv, const double2 *__restrict__ w,
        long long n, double2 *__restrict__ part, int ldp) {
    __shared__ double2 ws[OCH];
    long long b, e;
    chunk_of(n, b, e);
    const int len = (int)(e > b ? e - b : 0);
    for (int i = threadIdx.x; i < len; i += OT) ws[i] = w[b + i];
    __syncthreads();
    warp_dots(V, ld, nv, ws, b, len, part, ldp);
}

// w -= Σ_l h_l V_l; then (part_dots != null) partial dots V^H w, else partial ||w||².
__global__ void __launch_bounds__(OT)
k_oupdate(const double2 *__restrict__ V, long long ld, int nv, const double2 *__restrict__ h,
          double2 *__restrict__ w, long long n, double2 *__restrict__ part_dots, int ldp,
          double *__restrict__ part_norm) {
    extern __shared__ double2 hs[];
    __shared__ double2 ws[OCH];
    __shared__ double red[OT / 32];
    long long b, e;
    chunk_of(n, b, e);
    const int len = (int)(e > b ? e - b : 0);
    for (int l = threadIdx.x; l < nv; l += OT) hs[l] = h[l];
    __syncthreads();
    double nrm = 0.0;
    for (int i = threadIdx.x; i < len; i += OT) {
        double2 x0 = w[b + i], x1 = make_double2(0.0, 0.0);
        const double2 *vp = V + b + i;
        int l = 0;
        for (; l + 1 < nv; l += 2) {                // two independent accumulation chains
            caxpy_neg<double>(x0, hs[l], vp[(long long)l * ld]);
            caxpy_neg<double>(x1, hs[l + 1], vp[(long long)(l + 1) * ld]);
        }
        if (l < nv) caxpy_neg<double>(x0, hs[l], vp[(long long)l * ld]);
        x0.x += x1.x; x0.y += x1.y;
        w[b + i] = x0;
        ws[i] = x0;
        nrm = fma(x0.x, x0.x, fma(x0.y, x0.y, nrm));
    }
    if (part_dots) {
        __syncthreads();
        warp_dots(V, ld, nv, ws, b, len, part_dots, ldp);
    } else {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        for (int o = 16; o > 0; o >>= 1) nrm += shfl_xor(nrm, o);
        if (lane == 0) red[warp] = nrm;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int q = 0; q < OT / 32; q++) s += red[q];
            part_norm[blockIdx.x] = s;
        }
    }
}

// Partial ||x||² per CTA.
__global__ void __launch_bounds__(OT) k_onorm(const double2 *__restrict__ x, long long n, double *__restrict__ part) {
    __shared__ double red[OT / 32];
    long long b, e;
    chunk_of(n, b, e);
    double s = 0.0;
    for (long long i = b + threadIdx.x; i < e; i += OT) s = fma(x[i].x, x[i].x, fma(x[i].y, x[i].y, s));
    for (int o = 16; o > 0; o >>= 1) s += shfl_xor(s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < OT / 32; q++) t += red[q];
        part[blockIdx.x] = t;
    }
}

// out[l] = Σ_q part[q][l]: one warp per l, lane i adds q = i, i+32, ... in order, then a fixed
// shuffle tree (deterministic).
__global__ void k_oreduce(const double2 *__restrict__ part, int nparts, int ldp, int nv, double2 *__restrict__ out) {
    const int l = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (l >= nv) return;
    double2 s = make_double2(0.0, 0.0);
    for (int q = lane; q < nparts; q += 32) { double2 v = part[(long long)q * ldp + l]; s.x += v.x; s.y += v.y; }
    for (int o = 16; o > 0; o >>= 1) { s.x += shfl_xor(s.x, o); s.y += shfl_xor(s.y, o); }
    if (lane == 0) out[l] = s;
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

// Outer Arnoldi column j: h = h1 + h2 (CGS2), h_{j+1,j} = sqrt(Σ norm partials); rotate with the
// previous rotations, form rotation j, update g; flag = 1 while |g_{j+1}| > tol_abs and hn > 0.
__global__ void k_ogivens(double2 *__restrict__ H, long long ldh, double *__restrict__ cs,
                          double2 *__restrict__ sn, double2 *__restrict__ g, int j,
                          const double2 *__restrict__ h1, const double2 *__restrict__ h2,
                          const double *__restrict__ npart, int nparts, double tol_abs,
                          double *__restrict__ hn_out, int *__restrict__ flag,
                          double *__restrict__ hist, double fnorm) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s2 = 0.0;
    for (int q = 0; q < nparts; q++) s2 += npart[q];
    const double hn = sqrt(s2);
    double2 *hc = H + (long long)j * ldh;
    for (int l = 0; l <= j; l++) hc[l] = make_double2(h1[l].x + h2[l].x, h1[l].y + h2[l].y);
    for (int l = 0; l < j; l++) {
        double2 x = hc[l], y = hc[l + 1], sx = sn[l];
        double2 a = cmul<double>(sx, y);
        double2 bq = cmul<double>(make_double2(sx.x, -sx.y), x);
        hc[l] = make_double2(cs[l] * x.x + a.x, cs[l] * x.y + a.y);
        hc[l + 1] = make_double2(cs[l] * y.x - bq.x, cs[l] * y.y - bq.y);
    }
    double c; double2 s, r;
    zgivens(hc[j], make_double2(hn, 0.0), c, s, r);
    cs[j] = c; sn[j] = s;
    hc[j] = r;
    double2 gj = g[j];
    g[j + 1] = make_double2(-(s.x * gj.x + s.y * gj.y), -(s.x * gj.y - s.y * gj.x));
    g[j] = make_double2(c * gj.x, c * gj.y);
    const double res = hypot(g[j + 1].x, g[j + 1].y);
    *hn_out = hn;
    *hist = res / fnorm;                       // caller passes the slot of this iteration
    *flag = (res > tol_abs && hn > 0.0) ? 1 : 0;
}

// out = w / hn (hn read from device memory)
__global__ void k_oscale(double2 *__restrict__ out, const double2 *__restrict__ w, const double *__restrict__ hn, long long n) {
    const double h = *hn;
    if (!(h > 0.0)) return;
    const double inv = 1.0 / h;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = make_double2(w[i].x * inv, w[i].y * inv);
}

// y = H(0:k,0:k)⁻¹ g by column-oriented back substitution (one CTA).
__global__ void k_otrisolve(const double2 *__restrict__ H, long long ldh, const double2 *__restrict__ g,
                            int k, double2 *__restrict__ y) {
    extern __shared__ double2 rhs[];
    for (int i = threadIdx.x; i < k; i += blockDim.x) rhs[i] = g[i];
    __syncthreads();
    for (int i = k - 1; i >= 0; i--) {
        const double2 d = H[(long long)i * ldh + i];
        const double2 si = rhs[i];
        const double den = d.x * d.x + d.y * d.y;
        const double2 yi = make_double2((si.x * d.x + si.y * d.y) / den, (si.y * d.x - si.x * d.y) / den);
        __syncthreads();
        for (int r = threadIdx.x; r < i; r += blockDim.x) caxpy_neg<double>(rhs[r], yi, H[(long long)i * ldh + r]);
        if (threadIdx.x == 0) y[i] = yi;
        __syncthreads();
    }
}

// x += Σ_{l<k} y_l Z_l
__global__ void k_oaxpy(const double2 *__restrict__ y, int k, const double2 *__restrict__ Zb, long long ld,
                        double2 *__restrict__ x, long long n) {
    extern __shared__ double2 ys[];
    for (int l = threadIdx.x; l < k; l += blockDim.x) ys[l] = y[l];
    __syncthreads();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double2 acc = x[i];
        for (int l = 0; l < k; l++) caxpy<double>(acc, ys[l], Zb[(long long)l * ld + i]);
        x[i] = acc;
    }
}

// Cycle start: β = sqrt(Σ partials), v0 = r/β, g = [β, 0, ..., 0] (R+1 entries).
__global__ void k_oinit(const double2 *__restrict__ r, long long n, const double *__restrict__ npart,
                        int nparts, double2 *__restrict__ v0, double2 *__restrict__ g, int R,
                        double *__restrict__ beta_out) {
    __shared__ double beta_s;
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int q = 0; q < nparts; q++) s += npart[q];
        beta_s = sqrt(s);
        if (blockIdx.x == 0) *beta_out = beta_s;
    }
    __syncthreads();
    const double beta = beta_s;
    if (blockIdx.x == 0)
        for (int l = threadIdx.x; l <= R; l += blockDim.x) g[l] = make_double2(l == 0 ? beta : 0.0, 0.0);
    if (!(beta > 0.0)) return;
    const double inv = 1.0 / beta;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        v0[i] = make_double2(r[i].x * inv, r[i].y * inv);
}

static int grid_for(long long n, int threads) {
    long long g = (n + threads - 1) / threads;
    if (g > 8 * 152) g = 8 * 152;
    return g < 1 ? 1 : (int)g;
}

void launch_gstencil(const Stencil &st, int N, const double2 *x, double2 *y, const double2 *f, cudaStream_t s) {
    long long n = (long long)(N - 1) * (N - 1);
    k_gstencil<<<grid_for(n, 256), 256, 0, s>>>(st, N, x, y, f);
}
void launch_build_rhs(int N, double h, int diag, int npts, const double *pts, int nb, const double *bumps,
                      double2 *f, cudaStream_t s) {
    long long n = (long long)(N - 1) * (N - 1);
    k_build_rhs<<<grid_for(n, 256), 256, 0, s>>>(N, h, diag, npts, pts, nb, bumps, f);
}
void launch_odots(const double2 *V, long long ld, int nv, const double2 *w, long long n, double2 *part,
                  int ldp, cudaStream_t s) {
    k_odots<<<outer_grid(n), OT, 0, s>>>(V, ld, nv, w, n, part, ldp);
}
void launch_oupdate(const double2 *V, long long ld, int nv, const double2 *h, double2 *w, long long n,
                    double2 *part_dots, int ldp, double *part_norm, cudaStream_t s) {
    k_oupdate<<<outer_grid(n), OT, (size_t)nv * sizeof(double2), s>>>(V, ld, nv, h, w, n, part_dots, ldp, part_norm);
}
void launch_onorm(const double2 *x, long long n, double *part, cudaStream_t s) {
    k_onorm<<<outer_grid(n), OT, 0, s>>>(x, n, part);
}
void launch_oreduce(const double2 *part, int nparts, int ldp, int nv, double2 *out, cudaStream_t s) {
    k_oreduce<<<(nv + 7) / 8, 256, 0, s>>>(part, nparts, ldp, nv, out);
}
void launch_ogivens(double2 *H, long long ldh, double *cs, double2 *sn, double2 *g, int j, const double2 *h1,
                    const double2 *h2, const double *npart, int nparts, double tol_abs, double *hn_out, int *flag,
                    double *hist, double fnorm, cudaStream_t s) {
    k_ogivens<<<1, 32, 0, s>>>(H, ldh, cs, sn, g, j, h1, h2, npart, nparts, tol_abs, hn_out, flag, hist, fnorm);
}
void launch_oscale(double2 *out, const double2 *w, const double *hn, long long n, cudaStream_t s) {
    k_oscale<<<grid_for(n, 256), 256, 0, s>>>(out, w, hn, n);
}
void launch_otrisolve(const double2 *H, long long ldh, const double2 *g, int k, double2 *y, cudaStream_t s) {
    k_otrisolve<<<1, 256, (size_t)k * sizeof(double2), s>>>(H, ldh, g, k, y);
}
void launch_oaxpy(const double2 *y, int k, const double2 *Zb, long long ld, double2 *x, long long n, cudaStream_t s) {
    k_oaxpy<<<grid_for(n, 256), 256, (size_t)k * sizeof(double2), s>>>(y, k, Zb, ld, x, n);
}
void launch_oinit(const double2 *r, long long n, const double *npart, double2 *v0, double2 *g, int R,
                  double *beta_out, cudaStream_t s) {
    k_oinit<<<grid_for(n, 256), 256, 0, s>>>(r, n, npart, outer_grid(n), v0, g, R, beta_out);
}
cudaError_t set_outer_smem_limits(size_t bytes) {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_oupdate, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_otrisolve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_oaxpy, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes)) != cudaSuccess) return e;
    return cudaSuccess;
}

}  // namespace hdd
