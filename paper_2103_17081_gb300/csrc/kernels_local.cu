// kernels_local.cu — batched kernels of the inner deflated GMRES (§2 Eq. 4–5, §3), one CTA per
// tile of one task, every task of every subdomain (and right-hand side) in one launch.
//
// Fine tiles cover up to LocalArgs::frows box rows of one task (frows·nx <= LOCAL_THREADS·EPT);
// coarse tiles cover up to LocalArgs::crows coarse rows.  Kernels read each tile's height from the
// tile table; the host sizes shared memory for the largest heights.
// Reductions are two-stage and deterministic: each tile writes its partial sums to a slot of
// its own, and every consumer adds the partials of a task in tile order.
#include "hdd_common.cuh"

namespace hdd {

constexpr int LDP = MAX_RESTART + 2;     // partial-sum slots per tile
constexpr int EPT = FINE_EPT;            // fine elements per thread (frows*max_nx <= 2048)
constexpr int NWARP = LOCAL_THREADS / 32;

// 1D Bézier deflation weight (Eq. 5 factor): fine node f, coarse node c (0-based); column c is
// centred on fine node 2c+1 with weights (1,4,6,4,1)/8 on f = 2c-1 .. 2c+3.
__device__ __forceinline__ float zw_f(int t) {
    return t == 0 || t == 4 ? 0.125f : (t == 2 ? 0.75f : 0.5f);
}
template <typename R> __device__ __forceinline__ R zw(int t) { return (R)zw_f(t); }

template <typename R> __device__ __forceinline__ c2<R> load_c(const c2<R> *p) { return *p; }

// Row of a boundary node (impedance condition): Σ_q cf[q] v_q over the 7 stencil slots.
template <typename R>
__device__ __forceinline__ c2<R> boundary_row(const double2 *__restrict__ cf, c2<R> v0, c2<R> v1, c2<R> v2,
                                           c2<R> v3, c2<R> v4, c2<R> v5, c2<R> v6) {
    const c2<R> v[7] = {v0, v1, v2, v3, v4, v5, v6};
    c2<R> r = mk<R>(0, 0);
#pragma unroll
    for (int q = 0; q < 7; q++) {
        const double2 a = cf[q];
        r = cadd<R>(r, cmul<R>(mk<R>((R)a.x, (R)a.y), v[q]));
    }
    return r;
}

// w = A u at local (x, y) from a shared-memory row buffer u[rows][nx] whose row 0 is box row
// `ybase`; rows outside [0, ny) and columns outside [0, nx) are zero (Dirichlet around the box).
// (gx0, gy0): mesh node of the box's local (0, 0); under the impedance condition the rows of
// nodes on the boundary of the square take their class's complex coefficients.
// IMP: compiled for the impedance condition (the Dirichlet instantiation carries no boundary code).
template <typename R, bool IMP>
__device__ __forceinline__ c2<R> stencil_smem(const Stencil &st, const c2<R> *u, int ybase,
                                              int nrows, int nx, int ny, int x, int y, int gx0, int gy0) {
    const R c0 = (R)st.c0, c1 = (R)st.c1, c2v = (R)st.c2;
    auto U = [&](int xx, int yy) -> c2<R> {
        if (xx < 0 || xx >= nx || yy < 0 || yy >= ny) return mk<R>(0, 0);
        int r = yy - ybase;
        if (r < 0 || r >= nrows) return mk<R>(0, 0);
        return u[r * nx + xx];
    };
    c2<R> cc = U(x, y);
    c2<R> e = U(x + 1, y), wv = U(x - 1, y), n = U(x, y + 1), s = U(x, y - 1);
    c2<R> d1, d2;
    if (st.diag == 0) { d1 = U(x + 1, y + 1); d2 = U(x - 1, y - 1); }
    else { d1 = U(x + 1, y - 1); d2 = U(x - 1, y + 1); }
    c2<R> r;
    if (IMP) {
        const int cls = node_class(st.N, gx0 + x, gy0 + y);
        if (cls != 4) return boundary_row<R>(st.bcoef + cls * 7, cc, e, wv, n, s, d1, d2);
    }
    r.x = c0 * cc.x + c1 * (((e.x + wv.x) + n.x) + s.x) + c2v * (d1.x + d2.x);
    r.y = c0 * cc.y + c1 * (((e.y + wv.y) + n.y) + s.y) + c2v * (d1.y + d2.y);
    return r;
}

// Block reduction of `nv` complex partial sums held by every thread (acc computed per l by
// the caller through `get`), written to out[0..nv).
template <typename R, typename F>
__device__ void block_reduce_many(int nv, F get, c2<R> *red /*[NWARP][LDP]*/, c2<R> *out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int l = 0; l < nv; l++) {
        c2<R> a = get(l);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) { a.x += shfl_xor(a.x, o); a.y += shfl_xor(a.y, o); }
        if (lane == 0) red[warp * LDP + l] = a;
    }
    __syncthreads();
    for (int l = threadIdx.x; l < nv; l += blockDim.x) {
        c2<R> s = mk<R>(0, 0);
        for (int q = 0; q < NWARP; q++) s = cadd<R>(s, red[q * LDP + l]);
        out[l] = s;
    }
}

template <typename R> __device__ R block_sum(R v, R *red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += shfl_xor(v, o);
    if (lane == 0) red[warp] = v;
    __syncthreads();
    R s = 0;
    if (threadIdx.x == 0)
        for (int q = 0; q < NWARP; q++) s += red[q];
    return s;
}

// ------------------------------------------------------------------------------------------
// restriction f̃_j = R_j v (Eq. 3), global complex128 → packed local precision R
// ------------------------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(LOCAL_THREADS)
k_restrict(LocalArgs<R> a, int gw, long long nglob, const double2 *__restrict__ glob,
           c2<R> *__restrict__ out, const int *__restrict__ flag) {
    const Tile tl = a.ftiles[blockIdx.x];
    if (flag && !flag[tl.task]) return;
    const Task T = a.tasks[tl.task];
    const int cnt = tl.nr * T.nx;
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
        int y = tl.r0 + e / T.nx, x = e % T.nx;
        long long gi = (long long)(T.ix0 + x - a.glo) + (long long)(T.iy0 + y - a.glo) * gw +
                       (long long)T.rhs * nglob;
        double2 v = glob[gi];
        out[T.foff + (long long)y * T.nx + x] = mk<R>((R)v.x, (R)v.y);
    }
}

// z = Σ_j R_jᵀ D_j x_j: every owned node is written by exactly one task (no atomics).
template <typename R>
__global__ void __launch_bounds__(LOCAL_THREADS)
k_scatter(LocalArgs<R> a, int gw, long long nglob, const c2<R> *__restrict__ x,
          double2 *__restrict__ glob, const int *__restrict__ flag) {
    const Tile tl = a.ftiles[blockIdx.x];
    if (flag && !flag[tl.task]) return;
    const Task T = a.tasks[tl.task];
    const int cnt = tl.nr * T.nx;
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
        int y = tl.r0 + e / T.nx, xx = e % T.nx;
        int gx = T.ix0 + xx, gy = T.iy0 + y;
        if (gx < T.ox0 || gx > T.ox1 || gy < T.oy0 || gy > T.oy1) continue;
        c2<R> v = x[T.foff + (long long)y * T.nx + xx];
        glob[(long long)(gx - a.glo) + (long long)(gy - a.glo) * gw + (long long)T.rhs * nglob] =
            make_double2((double)v.x, (double)v.y);
    }
}

// out = A_j in   or   out = f - A_j in   (fine tiles, neighbours read through L1)
template <typename R, bool IMP>
__global__ void __launch_bounds__(LOCAL_THREADS)
k_local_A(LocalArgs<R> a, const c2<R> *__restrict__ in, c2<R> *__restrict__ out,
          const c2<R> *__restrict__ f, const int *__restrict__ flag) {
    extern __shared__ unsigned char smem_raw[];
    c2<R> *u = reinterpret_cast<c2<R> *>(smem_raw);
    const Tile tl = a.ftiles[blockIdx.x];
    if (flag && !flag[tl.task]) return;
    const Task T = a.tasks[tl.task];
    const int y0 = tl.r0 - 1, nrows = tl.nr + 2;
    for (int e = threadIdx.x; e < nrows * T.nx; e += blockDim.x) {
        int yy = y0 + e / T.nx, xx = e % T.nx;
        u[e] = (yy >= 0 && yy < T.ny) ? in[T.foff + (long long)yy * T.nx + xx] : mk<R>(0, 0);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < tl.nr * T.nx; e += blockDim.x) {
        int y = tl.r0 + e / T.nx, x = e % T.nx;
        c2<R> w = stencil_smem<R, IMP>(a.st, u, y0, nrows, T.nx, T.ny, x, y, T.ix0, T.iy0);
        long long gi = T.foff + (long long)y * T.nx + x;
        if (f) w = csub<R>(f[gi], w);
        out[gi] = w;
    }
}

// y = Z_jᵀ t (coarse tiles), with t = A_j in (apply_A) or t = in; y in FP64.
template <typename R, bool IMP>
__global__ void __launch_bounds__(LOCAL_THREADS)
k_zt(LocalArgs<R> a, const c2<R> *__restrict__ in, double2 *__restrict__ yout, int apply_A,
     const int *__restrict__ flag) {
    extern __shared__ unsigned char smem_raw[];
    const Tile tl = a.ctiles[blockIdx.x];
    if (flag && !flag[tl.task]) return;
    const Task T = a.tasks[tl.task];
    const int nx = T.nx, ny = T.ny, mx = T.mx;
    // fine rows feeding coarse rows [r0, r0+nr): 2c-1 .. 2c+3
    const int F0 = 2 * tl.r0 - 1, F1 = 2 * (tl.r0 + tl.nr - 1) + 3;
    const int nF = F1 - F0 + 1;                    // 2*nr + 3
    const int V0 = F0 - 1, nV = nF + 2;            // input rows for the stencil
    c2<R> *vin = reinterpret_cast<c2<R> *>(smem_raw);
    c2<R> *t = vin + (apply_A ? nV * nx : 0);
    c2<R> *sx = t + nF * nx;
    if (apply_A) {
        for (int e = threadIdx.x; e < nV * nx; e += blockDim.x) {
            int yy = V0 + e / nx, xx = e % nx;
            vin[e] = (yy >= 0 && yy < ny) ? in[T.foff + (long long)yy * nx + xx] : mk<R>(0, 0);
        }
        __syncthreads();
        for (int e = threadIdx.x; e < nF * nx; e += blockDim.x) {
            int yy = F0 + e / nx, xx = e % nx;
            t[e] = (yy >= 0 && yy < ny) ? stencil_smem<R, IMP>(a.st, vin, V0, nV, nx, ny, xx, yy, T.ix0, T.iy0)
                                        : mk<R>(0, 0);
        }
    } else {
        for (int e = threadIdx.x; e < nF * nx; e += blockDim.x) {
            int yy = F0 + e / nx, xx = e % nx;
            t[e] = (yy >= 0 && yy < ny) ? in[T.foff + (long long)yy * nx + xx] : mk<R>(0, 0);
        }
    }
    __syncthreads();
    // x-direction: sx[f][cx] = Σ_a w_a t[f][2cx-1+a]
    for (int e = threadIdx.x; e < nF * mx; e += blockDim.x) {
        int fr = e / mx, cx = e % mx;
        c2<R> s = mk<R>(0, 0);
#pragma unroll
        for (int q = 0; q < 5; q++) {
            int fx = 2 * cx - 1 + q;
            if (fx >= 0 && fx < nx) {
                c2<R> v = t[fr * nx + fx];
                s.x = fma(zw<R>(q), v.x, s.x);
                s.y = fma(zw<R>(q), v.y, s.y);
            }
        }
        sx[e] = s;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < tl.nr * mx; e += blockDim.x) {
        int cy = tl.r0 + e / mx, cx = e % mx;
        c2<R> s = mk<R>(0, 0);
#pragma unroll
        for (int q = 0; q < 5; q++) {
            int fy = 2 * cy - 1 + q;
            if (fy >= 0 && fy < ny) {
                c2<R> v = sx[(fy - F0) * mx + cx];
                s.x = fma(zw<R>(q), v.x, s.x);
                s.y = fma(zw<R>(q), v.y, s.y);
            }
        }
        yout[T.coff + (long long)cy * mx + cx] = make_double2((double)s.x, (double)s.y);
    }
}

// Z s for box rows [F0, F0+nF): s (FP64 coarse) → px (x-interpolated coarse rows) → zs.
// Shared buffers: sc[ncy*mx], px[ncy*nx].  Returns via zs[nF*nx].
template <typename R>
__device__ void prolong_rows(const Task &T, const double2 *__restrict__ s, int F0, int nF,
                             c2<R> *sc, c2<R> *px, c2<R> *zs) {
    const int nx = T.nx, ny = T.ny, mx = T.mx, my = T.my;
    // coarse rows cy with 2cy-1 <= f <= 2cy+3 for some f in [F0, F0+nF)
    int C0 = (F0 - 3) >= 0 ? (F0 - 3 + 1) / 2 : -((3 - F0) / 2);
    int C1 = (F0 + nF - 1 + 1) / 2;
    if (C0 < 0) C0 = 0;
    if (C1 > my - 1) C1 = my - 1;
    const int ncy = C1 - C0 + 1;
    const BoxDiv dmx(mx), dnx(nx);
    for (int e = threadIdx.x; e < ncy * mx; e += blockDim.x) {
        const int rr = dmx.q(e);
        double2 v = s[T.coff + (long long)(C0 + rr) * mx + (e - rr * mx)];
        sc[e] = mk<R>((R)v.x, (R)v.y);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < ncy * nx; e += blockDim.x) {
        const int r = dnx.q(e), fx = e - r * nx;
        c2<R> acc = mk<R>(0, 0);
        int cx0 = (fx - 3) >= 0 ? (fx - 3 + 1) / 2 : 0;
        int cx1 = (fx + 1) / 2;
        if (cx1 > mx - 1) cx1 = mx - 1;
        for (int cx = cx0; cx <= cx1; cx++) {
            R wgt = zw<R>(fx - 2 * cx + 1);
            c2<R> v = sc[r * mx + cx];
            acc.x = fma(wgt, v.x, acc.x);
            acc.y = fma(wgt, v.y, acc.y);
        }
        px[e] = acc;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nF * nx; e += blockDim.x) {
        const int qy = dnx.q(e);
        int fy = F0 + qy, fx = e - qy * nx;
        c2<R> acc = mk<R>(0, 0);
        if (fy >= 0 && fy < ny) {
            int cy0 = (fy - 3) >= 0 ? (fy - 3 + 1) / 2 : 0;
            int cy1 = (fy + 1) / 2;
            if (cy1 > my - 1) cy1 = my - 1;
            for (int cy = cy0; cy <= cy1; cy++) {
                R wgt = zw<R>(fy - 2 * cy + 1);
                c2<R> v = px[(cy - C0) * nx + fx];
                acc.x = fma(wgt, v.x, acc.x);
                acc.y = fma(wgt, v.y, acc.y);
            }
        }
        zs[e] = acc;
    }
    __syncthreads();
}

__host__ __device__ inline int prolong_max_cy(int nrows_fine) { return nrows_fine / 2 + 4; }

// out = add + Z s on fine tiles (add may be null)
template <typename R>
__global__ void __launch_bounds__(LOCAL_THREADS)
k_z(LocalArgs<R> a, const double2 *__restrict__ s, const c2<R> *__restrict__ add,
    c2<R> *__restrict__ out, const int *__restrict__ flag, R sign) {
    extern __shared__ unsigned char smem_raw[];
    const Tile tl = a.ftiles[blockIdx.x];
    if (flag && !flag[tl.task]) return;
    const Task T = a.tasks[tl.task];
    const int maxc = prolong_max_cy(tl.nr);
    c2<R> *sc = reinterpret_cast<c2<R> *>(smem_raw);
    c2<R> *px = sc + maxc * T.mx;
    c2<R> *zs = px + maxc * T.nx;
    prolong_rows<R>(T, s, tl.r0, tl.nr, sc, px, zs);
    for (int e = threadIdx.x; e < tl.nr * T.nx; e += blockDim.x) {
        long long gi = T.foff + (long long)tl.r0 * T.nx + e;
        c2<R> v = cscale<R>(sign, zs[e]);
        if (add) v = cadd<R>(add[gi], v);
        out[gi] = v;
    }
}

// Arnoldi (mode 0): out = A (in - Z s), partial dots V_l^H out (l < nv);
// residual (mode 1): out = in - A (Z s), partial ||out||².
template <typename R, bool IMP>
__global__ void __launch_bounds__(LOCAL_THREADS)
k_prolong_stencil(LocalArgs<R> a, int mode, const c2<R> *__restrict__ in,
                  const double2 *__restrict__ s, c2<R> *__restrict__ out,
                  const c2<R> *__restrict__ V, int nv, c2<R> *__restrict__ part,
                  const int *__restrict__ flag) {
    extern __shared__ unsigned char smem_raw[];
    const Tile tl = a.ftiles[blockIdx.x];
    if (flag && !flag[tl.task]) return;
    const Task T = a.tasks[tl.task];
    const int nx = T.nx, ny = T.ny;
    const int F0 = tl.r0 - 1, nF = tl.nr + 2;
    const int maxc = prolong_max_cy(nF);
    c2<R> *sc = reinterpret_cast<c2<R> *>(smem_raw);
    c2<R> *px = sc + maxc * T.mx;
    c2<R> *u = px + maxc * nx;                     // nF*nx
    c2<R> *red = u + nF * nx;                      // NWARP*LDP
    prolong_rows<R>(T, s, F0, nF, sc, px, u);      // u = Z s on rows F0..F0+nF-1
    if (mode == 0) {
        for (int e = threadIdx.x; e < nF * nx; e += blockDim.x) {
            int yy = F0 + e / nx;
            if (yy >= 0 && yy < ny) u[e] = csub<R>(in[T.foff + (long long)yy * nx + e % nx], u[e]);
        }
        __syncthreads();
    }
    c2<R> wv[EPT];
    const int cnt = tl.nr * nx;
    R nrm = 0;
#pragma unroll
    for (int k = 0; k < EPT; k++) {
        int e = threadIdx.x + k * LOCAL_THREADS;
        wv[k] = mk<R>(0, 0);
        if (e < cnt) {
            int y = tl.r0 + e / nx, x = e % nx;
            c2<R> w = stencil_smem<R, IMP>(a.st, u, F0, nF, nx, ny, x, y, T.ix0, T.iy0);
            long long gi = T.foff + (long long)y * nx + x;
            if (mode == 1) w = csub<R>(in[gi], w);
            out[gi] = w;
            wv[k] = w;
            nrm = fma(w.x, w.x, fma(w.y, w.y, nrm));
        }
    }
    c2<R> *mypart = part + (long long)blockIdx.x * LDP;
    if (mode == 0) {
        const long long base = T.foff + (long long)tl.r0 * nx;
        block_reduce_many<R>(nv, [&](int l) {
            c2<R> acc = mk<R>(0, 0);
            const c2<R> *vl = V + (long long)l * a.ld + base;
#pragma unroll
            for (int k = 0; k < EPT; k++) {
                int e = threadIdx.x + k * LOCAL_THREADS;
                if (e < cnt) cdotc_acc<R>(acc, vl[e], wv[k]);
            }
            return acc;
        }, red, mypart);
    } else {
        R *redr = reinterpret_cast<R *>(red);
        R tot = block_sum<R>(nrm, redr);
        if (threadIdx.x == 0) mypart[LDP - 1] = mk<R>(tot, 0);
    }
}

// Sum over the task's tiles of the squared-norm slot (LDP-1), by one warp: lane q adds tiles
// q, q+32, ..., then a fixed shuffle tree (deterministic); every lane returns the total.
template <typename R>
__device__ __forceinline__ R task_norm2_warp(const c2<R> *part, const Task &T) {
    const int lane = threadIdx.x & 31;
    R s = 0;
    for (int q = lane; q < T.ntiles; q += 32) s += part[(long long)(T.tile0 + q) * LDP + LDP - 1].x;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// Task sums of partial slots l < nv (and, if part2, plus the same slots of part2) into out[l]:
// warp w takes l = w, w + NWARP, ...; its lane q adds tiles q, q+32, ..., then a fixed shuffle
// tree (deterministic).  All tile partials of a slot are loaded at once instead of one after
// another.
template <typename R>
__device__ __forceinline__ void task_sums_warp(const c2<R> *part, const c2<R> *part2, const Task &T, int nv,
                                               c2<R> *out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int l = warp; l < nv; l += NWARP) {
        c2<R> s = mk<R>(0, 0);
        for (int q = lane; q < T.ntiles; q += 32) {
            s = cadd<R>(s, part[(long long)(T.tile0 + q) * LDP + l]);
            if (part2) s = cadd<R>(s, part2[(long long)(T.tile0 + q) * LDP + l]);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) { s.x += shfl_xor(s.x, o); s.y += shfl_xor(s.y, o); }
        if (lane == 0) out[l] = s;
    }
}

// Classical Gram-Schmidt passes 2 and 3 (CGS2): w -= V h (h = task sum of part_in);
// pass 2 also forms the partial dots V^H w, pass 3 the partial ||w||².
template <typename R>
__global__ void __launch_bounds__(LOCAL_THREADS)
k_cgs_update(LocalArgs<R> a, int pass, c2<R> *__restrict__ w, const c2<R> *__restrict__ V, int nv,
             const c2<R> *__restrict__ part_in, c2<R> *__restrict__ part_out,
             const int *__restrict__ flag) {
    __shared__ c2<R> hv[LDP];
    __shared__ c2<R> red[NWARP * LDP];
    const Tile tl = a.ftiles[blockIdx.x];
    if (flag && !flag[tl.task]) return;
    const Task T = a.tasks[tl.task];
    task_sums_warp<R>(part_in, nullptr, T, nv, hv);
    __syncthreads();
    const int cnt = tl.nr * T.nx;
    const long long base = T.foff + (long long)tl.r0 * T.nx;
    c2<R> wv[EPT];
    R nrm = 0;
#pragma unroll
    for (int k = 0; k < EPT; k++) {
        int e = threadIdx.x + k * LOCAL_THREADS;
        wv[k] = mk<R>(0, 0);
        if (e < cnt) {
            c2<R> x = w[base + e];
            for (int l = 0; l < nv; l++) caxpy_neg<R>(x, hv[l], V[(long long)l * a.ld + base + e]);
            w[base + e] = x;
            wv[k] = x;
            nrm = fma(x.x, x.x, fma(x.y, x.y, nrm));
        }
    }
    c2<R> *mypart = part_out + (long long)blockIdx.x * LDP;
    if (pass == 2) {
        block_reduce_many<R>(nv, [&](int l) {
            c2<R> acc = mk<R>(0, 0);
            const c2<R> *vl = V + (long long)l * a.ld + base;
#pragma unroll
            for (int k = 0; k < EPT; k++) {
                int e = threadIdx.x + k * LOCAL_THREADS;
                if (e < cnt) cdotc_acc<R>(acc, vl[e], wv[k]);
            }
            return acc;
        }, red, mypart);
    } else {
        R tot = block_sum<R>(nrm, reinterpret_cast<R *>(red));
        if (threadIdx.x == 0) mypart[LDP - 1] = mk<R>(tot, 0);
    }
}

// Complex Givens rotation G = [c s; -conj(s) c], c real, with G [a; b] = [r; 0] (the standard
// complex form, cf. Bindel, Demmel, Kahan & Marques, ACM TOMS 2002), magnitudes by hypot.
template <typename R>
__device__ void givens(c2<R> a, c2<R> b, R &c, c2<R> &s, c2<R> &r) {
    R aa = hypot(a.x, a.y), bb = hypot(b.x, b.y);
    if (bb == (R)0) { c = 1; s = mk<R>(0, 0); r = a; return; }
    if (aa == (R)0) { c = 0; s = mk<R>(b.x / bb, -b.y / bb); r = mk<R>(bb, 0); return; }
    R t = hypot(aa, bb);
    c2<R> ph = mk<R>(a.x / aa, a.y / aa);
    c = aa / t;
    c2<R> cb = mk<R>(b.x / t, -b.y / t);       // conj(b)/t
    s = cmul<R>(ph, cb);
    r = mk<R>(ph.x * t, ph.y * t);
}

// End of Arnoldi step i: normalise v_{i+1} = w/||w|| (every tile of the task) and, on the
// task's first tile, rotate the new Hessenberg column, update g and test |g_{i+1}| <= tol·ref.
template <typename R>
__global__ void __launch_bounds__(LOCAL_THREADS)
k_givens_normalize(LocalArgs<R> a, InnerState<R> S, int restart, int i, c2<R> *__restrict__ w,
                   const c2<R> *__restrict__ p1, const c2<R> *__restrict__ p2,
                   const c2<R> *__restrict__ p3, const int *__restrict__ act_in,
                   int *__restrict__ act_out, int *__restrict__ counter, R tol, int maxit) {
    __shared__ R hn_s;
    __shared__ c2<R> hsum[LDP];
    const Tile tl = a.ftiles[blockIdx.x];
    if (!act_in[tl.task]) return;
    const Task T = a.tasks[tl.task];
    const bool first = blockIdx.x == T.tile0;          // this tile also updates the task's rotations
    if (threadIdx.x < 32) {
        const R s = task_norm2_warp<R>(p3, T);
        if (threadIdx.x == 0) hn_s = sqrt(s);
    }
    // Hessenberg column entries h_l = (pass 1 + pass 2 dots), one task sum per thread
    if (first) task_sums_warp<R>(p1, p2, T, i + 1, hsum);
    __syncthreads();
    const R hn = hn_s;
    if (hn > (R)0) {
        const R inv = (R)1 / hn;
        const long long base = T.foff + (long long)tl.r0 * T.nx;
        for (int e = threadIdx.x; e < tl.nr * T.nx; e += blockDim.x) {
            c2<R> v = w[base + e];
            w[base + e] = mk<R>(v.x * inv, v.y * inv);
        }
    }
    if (!first || threadIdx.x != 0) return;
    const int t = tl.task;
    c2<R> *H = S.H + (long long)t * (restart + 1) * restart;
    c2<R> *hc = H + (long long)i * (restart + 1);
    R *cs = S.cs + (long long)t * restart;
    c2<R> *sn = S.sn + (long long)t * restart;
    c2<R> *g = S.g + (long long)t * (restart + 1);
    for (int l = 0; l <= i; l++) hc[l] = hsum[l];
    for (int l = 0; l < i; l++) {
        c2<R> x = hc[l], y = hc[l + 1];
        c2<R> sx = sn[l];
        // [c s; -conj(s) c] [x; y]
        hc[l] = cadd<R>(cscale<R>(cs[l], x), cmul<R>(sx, y));
        hc[l + 1] = csub<R>(cscale<R>(cs[l], y), cmul<R>(mk<R>(sx.x, -sx.y), x));
    }
    R c; c2<R> s, r;
    givens<R>(hc[i], mk<R>(hn, 0), c, s, r);
    cs[i] = c; sn[i] = s;
    hc[i] = r;
    hc[i + 1] = mk<R>(0, 0);
    c2<R> gi = g[i];
    g[i + 1] = mk<R>(-(s.x * gi.x + s.y * gi.y), -(s.x * gi.y - s.y * gi.x));   // -conj(s) g_i
    g[i] = cscale<R>(c, gi);
    const int its = S.its[t] + 1;
    S.its[t] = its;
    S.kcols[t] = i + 1;
    const R res = hypot(g[i + 1].x, g[i + 1].y);
    const bool conv = res <= tol * S.ref[t] || !(hn > (R)0);
    const bool stop = conv || its >= maxit || i + 1 >= restart;
    if (conv || its >= maxit) S.conv[t] = 1;
    act_out[t] = stop ? 0 : 1;
    if (!stop) atomicAdd(counter, 1);
}

// Start of a cycle: r = P(f̃ - A u) was written into v0 by k_prolong_stencil (mode 1) with its
// partial norms in p3; normalise, set g = [β, 0, ...] and decide whether Arnoldi is needed.
template <typename R>
__global__ void __launch_bounds__(LOCAL_THREADS)
k_init_cycle(LocalArgs<R> a, InnerState<R> S, int restart, c2<R> *__restrict__ v0,
             const c2<R> *__restrict__ p3, const int *__restrict__ flag, int *__restrict__ act_out,
             int *__restrict__ counter, R tol, int maxit, int set_ref) {
    __shared__ R beta_s;
    const Tile tl = a.ftiles[blockIdx.x];
    if (!flag[tl.task]) return;
    const Task T = a.tasks[tl.task];
    if (threadIdx.x < 32) {
        const R s = task_norm2_warp<R>(p3, T);
        if (threadIdx.x == 0) beta_s = sqrt(s);
    }
    __syncthreads();
    const R beta = beta_s;
    if (beta > (R)0) {
        const R inv = (R)1 / beta;
        const long long base = T.foff + (long long)tl.r0 * T.nx;
        for (int e = threadIdx.x; e < tl.nr * T.nx; e += blockDim.x) {
            c2<R> v = v0[base + e];
            v0[base + e] = mk<R>(v.x * inv, v.y * inv);
        }
    }
    if (blockIdx.x != T.tile0 || threadIdx.x != 0) return;
    const int t = tl.task;
    if (set_ref) S.ref[t] = beta;
    c2<R> *g = S.g + (long long)t * (restart + 1);
    g[0] = mk<R>(beta, 0);
    for (int l = 1; l <= restart; l++) g[l] = mk<R>(0, 0);
    S.kcols[t] = 0;
    const bool done = !(beta > tol * S.ref[t]) || S.its[t] >= maxit;
    if (done) S.conv[t] = 1;
    act_out[t] = done ? 0 : 1;
    if (!done) atomicAdd(counter, 1);
}

// y = H(0:k,0:k)⁻¹ g(0:k) for task t, by one thread (k <= restart <= 64).
template <typename R>
__device__ void solve_small(const InnerState<R> &S, int restart, int t, int k, c2<R> *y) {
    const c2<R> *H = S.H + (long long)t * (restart + 1) * restart;
    const c2<R> *g = S.g + (long long)t * (restart + 1);
    for (int r = k - 1; r >= 0; r--) {
        c2<R> sacc = g[r];
        for (int l = r + 1; l < k; l++) sacc = csub<R>(sacc, cmul<R>(H[(long long)l * (restart + 1) + r], y[l]));
        c2<R> d = H[(long long)r * (restart + 1) + r];
        R den = d.x * d.x + d.y * d.y;
        y[r] = mk<R>((sacc.x * d.x + sacc.y * d.y) / den, (sacc.y * d.x - sacc.x * d.y) / den);
    }
}

// Coarse part of the completion x = ũ + Z E⁻¹ Zᵀ(f̃ - A ũ): with ũ = ũ₀ + V y, linearity gives
// E⁻¹ Zᵀ(f̃ - A ũ) = s₀ - Σ_i y_i s_{i+1}, where s₀ = E⁻¹ Zᵀ(f̃ - A ũ₀) was solved at the start of
// the cycle and s_{i+1} = E⁻¹ Zᵀ A v_i in Arnoldi step i (slots of sbuf, stride ldc).
template <typename R>
__global__ void __launch_bounds__(LOCAL_THREADS)
k_coarse_combine(LocalArgs<R> a, InnerState<R> S, int restart, const double2 *__restrict__ sbuf,
                 double2 *__restrict__ sc, const int *__restrict__ flag) {
    __shared__ c2<R> y[MAX_RESTART];
    const Tile tl = a.ctiles[blockIdx.x];
    if (flag && !flag[tl.task]) return;
    const Task T = a.tasks[tl.task];
    const int k = S.kcols[tl.task];
    if (threadIdx.x == 0) solve_small<R>(S, restart, tl.task, k, y);
    __syncthreads();
    for (int e = threadIdx.x; e < tl.nr * T.mx; e += blockDim.x) {
        const long long idx = T.coff + (long long)tl.r0 * T.mx + e;
        double2 acc = sbuf[idx];
        for (int l = 0; l < k; l++) {
            const double2 sv = sbuf[(long long)(l + 1) * a.ldc + idx];
            const double yr = (double)y[l].x, yi = (double)y[l].y;
            acc.x -= yr * sv.x - yi * sv.y;
            acc.y -= yr * sv.y + yi * sv.x;
        }
        sc[idx] = acc;
    }
}

// u += V y with y = H⁻¹ g (each tile solves the small triangle itself); the first tile of a
// task flags it for another cycle when it neither converged nor ran out of iterations.
template <typename R>
__global__ void __launch_bounds__(LOCAL_THREADS)
k_update_u(LocalArgs<R> a, InnerState<R> S, int restart, c2<R> *__restrict__ u,
           const c2<R> *__restrict__ V, const int *__restrict__ flag, int *__restrict__ rs_out,
           int *__restrict__ counter, int maxit) {
    __shared__ c2<R> y[MAX_RESTART];
    const Tile tl = a.ftiles[blockIdx.x];
    if (!flag[tl.task]) return;
    const Task T = a.tasks[tl.task];
    const int t = tl.task;
    const int k = S.kcols[t];
    if (threadIdx.x == 0) {
        solve_small<R>(S, restart, t, k, y);
        if (blockIdx.x == T.tile0) {
            const bool again = !S.conv[t] && S.its[t] < maxit;
            rs_out[t] = again ? 1 : 0;
            if (again) atomicAdd(counter, 1);
        }
    }
    __syncthreads();
    if (k == 0) return;
    const long long base = T.foff + (long long)tl.r0 * T.nx;
    for (int e = threadIdx.x; e < tl.nr * T.nx; e += blockDim.x) {
        c2<R> x = u[base + e];
        for (int l = 0; l < k; l++) caxpy<R>(x, y[l], V[(long long)l * a.ld + base + e]);
        u[base + e] = x;
    }
}

// ref_t = ||P f̃_t|| from the per-tile partial norms of P f̃ (one thread per task); used when
// the cycle starts from a non-zero initial guess.
template <typename R>
__global__ void k_set_ref(LocalArgs<R> a, InnerState<R> S, const c2<R> *__restrict__ p3,
                          const int *__restrict__ flag) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.ntasks || (flag && !flag[t])) return;
    const Task T = a.tasks[t];
    R s = 0;
    for (int q = 0; q < T.ntiles; q++) s += p3[(long long)(T.tile0 + q) * LDP + LDP - 1].x;
    S.ref[t] = sqrt(s);
}

template <typename RI, typename RO>
__global__ void k_cast(long long n, const c2<RI> *__restrict__ in, c2<RO> *__restrict__ out) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = mk<RO>((RO)in[i].x, (RO)in[i].y);
}

// ------------------------------------------------------------------------------------------
// One inner Arnoldi step in one launch (every phase between two coarse solves), one cluster of
// C CTAs per task: CTA `rank` holds box rows [rank·ny/C, (rank+1)·ny/C) and coarse rows
// [rank·my/C, (rank+1)·my/C).  The new vector w stays in registers from the stencil to the
// normalisation; the three task-wide sums (first CGS dots, second CGS dots, ||w||²) are
// all-gathered through distributed shared memory, one cluster barrier each, and every CTA adds
// the C partials in rank order (deterministic, bitwise the same in every CTA).  Steps:
//   A  w = A_j(v_i - Z_j s_{i+1}) (s_{i+1} = E_j⁻¹ Z_jᵀ A_j v_i from the coarse solve), h1 = V^H w
//   B  w -= V h1, h2 = V^H w          (CGS2, both passes against V_0..V_i)
//   C  w -= V h2, ||w||
//   D  v_{i+1} = w/||w||; Hessenberg column h1 + h2, Givens rotation, stop test (every CTA
//      computes the same decision; rank 0 writes the state)
//   E  if the task goes on: y = Z_jᵀ A_j v_{i+1} for the next step's coarse solve (after a
//      cluster barrier that publishes v_{i+1})
// ------------------------------------------------------------------------------------------
constexpr int STEP_CMAX = 8;                       // largest cluster (portable size)

template <typename R> struct StepArgs {
    const Task *tasks;
    Stencil st;
    long long ld;
    int C;                  // CTAs per task (cluster size)
    int i;                  // Arnoldi index
    int restart;
    c2<R> *V;               // basis, vector l at V + l·ld
    const double2 *s;       // s_{i+1} (coarse, FP64)
    double2 *y;             // out: Zᵀ A v_{i+1}
    InnerState<R> S;
    const int *act_in;
    int *act_out;
    int *counter;
    R tol;
    int maxit;
};

__device__ __forceinline__ unsigned cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;\n" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cluster_barrier() {
    asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}
// generic address of the same shared-memory object in CTA `rank` of the cluster
template <typename T> __device__ __forceinline__ T *cluster_map(T *p, unsigned rank) {
    uint64_t out;
    asm volatile("mapa.u64 %0, %1, %2;\n" : "=l"(out) : "l"(reinterpret_cast<uint64_t>(p)), "r"(rank));
    return reinterpret_cast<T *>(out);
}

size_t step_smem_bytes(int max_nx, int max_ny, int C, int bytes_per_c) {
    const int nr = (max_ny + C - 1) / C, nF = nr + 2, maxc = nF / 2 + 4;
    const int mx = max_nx / 2 + 1, my = max_ny / 2;
    const int ncy = (my + C - 1) / C, nFz = 2 * ncy + 3, nVz = nFz + 2;
    const size_t a = (size_t)maxc * mx + (size_t)maxc * max_nx + (size_t)nF * max_nx;
    const size_t e = (size_t)nVz * max_nx + (size_t)nFz * max_nx + (size_t)nFz * mx;
    return (a > e ? a : e) * bytes_per_c;
}

template <typename R, bool IMP>
__global__ void __launch_bounds__(LOCAL_THREADS)
k_arnoldi_step(StepArgs<R> a) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ c2<R> red[NWARP * LDP];            // per-warp partials
    __shared__ c2<R> gat[2][STEP_CMAX][LDP];      // cluster all-gather slots (written remotely)
    __shared__ c2<R> h1s[LDP], h2s[LDP], nrm_s[1];   // task sums: the two CGS passes, ||w||²
    __shared__ R cs_s[MAX_RESTART];
    __shared__ c2<R> sn_s[MAX_RESTART];
    __shared__ c2<R> g_s;
    __shared__ R ref_s, hn_s;
    __shared__ int its_s, stop_s;
    const int C = a.C;
    const int t = (int)blockIdx.x / C;
    const unsigned rank = cluster_rank();
    if (!a.act_in[t]) return;                     // the same flag for every CTA of the cluster
    const Task T = a.tasks[t];
    const int nx = T.nx, ny = T.ny, mx = T.mx, my = T.my;
    const BoxDiv dnx(nx), dmx(mx);
    const int i = a.i, nv = i + 1;
    const int r0 = (int)(rank * ny) / C, r1 = (int)((rank + 1) * ny) / C, nr = r1 - r0;
    const int cnt = nr * nx;
    const long long base = T.foff + (long long)r0 * nx;
    const int tid = threadIdx.x;
    // Givens state of earlier steps (written by earlier launches; rank 0 rewrites it below, after
    // every CTA has passed the first cluster barrier)
    if (tid < i) {
        cs_s[tid] = a.S.cs[(long long)t * a.restart + tid];
        sn_s[tid] = a.S.sn[(long long)t * a.restart + tid];
    }
    if (tid == 0) {
        g_s = a.S.g[(long long)t * (a.restart + 1) + i];
        ref_s = a.S.ref[t];
        its_s = a.S.its[t];
    }
    // ---- A: u = v_i - Z s on rows [r0-1, r1], w = A u on own rows, partial h1 ----
    c2<R> *sc = reinterpret_cast<c2<R> *>(smem_raw);
    const int F0 = r0 - 1, nF = nr + 2, maxc = prolong_max_cy(nF);
    c2<R> *px = sc + maxc * mx;
    c2<R> *u = px + maxc * nx;
    const c2<R> *vi = a.V + (long long)i * a.ld;
    c2<R> wv[EPT];
#pragma unroll
    for (int k = 0; k < EPT; k++) wv[k] = mk<R>(0, 0);
    if (nr > 0) {
        prolong_rows<R>(T, a.s, F0, nF, sc, px, u);
        for (int e = tid; e < nF * nx; e += blockDim.x) {
            const int qy = dnx.q(e), yy = F0 + qy;
            if (yy >= 0 && yy < ny) u[e] = csub<R>(vi[T.foff + (long long)yy * nx + (e - qy * nx)], u[e]);
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < EPT; k++) {
            const int e = tid + k * LOCAL_THREADS;
            if (e < cnt) {
                const int qy = dnx.q(e), yy = r0 + qy, xx = e - qy * nx;
                wv[k] = stencil_smem<R, IMP>(a.st, u, F0, nF, nx, ny, xx, yy, T.ix0, T.iy0);
            }
        }
    }
    // task-wide sums of n values: the per-warp partials in red[warp][l] are added per CTA and
    // sent to slot gat[b][rank][l] of every CTA, then one cluster barrier, then each CTA adds
    // the C slots in rank order into out[l]
    const int lane = tid & 31, warp = tid >> 5;
    auto gather = [&](int b, int n, c2<R> *out) {
        __syncthreads();
        for (int idx = tid; idx < n * C; idx += blockDim.x) {
            const int l = idx % n, dst = idx / n;
            c2<R> sum = mk<R>(0, 0);
            for (int q = 0; q < NWARP; q++) sum = cadd<R>(sum, red[q * LDP + l]);
            *cluster_map(&gat[b][rank][l], (unsigned)dst) = sum;
        }
        cluster_barrier();
        for (int l = tid; l < n; l += blockDim.x) {
            c2<R> sum = mk<R>(0, 0);
            for (int q = 0; q < C; q++) sum = cadd<R>(sum, gat[b][q][l]);
            out[l] = sum;
        }
        __syncthreads();
    };
    auto warp_store = [&](int l, c2<R> v) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) { v.x += shfl_xor(v.x, o); v.y += shfl_xor(v.y, o); }
        if (lane == 0) red[warp * LDP + l] = v;
    };
    // h = V^H w over the task (per-warp partials, then the cluster gather)
    auto reduce_dots = [&](int b, c2<R> *out) {
        for (int l = 0; l < nv; l++) {
            c2<R> acc = mk<R>(0, 0);
            const c2<R> *vl = a.V + (long long)l * a.ld + base;
#pragma unroll
            for (int k = 0; k < EPT; k++) {
                const int e = tid + k * LOCAL_THREADS;
                if (e < cnt) cdotc_acc<R>(acc, vl[e], wv[k]);
            }
            warp_store(l, acc);
        }
        gather(b, nv, out);
    };
    // w -= V h
    auto update = [&](const c2<R> *h) {
        for (int l = 0; l < nv; l++) {
            const c2<R> hl = h[l];
            const c2<R> *vl = a.V + (long long)l * a.ld + base;
#pragma unroll
            for (int k = 0; k < EPT; k++) {
                const int e = tid + k * LOCAL_THREADS;
                if (e < cnt) caxpy_neg<R>(wv[k], hl, vl[e]);
            }
        }
    };
    reduce_dots(0, h1s);
    // ---- B: w -= V h1, partial h2 ----
    update(h1s);
    reduce_dots(1, h2s);
    // ---- C: w -= V h2, ||w||² ----
    update(h2s);
    {
        R nrm = 0;
#pragma unroll
        for (int k = 0; k < EPT; k++) nrm = fma(wv[k].x, wv[k].x, fma(wv[k].y, wv[k].y, nrm));
        warp_store(0, mk<R>(nrm, 0));
        gather(0, 1, nrm_s);
    }
    if (tid == 0) hn_s = sqrt(nrm_s[0].x);
    __syncthreads();
    const R hn = hn_s;
    // ---- D: v_{i+1} = w/||w||; Givens rotation and stop test ----
    c2<R> *vn = a.V + (long long)(i + 1) * a.ld + base;
    if (hn > (R)0) {
        const R inv = (R)1 / hn;
#pragma unroll
        for (int k = 0; k < EPT; k++) {
            const int e = tid + k * LOCAL_THREADS;
            if (e < cnt) vn[e] = mk<R>(wv[k].x * inv, wv[k].y * inv);
        }
    }
    if (tid == 0) {
        c2<R> hc[MAX_RESTART + 1];
        for (int l = 0; l <= i; l++) hc[l] = cadd<R>(h1s[l], h2s[l]);
        for (int l = 0; l < i; l++) {
            const c2<R> x = hc[l], yv = hc[l + 1], sx = sn_s[l];
            hc[l] = cadd<R>(cscale<R>(cs_s[l], x), cmul<R>(sx, yv));
            hc[l + 1] = csub<R>(cscale<R>(cs_s[l], yv), cmul<R>(mk<R>(sx.x, -sx.y), x));
        }
        R c; c2<R> sv, rr;
        givens<R>(hc[i], mk<R>(hn, 0), c, sv, rr);
        hc[i] = rr;
        hc[i + 1] = mk<R>(0, 0);
        const c2<R> gi = g_s;
        const c2<R> gn = mk<R>(-(sv.x * gi.x + sv.y * gi.y), -(sv.x * gi.y - sv.y * gi.x));   // -conj(s) g_i
        const int its = its_s + 1;
        const R res = hypot(gn.x, gn.y);
        const bool conv = res <= a.tol * ref_s || !(hn > (R)0);
        const bool stop = conv || its >= a.maxit || i + 1 >= a.restart;
        stop_s = stop ? 1 : 0;
        if (rank == 0) {
            c2<R> *Hc = a.S.H + (long long)t * (a.restart + 1) * a.restart + (long long)i * (a.restart + 1);
            for (int l = 0; l <= i + 1; l++) Hc[l] = hc[l];
            a.S.cs[(long long)t * a.restart + i] = c;
            a.S.sn[(long long)t * a.restart + i] = sv;
            c2<R> *g = a.S.g + (long long)t * (a.restart + 1);
            g[i] = cscale<R>(c, gi);
            g[i + 1] = gn;
            a.S.its[t] = its;
            a.S.kcols[t] = i + 1;
            if (conv || its >= a.maxit) a.S.conv[t] = 1;
            a.act_out[t] = stop ? 0 : 1;
            if (!stop) atomicAdd(a.counter, 1);
        }
    }
    __syncthreads();
    if (stop_s) return;                           // the same decision in every CTA
    // ---- E: y = Zᵀ A v_{i+1} on coarse rows [c0, c1) ----
    cluster_barrier();                            // v_{i+1} of every CTA written and visible
    const int c0 = (int)(rank * my) / C, c1 = (int)((rank + 1) * my) / C;
    if (c1 <= c0) return;
    const int G0 = 2 * c0 - 1, G1 = 2 * (c1 - 1) + 3, nG = G1 - G0 + 1;
    const int W0 = G0 - 1, nW = nG + 2;
    c2<R> *vin = reinterpret_cast<c2<R> *>(smem_raw);
    c2<R> *tt = vin + nW * nx;
    c2<R> *sx = tt + nG * nx;
    const c2<R> *vnf = a.V + (long long)(i + 1) * a.ld + T.foff;
    for (int e = tid; e < nW * nx; e += blockDim.x) {
        const int qy = dnx.q(e), yy = W0 + qy;
        vin[e] = (yy >= 0 && yy < ny) ? vnf[(long long)yy * nx + (e - qy * nx)] : mk<R>(0, 0);
    }
    __syncthreads();
    for (int e = tid; e < nG * nx; e += blockDim.x) {
        const int qy = dnx.q(e), yy = G0 + qy, xx = e - qy * nx;
        tt[e] = (yy >= 0 && yy < ny) ? stencil_smem<R, IMP>(a.st, vin, W0, nW, nx, ny, xx, yy, T.ix0, T.iy0)
                                     : mk<R>(0, 0);
    }
    __syncthreads();
    for (int e = tid; e < nG * mx; e += blockDim.x) {
        const int fr = dmx.q(e), cx = e - fr * mx;
        c2<R> acc = mk<R>(0, 0);
#pragma unroll
        for (int qq = 0; qq < 5; qq++) {
            const int fx = 2 * cx - 1 + qq;
            if (fx >= 0 && fx < nx) {
                const c2<R> v = tt[fr * nx + fx];
                acc.x = fma(zw<R>(qq), v.x, acc.x);
                acc.y = fma(zw<R>(qq), v.y, acc.y);
            }
        }
        sx[e] = acc;
    }
    __syncthreads();
    for (int e = tid; e < (c1 - c0) * mx; e += blockDim.x) {
        const int qc = dmx.q(e), cy = c0 + qc, cx = e - qc * mx;
        c2<R> acc = mk<R>(0, 0);
#pragma unroll
        for (int qq = 0; qq < 5; qq++) {
            const int fy = 2 * cy - 1 + qq;
            if (fy >= 0 && fy < ny) {
                const c2<R> v = sx[(fy - G0) * mx + cx];
                acc.x = fma(zw<R>(qq), v.x, acc.x);
                acc.y = fma(zw<R>(qq), v.y, acc.y);
            }
        }
        a.y[T.coff + (long long)cy * mx + cx] = make_double2((double)acc.x, (double)acc.y);
    }
}

// ------------------------------------------------------------------------------------------
// launchers
// ------------------------------------------------------------------------------------------
template <typename R> static size_t csz() { return sizeof(c2<R>); }

template <typename R>
void launch_restrict(const LocalArgs<R> &a, const double2 *glob, long long nglob, c2<R> *out,
                     const int *flag, cudaStream_t s) {
    k_restrict<R><<<a.nftiles, LOCAL_THREADS, 0, s>>>(a, a.gw, nglob, glob, out, flag);
}
template <typename R>
void launch_scatter(const LocalArgs<R> &a, const c2<R> *x, double2 *glob, long long nglob,
                    const int *flag, cudaStream_t s) {
    k_scatter<R><<<a.nftiles, LOCAL_THREADS, 0, s>>>(a, a.gw, nglob, x, glob, flag);
}
template <typename R>
void launch_local_A(const LocalArgs<R> &a, const c2<R> *in, c2<R> *out, const c2<R> *f,
                    const int *flag, cudaStream_t s) {
    size_t sm = (size_t)(a.frows + 2) * a.max_nx * csz<R>();
    if (a.st.bc) k_local_A<R, true><<<a.nftiles, LOCAL_THREADS, sm, s>>>(a, in, out, f, flag);
    else k_local_A<R, false><<<a.nftiles, LOCAL_THREADS, sm, s>>>(a, in, out, f, flag);
}
template <typename R>
size_t zt_smem(const LocalArgs<R> &a, int apply_A) {
    int nF = 2 * a.crows + 3, nV = nF + 2;
    return ((size_t)(apply_A ? nV : 0) * a.max_nx + (size_t)nF * a.max_nx + (size_t)nF * (a.max_nx / 2 + 1)) * csz<R>();
}
template <typename R>
void launch_zt(const LocalArgs<R> &a, const c2<R> *in, double2 *y, int apply_A, const int *flag,
               cudaStream_t s) {
    if (a.st.bc) k_zt<R, true><<<a.nctiles, LOCAL_THREADS, zt_smem(a, apply_A), s>>>(a, in, y, apply_A, flag);
    else k_zt<R, false><<<a.nctiles, LOCAL_THREADS, zt_smem(a, apply_A), s>>>(a, in, y, apply_A, flag);
}
template <typename R>
void launch_z(const LocalArgs<R> &a, const double2 *sc, const c2<R> *add, c2<R> *out,
              const int *flag, cudaStream_t s, R sign) {
    int maxc = prolong_max_cy(a.frows);
    size_t sm = ((size_t)maxc * (a.max_nx / 2 + 1) + (size_t)maxc * a.max_nx + (size_t)a.frows * a.max_nx) * csz<R>();
    k_z<R><<<a.nftiles, LOCAL_THREADS, sm, s>>>(a, sc, add, out, flag, sign);
}
template <typename R>
size_t ps_smem(const LocalArgs<R> &a) {
    int nF = a.frows + 2, maxc = prolong_max_cy(nF);
    return ((size_t)maxc * (a.max_nx / 2 + 1) + (size_t)maxc * a.max_nx + (size_t)nF * a.max_nx +
            (size_t)NWARP * LDP) * csz<R>();
}
template <typename R>
void launch_prolong_stencil(const LocalArgs<R> &a, int mode, const c2<R> *in, const double2 *sc,
                            c2<R> *out, const c2<R> *V, int nv, c2<R> *part, const int *flag,
                            cudaStream_t s) {
    if (a.st.bc)
        k_prolong_stencil<R, true><<<a.nftiles, LOCAL_THREADS, ps_smem(a), s>>>(a, mode, in, sc, out, V, nv,
                                                                                part, flag);
    else
        k_prolong_stencil<R, false><<<a.nftiles, LOCAL_THREADS, ps_smem(a), s>>>(a, mode, in, sc, out, V, nv,
                                                                                 part, flag);
}
template <typename R>
void launch_cgs_update(const LocalArgs<R> &a, int pass, c2<R> *w, const c2<R> *V, int nv,
                       const c2<R> *part_in, c2<R> *part_out, const int *flag, cudaStream_t s) {
    k_cgs_update<R><<<a.nftiles, LOCAL_THREADS, 0, s>>>(a, pass, w, V, nv, part_in, part_out, flag);
}
template <typename R>
void launch_givens_normalize(const LocalArgs<R> &a, const InnerState<R> &S, int restart, int i,
                             c2<R> *w, const c2<R> *p1, const c2<R> *p2, const c2<R> *p3,
                             const int *act_in, int *act_out, int *counter, R tol, int maxit,
                             cudaStream_t s) {
    k_givens_normalize<R><<<a.nftiles, LOCAL_THREADS, 0, s>>>(a, S, restart, i, w, p1, p2, p3, act_in,
                                                               act_out, counter, tol, maxit);
}
template <typename R>
void launch_init_cycle(const LocalArgs<R> &a, const InnerState<R> &S, int restart, c2<R> *v0,
                       const c2<R> *p3, const int *flag, int *act_out, int *counter, R tol,
                       int maxit, int set_ref, cudaStream_t s) {
    k_init_cycle<R><<<a.nftiles, LOCAL_THREADS, 0, s>>>(a, S, restart, v0, p3, flag, act_out, counter,
                                                         tol, maxit, set_ref);
}
template <typename R>
void launch_update_u(const LocalArgs<R> &a, const InnerState<R> &S, int restart, c2<R> *u,
                     const c2<R> *V, const int *flag, int *rs_out, int *counter, int maxit,
                     cudaStream_t s) {
    k_update_u<R><<<a.nftiles, LOCAL_THREADS, 0, s>>>(a, S, restart, u, V, flag, rs_out, counter, maxit);
}
template <typename R>
void launch_set_ref(const LocalArgs<R> &a, const InnerState<R> &S, const c2<R> *p3, const int *flag,
                    cudaStream_t s) {
    k_set_ref<R><<<(a.ntasks + 127) / 128, 128, 0, s>>>(a, S, p3, flag);
}
template <typename R>
void launch_coarse_combine(const LocalArgs<R> &a, const InnerState<R> &S, int restart,
                           const double2 *sbuf, double2 *sc, const int *flag, cudaStream_t s) {
    k_coarse_combine<R><<<a.nctiles, LOCAL_THREADS, 0, s>>>(a, S, restart, sbuf, sc, flag);
}
template <typename R>
cudaError_t launch_arnoldi_step(const LocalArgs<R> &la, int C, int i, int restart, c2<R> *V, const double2 *sc,
                                double2 *y, const InnerState<R> &S, const int *act_in, int *act_out,
                                int *counter, R tol, int maxit, size_t smem, cudaStream_t s) {
    StepArgs<R> a;
    a.tasks = la.tasks; a.st = la.st; a.ld = la.ld; a.C = C; a.i = i; a.restart = restart;
    a.V = V; a.s = sc; a.y = y; a.S = S; a.act_in = act_in; a.act_out = act_out; a.counter = counter;
    a.tol = tol; a.maxit = maxit;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(la.ntasks * C));
    cfg.blockDim = dim3(LOCAL_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (la.st.bc) return cudaLaunchKernelEx(&cfg, k_arnoldi_step<R, true>, a);
    return cudaLaunchKernelEx(&cfg, k_arnoldi_step<R, false>, a);
}

// Largest cluster of CTAs holding `smem` bytes of dynamic shared memory each that the device can
// co-schedule (0 on error); sets the kernels' dynamic shared-memory limit to `smem` first.
template <typename R> int arnoldi_step_max_cluster(size_t smem, int C) {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_arnoldi_step<R, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
        return 0;
    if ((e = cudaFuncSetAttribute(k_arnoldi_step<R, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
        return 0;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)C);
    cfg.blockDim = dim3(LOCAL_THREADS);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_arnoldi_step<R, false>, &cfg) != cudaSuccess) return 0;
    return n;
}

void launch_cast(long long n, const void *in, int in_double, void *out, int out_double,
                 cudaStream_t s) {
    int grid = (int)((n + 255) / 256);
    if (grid > 4096) grid = 4096;
    if (grid < 1) grid = 1;
    if (in_double && out_double)
        k_cast<double, double><<<grid, 256, 0, s>>>(n, (const double2 *)in, (double2 *)out);
    else if (in_double)
        k_cast<double, float><<<grid, 256, 0, s>>>(n, (const double2 *)in, (float2 *)out);
    else if (out_double)
        k_cast<float, double><<<grid, 256, 0, s>>>(n, (const float2 *)in, (double2 *)out);
    else
        k_cast<float, float><<<grid, 256, 0, s>>>(n, (const float2 *)in, (float2 *)out);
}

size_t local_max_dynamic_smem(int max_nx, int bytes_per_c, int frows, int crows) {
    int nF = frows + 2, maxc = prolong_max_cy(nF);
    size_t ps = ((size_t)maxc * (max_nx / 2 + 1) + (size_t)maxc * max_nx + (size_t)nF * max_nx +
                 (size_t)NWARP * LDP) * bytes_per_c;
    int cF = 2 * crows + 3;
    size_t zt = ((size_t)(cF + 2) * max_nx + (size_t)cF * max_nx + (size_t)cF * (max_nx / 2 + 1)) * bytes_per_c;
    return ps > zt ? ps : zt;
}

template <typename R> cudaError_t set_local_smem_limits(size_t bytes) {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_prolong_stencil<R, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_prolong_stencil<R, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_zt<R, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_zt<R, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_z<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_local_A<R, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_local_A<R, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes)) != cudaSuccess) return e;
    return cudaSuccess;
}

#define INST(R)                                                                                         \
    template void launch_restrict<R>(const LocalArgs<R> &, const double2 *, long long, c2<R> *, const int *, cudaStream_t); \
    template void launch_scatter<R>(const LocalArgs<R> &, const c2<R> *, double2 *, long long, const int *, cudaStream_t); \
    template void launch_local_A<R>(const LocalArgs<R> &, const c2<R> *, c2<R> *, const c2<R> *, const int *, cudaStream_t); \
    template void launch_zt<R>(const LocalArgs<R> &, const c2<R> *, double2 *, int, const int *, cudaStream_t); \
    template void launch_z<R>(const LocalArgs<R> &, const double2 *, const c2<R> *, c2<R> *, const int *, cudaStream_t, R); \
    template void launch_prolong_stencil<R>(const LocalArgs<R> &, int, const c2<R> *, const double2 *, c2<R> *, const c2<R> *, int, c2<R> *, const int *, cudaStream_t); \
    template void launch_cgs_update<R>(const LocalArgs<R> &, int, c2<R> *, const c2<R> *, int, const c2<R> *, c2<R> *, const int *, cudaStream_t); \
    template void launch_givens_normalize<R>(const LocalArgs<R> &, const InnerState<R> &, int, int, c2<R> *, const c2<R> *, const c2<R> *, const c2<R> *, const int *, int *, int *, R, int, cudaStream_t); \
    template void launch_init_cycle<R>(const LocalArgs<R> &, const InnerState<R> &, int, c2<R> *, const c2<R> *, const int *, int *, int *, R, int, int, cudaStream_t); \
    template void launch_update_u<R>(const LocalArgs<R> &, const InnerState<R> &, int, c2<R> *, const c2<R> *, const int *, int *, int *, int, cudaStream_t); \
    template cudaError_t set_local_smem_limits<R>(size_t); \
    template void launch_coarse_combine<R>(const LocalArgs<R> &, const InnerState<R> &, int, const double2 *, double2 *, const int *, cudaStream_t); \
    template void launch_set_ref<R>(const LocalArgs<R> &, const InnerState<R> &, const c2<R> *, const int *, cudaStream_t); \
    template cudaError_t launch_arnoldi_step<R>(const LocalArgs<R> &, int, int, int, c2<R> *, const double2 *, double2 *, const InnerState<R> &, const int *, int *, int *, R, int, size_t, cudaStream_t); \
    template int arnoldi_step_max_cluster<R>(size_t, int);

INST(float)
INST(double)

}  // namespace hdd
