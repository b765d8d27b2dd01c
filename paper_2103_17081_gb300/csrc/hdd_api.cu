// hdd_api.cu — context, set-up and solve driver behind the C ABI declared in include/hdd.h.
//
// Host code only orchestrates: every arithmetic step of assembly, deflation set-up, inner and
// outer solves runs in the kernels of kernels_local.cu, kernels_coarse.cu and kernels_outer.cu.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "hdd.h"
#include "hdd_common.cuh"

using namespace hdd;

namespace {

struct DevMem {
    void *p = nullptr;
    size_t bytes = 0;
    ~DevMem() { if (p) cudaFree(p); }
    cudaError_t ensure(size_t b) {
        if (b <= bytes && p) return cudaSuccess;
        if (p) { cudaFree(p); p = nullptr; bytes = 0; }
        cudaError_t e = cudaMalloc(&p, b > 0 ? b : 16);
        if (e == cudaSuccess) bytes = b;
        return e;
    }
    void release() { if (p) cudaFree(p); p = nullptr; bytes = 0; }
    template <typename T> T *as() const { return reinterpret_cast<T *>(p); }
};

struct SubBox {
    int ix0, ix1, iy0, iy1, ox0, ox1, oy0, oy1, nx, ny, mx, my;
};

struct FactorSet {            // banded FP64 factors of one matrix per shape, blocked solve form
    DevMem M, Mdf, P, Meta, table;  // Mdf: the operators M as (hi, lo) FP32 pairs (double-FP32 solve)
    DevMem G, spk;                  // SPIKE plans: spike matrices (pairs), SpikeInfo level-major
    int spike_level[SPIKE_LEVELS] = {0, 0};   // level L (P = 2, 4) available for every shape
    int spike_levels_built = 0;
    std::vector<BlockFactor> h;
    std::vector<double> fma_col;    // FP64 FMAs of one real column by banded substitution, per shape
    BlockSolveCfg cfg;              // shared-memory plan of the blocked solve
    bool re2 = false;               // factors of real-equivalent systems (complex matrices)
    bool ready = false;
    void clear() { G.release(); spk.release(); spike_level[0] = spike_level[1] = 0; spike_levels_built = 0;
                   M.release(); Mdf.release(); P.release(); Meta.release(); table.release(); h.clear(); fma_col.clear(); cfg = BlockSolveCfg{}; re2 = false; ready = false; }
};

template <typename R> struct InnerWork {   // inner GMRES buffers for one precision
    int restart = 0;
    DevMem f, u, x, t, V, y, s, p1, p2, p3;
    DevMem y2, s2;                              // two coarse vectors per task (warm start)
    DevMem H, cs, sn, g, ref, its, kcols, conv, rsf;
    DevMem act0, act1, flagA, flagB;
};

// Kernel families timed by the profiler (CUDA events around every launch on the launching
// stream).  bound: 0 = memory (HBM bytes), 1 = FP64 arithmetic.
enum Fam { F_ZT, F_COARSE, F_PS, F_CGS, F_GIVENS, F_LMISC, F_OCGS, F_OMISC, F_CNN, F_OREORTH, F_STEP, F_ODF,
           F_CGRID, F_OUDF, F_CDF, F_CSPK, NFAM };
const char *kFamName[NFAM] = {"local_stencil_zt", "coarse_solve_fp64", "local_prolong_stencil_dots",
                              "local_cgs2_update", "local_givens_normalize", "local_misc",
                              "outer_cgs2_fp64", "outer_misc_fp64", "warm_start_cnn",
                              "outer_reorth_fp32", "local_arnoldi_step", "outer_dots_df32",
                              "two_level_grid_coarse", "outer_update_df32", "coarse_solve_df32",
                              "coarse_solve_df32_spike"};
// (2: FP32 pipe; for the double-FP32 families the flop counts are FP32 instructions)
const int kFamBound[NFAM] = {0, 1, 0, 0, 0, 0, 1, 0, 2, 0, 0, 2, 0, 2, 2, 2};

struct Prof {
    bool on = false;
    long long launches = 0;
    long long cnt[NFAM] = {};
    double ms[NFAM] = {}, bytes[NFAM] = {}, flops[NFAM] = {};
    struct P { int f; cudaEvent_t a, b; double by, fl; };
    std::vector<P> pend;
    std::vector<cudaEvent_t> pool;
    ~Prof() {
        for (auto &p : pend) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
        for (auto e : pool) cudaEventDestroy(e);
    }
    void reset() {
        launches = 0;
        for (int f = 0; f < NFAM; f++) { cnt[f] = 0; ms[f] = bytes[f] = flops[f] = 0; }
    }
    cudaEvent_t get() {
        if (pool.empty()) { cudaEvent_t e; cudaEventCreate(&e); return e; }
        cudaEvent_t e = pool.back(); pool.pop_back(); return e;
    }
    // after a stream synchronisation every pending event pair is complete
    void harvest() {
        for (auto &p : pend) {
            float t = 0.f;
            if (cudaEventElapsedTime(&t, p.a, p.b) == cudaSuccess) ms[p.f] += t;
            cnt[p.f]++; bytes[p.f] += p.by; flops[p.f] += p.fl;
            pool.push_back(p.a); pool.push_back(p.b);
        }
        pend.clear();
    }
};

struct CnnState {            // learned warm start: parameters, Adam moments, activations
    bool ready = false;
    int step = 0;
    DevMem P, Pb, M, Vm, G, sigma, X0, A1, A2, A3, A4, dA4, Rr, dB1, dB2, part, lpart;
    DevMem Fh, Q, T2, Yc, Sc, Pf, Pr, scale, tloss;   // deflated loss: f̂, P r, Pᵀ P r, coarse, partials
    // tensor-core inference: BF16 padded planar activations (ping-pong), weight images, error flag
    DevMem Ba, Bb, Wimg, err;
    bool tc_dirty = true;      // weight images out of date (parameters changed)
    bool pad_ready = false;    // frame borders of Ba, Bb zeroed for the current task layout
};

struct OuterWork {
    DevMem V, V32, V32L, D, Z, w, r, H, cs, sn, g, Wq, h1, h2, part, npart, npart1, hn, flag, hist, beta, y, fnorm, act, kcols;
    DevMem fallbacks;
    DevMem part2, invs, err, close;             // delayed CGS2: second dot partials, 1/σ, breakdown, end-of-cycle mask
    DevMem vmax;                                // delayed CGS2: max |hi part| per basis slot (bias of the dots)
};

}  // namespace

struct hdd_ctx {
    int device = 0;
    std::string err;
    bool assembled = false, dd = false;
    // problem
    int N = 0, diag = 0;
    int bc = 0;                                 // 0: Dirichlet, 1: impedance on all four sides
    double k = 0, h = 0;
    Stencil st{};
    DevMem d_bcoef, d_bmass;                    // boundary-class rows of A and M (bc = 1)
    long long nglob = 0;
    // decomposition
    int Sx = 0, Sy = 0, overlap = 0;
    std::vector<SubBox> subs;
    std::vector<int> sub_shape;
    std::vector<std::pair<int, int>> shapes;   // (nx, ny)
    std::vector<std::pair<int, int>> shape_org; // box origin (ix0, iy0) of one subdomain of each shape
    int nrhs = 1;                               // right-hand sides batched per solve
    std::vector<Task> h_tasks;                  // task t = r·nsub + s
    std::vector<Tile> h_ftiles, h_ctiles;
    DevMem d_tasks, d_ftiles, d_ctiles, d_ones, d_mask;
    DevMem d_tasks2, d_mask2;                   // every task twice, the copy's coarse offsets + ldc (two
                                                // coarse solves per task in one launch)
    long long ld = 0, ldc = 0;
    int max_nx = 0, max_n = 0;
    int frows = FINE_ROWS, crows = COARSE_ROWS;  // tile heights (hdd_autotune)
    std::vector<long long> foffs, coffs;
    std::vector<int2> h_tct;                    // tensor-core conv tiles (task, first frame position)
    DevMem d_tct;
    long long ptot = 0;                         // frame positions over all tasks
    int tc_wmax = 0;                            // staged window positions per plane
    // factors
    FactorSet E, Aex;
    // work
    InnerWork<float> w32;
    InnerWork<double> w64;
    OuterWork ow;
    CnnState cnn;
    DevMem tmp_a, tmp_b, tmp_c;                // staging for test hooks
    DevMem d_alist;                            // active tasks of a SPIKE coarse solve, compacted
    int *h_counter = nullptr;                  // pinned
    DevMem d_counter;
    std::vector<double> hist;
    std::vector<int> h_its;
    Prof prof;
    int nsm = 152;                             // SMs of the device
    int coarse_la = 1;                         // HDD_OPT_COARSE_LOOKAHEAD
    int fused_inner = 1;                       // HDD_OPT_FUSED_INNER
    int outer_df = 1;                          // HDD_OPT_OUTER_DOTS_DF
    int outer_udf = 1;                         // HDD_OPT_OUTER_UPDATE_DF
    int outer_dcgs = 1;                        // HDD_OPT_OUTER_DCGS2
    int coarse_df = 1;                         // HDD_OPT_COARSE_DF
    int coarse_spike = 1;                      // HDD_OPT_COARSE_SPIKE
    int outer_bias = 1;                        // HDD_OPT_OUTER_DOTS_BIASED
    int step_C[2] = {-1, -1};                  // fused-step cluster size per inner precision (0: off, -1: unplanned)
    size_t step_smem[2] = {0, 0};
    bool poisoned = false;                     // a device wait gave up with work in flight
    // grid coarse space of the two-level variant: sine transform S and D⁻¹ (FP64 and FP32 copies),
    // two coarse work vectors, and the fine vectors Q v and v - A Q v of the hybrid step
    struct CoarseGrid {
        bool ready = false;
        int c = 0, Nc = 0, m = 0;
        DevMem S64, S32, D64, D32, bufA, bufB, z0, t;
    } cg;
    ~hdd_ctx() { if (h_counter) cudaFreeHost(h_counter); }
};

#define FAIL(code, ...)                                                                            \
    do {                                                                                           \
        char _b[512];                                                                              \
        snprintf(_b, sizeof(_b), __VA_ARGS__);                                                     \
        ctx->err = _b;                                                                             \
        return code;                                                                               \
    } while (0)

#define CK(call)                                                                                   \
    do {                                                                                           \
        cudaError_t _e = (call);                                                                   \
        if (_e != cudaSuccess) {                                                                   \
            if (_e == cudaErrorMemoryAllocation) FAIL(HDD_ERR_OOM, "%s: %s", #call, cudaGetErrorString(_e)); \
            FAIL(HDD_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(_e));                           \
        }                                                                                          \
    } while (0)

#define CKL() CK(cudaGetLastError())

namespace {

// Counts every kernel launch; with profiling on, brackets it with a CUDA event pair on the
// launching stream.  Use: { Launch L(ctx, family, bytes, flops, stream); launch(...); }
struct Launch {
    hdd_ctx *c; int f; double by, fl; cudaStream_t s; cudaEvent_t a = nullptr;
    Launch(hdd_ctx *ctx, int fam, double bytes, double flops, cudaStream_t st)
        : c(ctx), f(fam), by(bytes), fl(flops), s(st) {
        c->prof.launches++;
        if (c->prof.on) { a = c->prof.get(); cudaEventRecord(a, s); }
    }
    ~Launch() {
        if (a) {
            cudaEvent_t b = c->prof.get();
            cudaEventRecord(b, s);
            c->prof.pend.push_back(Prof::P{f, a, b, by, fl});
        }
    }
};
#define KL(fam, by, fl, stmt) do { Launch _l(ctx, fam, (double)(by), (double)(fl), s); stmt; } while (0)

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

template <typename R> LocalArgs<R> local_args(hdd_ctx *ctx) {
    LocalArgs<R> a;
    a.tasks = ctx->d_tasks.as<Task>();
    a.ftiles = ctx->d_ftiles.as<Tile>();
    a.ctiles = ctx->d_ctiles.as<Tile>();
    a.ntasks = (int)ctx->h_tasks.size();
    a.nftiles = (int)ctx->h_ftiles.size();
    a.nctiles = (int)ctx->h_ctiles.size();
    a.st = ctx->st;
    a.ld = ctx->ld;
    a.ldc = ctx->ldc;
    a.max_nx = ctx->max_nx;
    a.gw = ctx->bc ? ctx->N + 1 : ctx->N - 1;
    a.glo = ctx->bc ? 0 : 1;
    a.frows = ctx->frows;
    a.crows = ctx->crows;
    return a;
}

hdd_status read_counter(hdd_ctx *ctx, cudaStream_t s, int *out) {
    CK(cudaMemcpyAsync(ctx->h_counter, ctx->d_counter.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    ctx->prof.harvest();
    *out = *ctx->h_counter;
    return HDD_OK;
}

// E_j (or A_j) factors for every distinct shape, FP64, on the device: banded LU with partial
// pivoting, then the blocked solve operators.
// ---- SPIKE plans of a factor set (the double-FP32 coarse solve split over P parts) ----------
// Forward / backward sweeps of blocks [J0, J1) of one shape emulated in FP64 on the host with the
// device's own block operators, for W unit window vectors at once (zero inputs): Y holds rows
// [ybase, ybase + ny) of the sweep's vector, W values per row (row-major, row = vector index).
static void emu_fwd_cols(const double *M, const int4 *meta, int J0, int J1, int W, long long ybase,
                         std::vector<double> &Y) {
    std::vector<double> acc((size_t)BNB * W);
    for (int J = J0; J < J1; J++) {
        const int4 mt = meta[J];
        const int w = mt.y, Ks = op_stride(w);
        const double *MJ = M + mt.x;
        std::fill(acc.begin(), acc.end(), 0.0);
        for (int r = 0; r < BNB; r++) {
            const double *row = MJ + (size_t)r * Ks + BNB;
            double *a = acc.data() + (size_t)r * W;
            for (int c = 0; c < w; c++) {
                const double mv = row[c];
                if (mv == 0.0) continue;
                const double *yr = Y.data() + (size_t)((long long)J * BNB - w + c - ybase) * W;
                for (int k = 0; k < W; k++) a[k] += mv * yr[k];
            }
        }
        std::copy(acc.begin(), acc.end(), Y.begin() + (size_t)((long long)J * BNB - ybase) * W);
    }
}
static void emu_bwd_cols(const double *M, const int4 *meta, int J0, int J1, int W, long long xbase,
                         std::vector<double> &X) {
    std::vector<double> acc((size_t)BNB * W);
    for (int J = J1 - 1; J >= J0; J--) {
        const int4 mt = meta[J];
        const int w = mt.w, Ks = op_stride(w);
        const double *MJ = M + mt.z;
        std::fill(acc.begin(), acc.end(), 0.0);
        for (int r = 0; r < BNB; r++) {
            const double *row = MJ + (size_t)r * Ks + BNB;
            double *a = acc.data() + (size_t)r * W;
            for (int c = 0; c < w; c++) {
                const double mv = row[c];
                if (mv == 0.0) continue;
                const double *xr = X.data() + (size_t)((long long)(J + 1) * BNB + c - xbase) * W;
                for (int k = 0; k < W; k++) a[k] += mv * xr[k];
            }
        }
        std::copy(acc.begin(), acc.end(), X.begin() + (size_t)((long long)J * BNB - xbase) * W);
    }
}

// Spike matrices for P = 2 and 4 (SpikeInfo): parts of equal block counts, available for a shape
// when every part has at least max(wf, wb) + 16 rows, the last part starts before row m - wb and
// both windows fit the kernel's staging (SPIKE_WMAX).  Gf_p[:, k] is the forward response of part
// p to the unit value at row r_p - wf + k; Gb_p[:, k] the backward response of part p to the unit
// value at row r_{p+1} + k (column-major, stored as (hi, lo) FP32 pairs).
hdd_status build_spikes(hdd_ctx *ctx, FactorSet &F, const std::vector<int4> &meta, long long mo) {
    const int ns = (int)F.h.size();
    std::vector<double> M((size_t)std::max(mo, 1LL));
    CK(cudaMemcpy(M.data(), F.M.p, (size_t)mo * sizeof(double), cudaMemcpyDeviceToHost));
    std::vector<SpikeInfo> tab((size_t)ns * SPIKE_LEVELS);
    std::vector<float2> Gall;
    auto put = [&](const std::vector<double> &Y, long long ybase, int W, long long r0, int np) {
        const long long o = (long long)Gall.size();
        Gall.resize(Gall.size() + (size_t)np * W);
        for (int k = 0; k < W; k++)
            for (int i = 0; i < np; i++) {
                const double v = Y[(size_t)(r0 + i - ybase) * W + k];
                const float hi = (float)v;
                Gall[(size_t)o + (size_t)k * np + i] = make_float2(hi, (float)(v - (double)hi));
            }
        return o;
    };
    for (int L = 0; L < SPIKE_LEVELS; L++) F.spike_level[L] = 1;
    for (int q = 0; q < ns; q++) {
        const BlockFactor &b = F.h[q];
        const int4 *mt = meta.data() + b.meta_off;
        const int nbk = b.nblk, m = b.m, wf = b.wl, wb = b.wu;
        for (int L = 0; L < SPIKE_LEVELS; L++) {
            SpikeInfo &S = tab[(size_t)q * SPIKE_LEVELS + L];
            std::memset(&S, 0, sizeof(S));
            const int P = L == 0 ? 2 : 4;
            bool ok = wf >= 1 && wb >= 1 && wf <= SPIKE_WMAX && wb <= SPIKE_WMAX;
            for (int p = 0; p <= P; p++) S.B[p] = (int)(((long long)p * nbk) / P);
            for (int p = 0; p < P && ok; p++)
                if ((S.B[p + 1] - S.B[p]) * BNB < std::max(wf, wb) + BNB) ok = false;
            if (ok && (long long)S.B[P - 1] * BNB + wb > m) ok = false;
            if (!ok) { F.spike_level[L] = 0; continue; }
            S.P = P; S.wf = wf; S.wb = wb;
            for (int p = 1; p < P; p++) {             // forward spikes
                const long long r0 = (long long)S.B[p] * BNB, r1 = (long long)S.B[p + 1] * BNB;
                const long long ybase = r0 - wf;
                std::vector<double> Y((size_t)(r1 - ybase) * wf, 0.0);
                for (int k = 0; k < wf; k++) Y[(size_t)k * wf + k] = 1.0;
                emu_fwd_cols(M.data(), mt, S.B[p], S.B[p + 1], wf, ybase, Y);
                S.gf[p] = put(Y, ybase, wf, r0, (int)(r1 - r0));
            }
            for (int p = 0; p + 1 < P; p++) {         // backward spikes
                const long long r0 = (long long)S.B[p] * BNB, r1 = (long long)S.B[p + 1] * BNB;
                std::vector<double> X((size_t)(r1 + wb + BNB - r0) * wb, 0.0);
                for (int k = 0; k < wb; k++)
                    if (r1 + k < (long long)nbk * BNB) X[(size_t)(r1 + k - r0) * wb + k] = 1.0;
                emu_bwd_cols(M.data(), mt, S.B[p], S.B[p + 1], wb, r0, X);
                S.gb[p] = put(X, r0, wb, r0, (int)(r1 - r0));
            }
        }
    }
    F.spike_levels_built = 0;
    for (int L = 0; L < SPIKE_LEVELS; L++) F.spike_levels_built += F.spike_level[L];
    if (F.spike_levels_built == 0) return HDD_OK;
    CK(F.G.ensure(std::max<size_t>(Gall.size(), 1) * sizeof(float2)));
    CK(cudaMemcpy(F.G.p, Gall.data(), Gall.size() * sizeof(float2), cudaMemcpyHostToDevice));
    CK(F.spk.ensure(tab.size() * sizeof(SpikeInfo)));
    // level-major on the device: the table of level L is ns consecutive entries
    std::vector<SpikeInfo> dev(tab.size());
    for (int L = 0; L < SPIKE_LEVELS; L++)
        for (int q = 0; q < ns; q++) dev[(size_t)L * ns + q] = tab[(size_t)q * SPIKE_LEVELS + L];
    CK(cudaMemcpy(F.spk.p, dev.data(), dev.size() * sizeof(SpikeInfo), cudaMemcpyHostToDevice));
    (void)ctx;
    return HDD_OK;
}

hdd_status build_factors(hdd_ctx *ctx, FactorSet &F, bool coarse, cudaStream_t s) {
    F.clear();
    const int ns = (int)ctx->shapes.size();
    // under the impedance condition the matrices are complex: each is factored as its real
    // equivalent (order 2m, half-bandwidth 2·kl+1), which the same kernels handle
    const bool re2 = ctx->bc != 0;
    std::vector<int> m(ns), kl(ns), ku(ns);
    for (int q = 0; q < ns; q++) {
        int nx = ctx->shapes[q].first, ny = ctx->shapes[q].second;
        if (coarse) { m[q] = (nx / 2) * (ny / 2); kl[q] = ku[q] = 2 * (nx / 2) + 2; }
        else { m[q] = nx * ny; kl[q] = ku[q] = nx + 1; }
        if (re2) { m[q] *= 2; kl[q] = ku[q] = 2 * kl[q] + 1; }
    }
    std::vector<DevMem> ab(ns), piv(ns);
    std::vector<double *> abp(ns);
    std::vector<int *> pivp(ns);
    for (int q = 0; q < ns; q++) {
        size_t W = 2 * kl[q] + ku[q] + 1;
        CK(ab[q].ensure((size_t)m[q] * W * sizeof(double)));
        CK(cudaMemsetAsync(ab[q].p, 0, (size_t)m[q] * W * sizeof(double), s));
        CK(piv[q].ensure((size_t)m[q] * sizeof(int)));
        abp[q] = ab[q].as<double>();
        pivp[q] = piv[q].as<int>();
        int nx = ctx->shapes[q].first, ny = ctx->shapes[q].second;
        const int gx0 = ctx->shape_org[q].first, gy0 = ctx->shape_org[q].second;
        if (re2 && coarse) launch_assemble_E_re2(ctx->st, nx, ny, gx0, gy0, kl[q], ku[q], abp[q], s);
        else if (re2) launch_assemble_Aloc_re2(ctx->st, nx, ny, gx0, gy0, kl[q], ku[q], abp[q], s);
        else if (coarse) launch_assemble_E(ctx->st, nx, ny, kl[q], ku[q], abp[q], s);
        else launch_assemble_Aloc(ctx->st, nx, ny, kl[q], ku[q], abp[q], s);
        CKL();
    }
    DevMem dm, dkl, dku, dab, dpiv, dinfo;
    CK(dm.ensure(ns * sizeof(int))); CK(dkl.ensure(ns * sizeof(int))); CK(dku.ensure(ns * sizeof(int)));
    CK(dab.ensure(ns * sizeof(double *))); CK(dpiv.ensure(ns * sizeof(int *))); CK(dinfo.ensure(ns * sizeof(int)));
    CK(cudaMemcpyAsync(dm.p, m.data(), ns * sizeof(int), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(dkl.p, kl.data(), ns * sizeof(int), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(dku.p, ku.data(), ns * sizeof(int), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(dab.p, abp.data(), ns * sizeof(double *), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(dpiv.p, pivp.data(), ns * sizeof(int *), cudaMemcpyHostToDevice, s));
    launch_band_lu(ns, dm.as<int>(), dkl.as<int>(), dku.as<int>(), dab.as<double *>(), dpiv.as<int *>(),
                   dinfo.as<int>(), s);
    CKL();
    std::vector<int> info(ns);
    CK(cudaMemcpyAsync(info.data(), dinfo.p, ns * sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (int q = 0; q < ns; q++)
        if (info[q] != 0)
            FAIL(coarse ? HDD_ERR_SINGULAR_COARSE : HDD_ERR_SINGULAR_LOCAL,
                 "zero pivot in column %d of the %s factor of box %dx%d", info[q] - 1,
                 coarse ? "E" : "A_j", ctx->shapes[q].first, ctx->shapes[q].second);
    // permuted L, extents, permutation; then the panel widths (index bookkeeping on the host)
    F.h.resize(ns);
    F.fma_col.assign(ns, 0.0);
    long long totP = 0;
    std::vector<DevMem> Lp(ns), lext(ns), uext(ns);
    std::vector<int> KLW(ns);
    DevMem perm_all, derr;
    for (int q = 0; q < ns; q++) totP += m[q];
    CK(F.P.ensure((size_t)std::max(totP, 1LL) * sizeof(int)));
    CK(derr.ensure(sizeof(int)));
    CK(cudaMemsetAsync(derr.p, 0, sizeof(int), s));
    long long po = 0;
    for (int q = 0; q < ns; q++) {
        KLW[q] = 3 * kl[q];
        CK(Lp[q].ensure((size_t)m[q] * KLW[q] * sizeof(double)));
        CK(lext[q].ensure(m[q] * sizeof(int)));
        CK(uext[q].ensure(m[q] * sizeof(int)));
        launch_factor_prepare(m[q], kl[q], ku[q], abp[q], pivp[q], KLW[q], Lp[q].as<double>(),
                              lext[q].as<int>(), uext[q].as<int>(), F.P.as<int>() + po, derr.as<int>(), s);
        CKL();
        F.h[q].m = m[q];
        F.h[q].perm_off = po;
        po += m[q];
    }
    int herr = 0;
    CK(cudaMemcpyAsync(&herr, derr.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (herr) FAIL(HDD_ERR_INVALID_ARG, "row interchanges carried a multiplier beyond 3·kl rows");
    long long mo = 0;
    std::vector<int4> meta;
    for (int q = 0; q < ns; q++) {
        std::vector<int> le(m[q]), ue(m[q]);
        CK(cudaMemcpy(le.data(), lext[q].p, m[q] * sizeof(int), cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(ue.data(), uext[q].p, m[q] * sizeof(int), cudaMemcpyDeviceToHost));
        const int nbk = (m[q] + BNB - 1) / BNB;
        BlockFactor &b = F.h[q];
        b.nblk = nbk; b.wl = 0; b.wu = 0;
        b.meta_off = (long long)meta.size();
        long long so = 0;                      // operator offset relative to this shape
        const long long base = mo;
        for (int J = 0; J < nbk; J++) {
            const int r0 = J * BNB, r1 = std::min(m[q], r0 + BNB) - 1;
            int wl = 0, wu = 0;
            for (int c = std::max(0, r0 - KLW[q]); c < r0; c++)             // left panel
                if (c + le[c] >= r0) { wl = r0 - c; break; }
            for (int c = std::min(m[q] - 1, r1 + kl[q] + ku[q]); c > r1; c--)  // right panel
                if (c - ue[c] <= r1) { wu = c - r1; break; }
            wl += wl & 1; wu += wu & 1;
            int4 e;
            e.x = (int)(base + so); e.y = wl; so += (long long)BNB * op_stride(wl);
            e.z = (int)(base + so); e.w = wu; so += (long long)BNB * op_stride(wu);
            meta.push_back(e);
            b.wl = std::max(b.wl, wl); b.wu = std::max(b.wu, wu);
        }
        mo += so;
        double fm = 0;
        for (int j = 0; j < m[q]; j++) fm += std::min(kl[q], m[q] - 1 - j) + ue[j];
        F.fma_col[q] = fm;
        F.cfg.maxK = std::max(F.cfg.maxK, std::max(op_stride(b.wl), op_stride(b.wu)));
        while (F.cfg.cwy < BNB + b.wl) F.cfg.cwy = F.cfg.cwy ? 2 * F.cfg.cwy : BNB;
        while (F.cfg.cwx < BNB + b.wu) F.cfg.cwx = F.cfg.cwx ? 2 * F.cfg.cwx : BNB;
    }
    if (mo >= (1LL << 31)) FAIL(HDD_ERR_INVALID_ARG, "blocked factors exceed 2^31 doubles");
    CK(F.M.ensure((size_t)std::max(mo, 1LL) * sizeof(double)));
    CK(F.Meta.ensure(meta.size() * sizeof(int4)));
    CK(cudaMemcpy(F.Meta.p, meta.data(), meta.size() * sizeof(int4), cudaMemcpyHostToDevice));
    for (int q = 0; q < ns; q++) {
        launch_block_operators(m[q], kl[q], ku[q], abp[q], KLW[q], Lp[q].as<double>(),
                               F.Meta.as<int4>() + F.h[q].meta_off, F.M.as<double>(), s);
        CKL();
    }
    CK(F.Mdf.ensure((size_t)std::max(mo, 1LL) * sizeof(float2)));
    launch_ops_to_df(mo, F.M.as<double>(), F.Mdf.as<float2>(), s);
    CKL();
    // SPIKE plans of the coarse factors (their double-FP32 solves), where the host emulation that
    // forms the spike matrices stays cheap (about m·(wf² + wb²) multiply-adds per shape)
    if (coarse && ctx->coarse_spike) {
        CK(cudaStreamSynchronize(s));
        double cost = 0.0;
        for (int q = 0; q < ns; q++)
            cost += (double)F.h[q].m * ((double)F.h[q].wl * F.h[q].wl + (double)F.h[q].wu * F.h[q].wu);
        if (cost <= 1.5e9) {
            hdd_status sst = build_spikes(ctx, F, meta, mo);
            if (sst != HDD_OK) return sst;
        }
    }
    CK(F.table.ensure(ns * sizeof(BlockFactor)));
    CK(cudaMemcpyAsync(F.table.p, F.h.data(), ns * sizeof(BlockFactor), cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
    if (F.cfg.cwy == 0) F.cfg.cwy = BNB;
    if (F.cfg.cwx == 0) F.cfg.cwx = BNB;
    if (set_block_solve_smem(F.cfg) != cudaSuccess)
        FAIL(HDD_ERR_INVALID_ARG, "factor panels of width %d exceed the shared-memory solve", F.cfg.maxK);
    F.re2 = re2;
    F.ready = true;
    return HDD_OK;
}

// Banded solve of every flagged task (FP64; with df, in double-FP32 arithmetic on the FP32 pipe
// where the look-ahead kernel serves); `nact` tasks are expected to be flagged (profiling).
void band_solve(hdd_ctx *ctx, const FactorSet &F, const double2 *in, double2 *out, bool fine,
                const int *flag, cudaStream_t s, int nact = -1, bool df = false) {
    const int nt = (int)ctx->h_tasks.size();
    double fl = 0;
    for (int q = 0; q < nt; q++) fl += F.fma_col[ctx->h_tasks[q].shape];
    // 2 flops per FMA, over 2 real columns (or the one column of a real-equivalent factor)
    fl = (F.re2 ? 2.0 : 4.0) * fl * (nact < 0 ? 1.0 : (double)nact / nt);
    BlockSolveCfg cfg = F.cfg;
    cfg.lookahead = ctx->coarse_la;
    df = df && cfg.lookahead && cfg.la_ring >= 3;
    // SPIKE: each chain split over P parts (a cluster of P CTAs) while every part still gets an
    // SM of its own (two CTAs sharing an SM take as long as the unsplit chain); P = 4, else 2,
    // else the one-CTA solve
    int P = 0, lev = 0;
    if (df && ctx->coarse_spike && F.spike_levels_built && cfg.spike_ok) {
        const int act = nact < 0 ? nt : nact;
        const int chains = (F.re2 ? 1 : 2) * act;      // one cluster per active chain
        if (F.spike_level[1] && chains <= cfg.spike_cap[1]) { P = 4; lev = 1; }
        else if (F.spike_level[0] && chains <= cfg.spike_cap[0]) { P = 2; lev = 0; }
    }
    // double-FP32: 12 FP32 instructions per product of pairs, i.e. 6 per counted flop
    Launch L(ctx, P ? F_CSPK : df ? F_CDF : F_COARSE, F.re2 ? fl * 4.0 : fl * 2.0, df ? 6.0 * fl : fl, s);
    if (P) {
        // clusters for the active chains only: the flagged tasks compacted into a list first
        // (a grid over every task would put the active clusters behind the inactive ones in
        // waves of co-resident clusters)
        const int *list = nullptr;
        int ntl = nt;
        if (flag && nact >= 0 && ctx->d_alist.ensure((size_t)std::max(nt, 1) * sizeof(int)) == cudaSuccess) {
            launch_compact_flags(nt, flag, ctx->d_alist.as<int>(), s);
            ctx->prof.launches++;
            list = ctx->d_alist.as<int>();
            ntl = nact;
        }
        if (ntl == 0) return;
        if (launch_block_solve_spike(P, ctx->d_tasks.as<Task>(), ntl, F.table.as<BlockFactor>(), F.Mdf.as<float2>(),
                                     F.P.as<int>(), F.Meta.as<int4>(), F.spk.as<SpikeInfo>() + (size_t)lev * F.h.size(),
                                     F.G.as<float2>(), in, out, fine ? 1 : 0, flag, list, cfg, F.re2 ? 1 : 0, s))
            return;
    }
    launch_block_solve(ctx->d_tasks.as<Task>(), nt, F.table.as<BlockFactor>(), F.M.as<double>(),
                       F.P.as<int>(), F.Meta.as<int4>(), in, out, fine ? 1 : 0, flag, cfg, F.re2 ? 1 : 0, s,
                       df ? F.Mdf.as<float2>() : nullptr);
}

// Two coarse solves per flagged task in one launch: in[0, ldc) and in[ldc, 2·ldc) into the same
// halves of out (the doubled task table); `flag` (if not null) must cover 2·ntasks entries.
void band_solve2(hdd_ctx *ctx, const FactorSet &F, const double2 *in, double2 *out, const int *flag,
                 cudaStream_t s, bool df = false) {
    const int nt = (int)ctx->h_tasks.size();
    double fl = 0;
    for (int q = 0; q < nt; q++) fl += F.fma_col[ctx->h_tasks[q].shape];
    fl = 2.0 * (F.re2 ? 2.0 : 4.0) * fl;
    BlockSolveCfg cfg = F.cfg;
    cfg.lookahead = ctx->coarse_la;
    df = df && cfg.lookahead && cfg.la_ring >= 3;
    Launch L(ctx, df ? F_CDF : F_COARSE, F.re2 ? fl * 4.0 : fl * 2.0, df ? 6.0 * fl : fl, s);
    launch_block_solve(ctx->d_tasks2.as<Task>(), 2 * nt, F.table.as<BlockFactor>(), F.M.as<double>(),
                       F.P.as<int>(), F.Meta.as<int4>(), in, out, 0, flag, cfg, F.re2 ? 1 : 0, s,
                       df ? F.Mdf.as<float2>() : nullptr);
}

// ---- learned warm start ---------------------------------------------------------------------
hdd_status cnn_buffers(hdd_ctx *ctx) {
    CnnState &C = ctx->cnn;
    const long long ld = ctx->ld;
    const int nt = (int)ctx->h_tasks.size(), nft = (int)ctx->h_ftiles.size();
    CK(C.P.ensure(CNN_NPARAM * sizeof(float))); CK(C.Pb.ensure(CNN_NPARAM * sizeof(__nv_bfloat16)));
    CK(C.M.ensure(CNN_NPARAM * sizeof(float))); CK(C.Vm.ensure(CNN_NPARAM * sizeof(float)));
    CK(C.G.ensure(CNN_NPARAM * sizeof(float)));
    CK(C.sigma.ensure(nt * sizeof(float)));
    CK(C.X0.ensure(ld * 4 * sizeof(float)));
    CK(C.A1.ensure(ld * 32 * sizeof(float))); CK(C.A2.ensure(ld * 32 * sizeof(float)));
    CK(C.A3.ensure(ld * 32 * sizeof(float))); CK(C.A4.ensure(ld * 2 * sizeof(float)));
    CK(C.dA4.ensure(ld * 2 * sizeof(float))); CK(C.Rr.ensure(ld * 2 * sizeof(float)));
    CK(C.dB1.ensure(ld * 32 * sizeof(float))); CK(C.dB2.ensure(ld * 32 * sizeof(float)));
    CK(C.part.ensure((size_t)nft * (CNN_OFF[2] - CNN_OFF[1]) * sizeof(float)));
    CK(C.lpart.ensure(nft * sizeof(float)));
    CK(C.Fh.ensure(ld * sizeof(float2))); CK(C.Q.ensure(ld * sizeof(float2))); CK(C.T2.ensure(ld * sizeof(float2)));
    CK(C.Yc.ensure(ctx->ldc * sizeof(double2))); CK(C.Sc.ensure(ctx->ldc * sizeof(double2)));
    CK(C.Pf.ensure((size_t)nft * LOCAL_LDP * sizeof(float2))); CK(C.Pr.ensure((size_t)nft * LOCAL_LDP * sizeof(float2)));
    CK(C.scale.ensure(nt * sizeof(float))); CK(C.tloss.ensure(nt * sizeof(float)));
    return HDD_OK;
}

// forward pass: input image from the packed right-hand sides, 4 conv layers; A4 holds the output
template <typename R>
void cnn_forward(hdd_ctx *ctx, const c2<R> *f, cudaStream_t s) {
    CnnState &C = ctx->cnn;
    const Task *T = ctx->d_tasks.as<Task>();
    const Tile *ft = ctx->d_ftiles.as<Tile>();
    const int nt = (int)ctx->h_tasks.size(), nft = (int)ctx->h_ftiles.size();
    const __nv_bfloat16 *Wb = C.Pb.as<__nv_bfloat16>();
    const float *P = C.P.as<float>();
    const int CIN[4] = {4, 32, 32, 32}, COUT[4] = {32, 32, 32, 2};
    float *acts[5] = {C.X0.as<float>(), C.A1.as<float>(), C.A2.as<float>(), C.A3.as<float>(), C.A4.as<float>()};
    const double px = (double)ctx->ld;
    KL(F_CNN, px * (8 + 16), 0, launch_cnn_input<R>(T, nt, f, (float)(ctx->k * ctx->h), C.sigma.as<float>(), acts[0],
                                                      C.Fh.as<float2>(), s));
    for (int l = 0; l < 4; l++) {
        const int nw = COUT[l] * 9 * CIN[l];
        KL(F_CNN, px * 4.0 * (CIN[l] + COUT[l]), 2.0 * px * nw,
           launch_conv_fwd(l, T, ft, nft, Wb + CNN_OFF[l], P + CNN_OFF[l] + nw, acts[l], acts[l + 1], s));
    }
}

// Buffers of the tensor-core inference; frame borders zeroed once per task layout.
hdd_status cnn_tc_buffers(hdd_ctx *ctx, cudaStream_t s) {
    CnnState &C = ctx->cnn;
    const size_t act = (size_t)4 * ctx->ptot * sizeof(uint4);
    const bool grow = C.Ba.bytes < act || C.Bb.bytes < act;
    CK(C.Ba.ensure(act)); CK(C.Bb.ensure(act));
    CK(C.Wimg.ensure((size_t)(2 * 9 * 4 * 32 * 8 + 9 * 4 * 16 * 8) * sizeof(__nv_bfloat16)));
    CK(C.err.ensure(sizeof(int)));
    if (!C.pad_ready || grow) {
        CK(cudaMemsetAsync(C.Ba.p, 0, act, s)); CK(cudaMemsetAsync(C.Bb.p, 0, act, s));
        CK(cudaMemsetAsync(C.err.p, 0, sizeof(int), s));
        CK(set_conv_tc_smem(ctx->tc_wmax));
        C.pad_ready = true;
    }
    return HDD_OK;
}

// Inference on the tensor cores: input image (σ, X0), layer 1 on the CUDA cores into BF16
// frames, layers 2-4 as tcgen05 implicit GEMMs; A4 holds the output (FP32, packed layout).
template <typename R>
hdd_status cnn_infer(hdd_ctx *ctx, const c2<R> *f, cudaStream_t s) {
    CnnState &C = ctx->cnn;
    hdd_status st = cnn_tc_buffers(ctx, s);
    if (st != HDD_OK) return st;
    const Task *T = ctx->d_tasks.as<Task>();
    const Tile *ft = ctx->d_ftiles.as<Tile>();
    const int nt = (int)ctx->h_tasks.size(), nft = (int)ctx->h_ftiles.size(), ntc = (int)ctx->h_tct.size();
    const __nv_bfloat16 *Wb = C.Pb.as<__nv_bfloat16>();
    const float *P = C.P.as<float>();
    __nv_bfloat16 *img = C.Wimg.as<__nv_bfloat16>();
    __nv_bfloat16 *img2 = img, *img3 = img + 9 * 4 * 32 * 8, *img4 = img + 2 * 9 * 4 * 32 * 8;
    const double px = (double)ctx->ld, fr = (double)ctx->ptot;
    if (C.tc_dirty) {
        KL(F_CNN, 0, 0, launch_cnn_tc_weights(Wb, img2, img3, img4, s));
        C.tc_dirty = false;
    }
    KL(F_CNN, px * (8 + 16), 0, launch_cnn_input<R>(T, nt, f, (float)(ctx->k * ctx->h), C.sigma.as<float>(),
                                                      C.X0.as<float>(), nullptr, s));
    uint4 *Ba = C.Ba.as<uint4>(), *Bb = C.Bb.as<uint4>();
    KL(F_CNN, px * (16 + 64), 2.0 * px * 32 * 9 * 4,
       launch_cnn_l1_bf16(T, ft, nft, Wb + CNN_OFF[0], P + CNN_OFF[0] + 32 * 9 * 4, C.X0.as<float>(), Ba, ctx->ptot, s));
    int nsm = 0;
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device));
    const int grid = std::max(1, std::min(ntc, 4 * nsm));
    int *err = C.err.as<int>();
    const uint4 *im2 = reinterpret_cast<const uint4 *>(img2), *im3 = reinterpret_cast<const uint4 *>(img3),
                *im4 = reinterpret_cast<const uint4 *>(img4);
    const double fl32 = 2.0 * px * 32 * 9 * 32;
    KL(F_CNN, fr * 128, fl32, launch_conv_tc(32, grid, T, ctx->d_tct.as<int2>(), ntc, Ba, ctx->ptot, im2,
                                             P + CNN_OFF[1] + 32 * 9 * 32, Bb, nullptr, ctx->tc_wmax, err, s));
    KL(F_CNN, fr * 128, fl32, launch_conv_tc(32, grid, T, ctx->d_tct.as<int2>(), ntc, Bb, ctx->ptot, im3,
                                             P + CNN_OFF[2] + 32 * 9 * 32, Ba, nullptr, ctx->tc_wmax, err, s));
    KL(F_CNN, fr * 64 + px * 8, 2.0 * px * 2 * 9 * 32,
       launch_conv_tc(16, grid, T, ctx->d_tct.as<int2>(), ntc, Ba, ctx->ptot, im4, P + CNN_OFF[3] + 2 * 9 * 32,
                      nullptr, reinterpret_cast<float2 *>(C.A4.as<float>()), ctx->tc_wmax, err, s));
    return HDD_OK;
}

// Reads the tensor-core kernels' timeout flag (synchronises the stream); HDD_ERR_TIMEOUT if set.
hdd_status cnn_check_err(hdd_ctx *ctx, cudaStream_t s) {
    CnnState &C = ctx->cnn;
    if (!C.err.p) return HDD_OK;
    int e = 0;
    CK(cudaMemcpyAsync(&e, C.err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (e == 2) {
        // a bulk copy or MMA may have outlived its CTA (kernels_cnn_tc.cu): the context is lost
        ctx->poisoned = true;
        FAIL(HDD_ERR_TIMEOUT, "a tensor-core convolution wait and its drain timed out; work still in "
                              "flight may have written freed memory, so this context refuses further "
                              "work (discard it and its CUDA context)");
    }
    if (e) {
        CK(cudaMemsetAsync(C.err.p, 0, sizeof(int), s));
        FAIL(HDD_ERR_TIMEOUT, "a tensor-core convolution wait timed out");
    }
    return HDD_OK;
}

// mean over the batch of ||f̃/σ - A(a + i b)||²/n_t and its gradient w.r.t. every parameter
// (into C.G, FP32); returns the loss (synchronises).
template <typename R>
hdd_status cnn_loss_grad(hdd_ctx *ctx, const c2<R> *f, double *loss, cudaStream_t s) {
    CnnState &C = ctx->cnn;
    const Task *T = ctx->d_tasks.as<Task>();
    const Tile *ft = ctx->d_ftiles.as<Tile>();
    const int nt = (int)ctx->h_tasks.size(), nft = (int)ctx->h_ftiles.size();
    if (!ctx->E.ready) FAIL(HDD_ERR_STATE, "the training loss needs hdd_setup_deflation");
    cnn_forward<R>(ctx, f, s);
    // deflated residuals in FP32 with the solver's own kernels (coarse solves in FP64):
    //   P f̂, r = f̂ - A y, q = P r, Pᵀ q = q - Z E⁻¹ Zᵀ A q; dL/dy_t = scale_t · A Pᵀ q
    LocalArgs<float> a = local_args<float>(ctx);
    const size_t lsm = local_max_dynamic_smem(ctx->max_nx, (int)sizeof(float2), ctx->frows, ctx->crows);
    if (lsm > 48 * 1024) CK(set_local_smem_limits<float>(lsm));
    float2 *Fh = C.Fh.as<float2>(), *Q = C.Q.as<float2>(), *T2 = C.T2.as<float2>();
    float2 *Rr = reinterpret_cast<float2 *>(C.Rr.as<float>());
    double2 *Yc = C.Yc.as<double2>(), *Sc = C.Sc.as<double2>();
    KL(F_CNN, 0, 0, launch_zt<float>(a, Fh, Yc, 0, nullptr, s));
    band_solve(ctx, ctx->E, Yc, Sc, false, nullptr, s);
    KL(F_CNN, 0, 0, launch_prolong_stencil<float>(a, 1, Fh, Sc, T2, nullptr, 0, C.Pf.as<float2>(), nullptr, s));
    KL(F_CNN, 0, 0, launch_cnn_resid(T, ft, nft, ctx->st, C.X0.as<float>(), C.A4.as<float>(), C.Rr.as<float>(),
                                       C.lpart.as<float>(), s));
    KL(F_CNN, 0, 0, launch_zt<float>(a, Rr, Yc, 0, nullptr, s));
    band_solve(ctx, ctx->E, Yc, Sc, false, nullptr, s);
    KL(F_CNN, 0, 0, launch_prolong_stencil<float>(a, 1, Rr, Sc, Q, nullptr, 0, C.Pr.as<float2>(), nullptr, s));
    KL(F_CNN, 0, 0, launch_zt<float>(a, Q, Yc, 1, nullptr, s));
    band_solve(ctx, ctx->E, Yc, Sc, false, nullptr, s);
    KL(F_CNN, 0, 0, launch_z<float>(a, Sc, Q, T2, nullptr, s, -1.0f));
    KL(F_CNN, 0, 0, launch_cnn_task_scale(T, nt, C.Pf.as<float2>(), C.scale.as<float>(), s));
    KL(F_CNN, 0, 0, launch_cnn_task_loss(T, nt, C.Pr.as<float2>(), C.Pf.as<float2>(), C.tloss.as<float>(), s));
    KL(F_CNN, 0, 0, launch_cnn_out_grad(T, ft, nft, ctx->st, reinterpret_cast<float *>(T2), C.scale.as<float>(),
                                          C.dA4.as<float>(), s));
    const __nv_bfloat16 *Wb = C.Pb.as<__nv_bfloat16>();
    float *G = C.G.as<float>(), *part = C.part.as<float>();
    const int CIN[4] = {4, 32, 32, 32}, COUT[4] = {32, 32, 32, 2};
    float *acts[5] = {C.X0.as<float>(), C.A1.as<float>(), C.A2.as<float>(), C.A3.as<float>(), C.A4.as<float>()};
    // dY of layer 3 is dA4; walk back, alternating the two gradient buffers
    const float *dY = C.dA4.as<float>();
    float *bufs[2] = {C.dB1.as<float>(), C.dB2.as<float>()};
    for (int l = 3; l >= 0; l--) {
        const float *mask = l == 3 ? nullptr : acts[l + 1];            // ReLU of this layer's output
        const int nw = CNN_OFF[l + 1] - CNN_OFF[l];
        KL(F_CNN, 0, 0, launch_conv_bwd_w(l, T, ft, nft, dY, mask, acts[l], part, s));
        KL(F_CNN, 0, 0, launch_sum_partials(part, nft, nw, 1.0f, G + CNN_OFF[l], s));
        if (l > 0) {
            float *dX = bufs[l & 1];
            KL(F_CNN, 0, 0, launch_conv_bwd_data(l, T, ft, nft, Wb + CNN_OFF[l], dY, mask, dX, s));
            dY = dX;
        }
        (void)CIN; (void)COUT;
    }
    CKL();
    std::vector<float> lt(nt);
    CK(cudaMemcpyAsync(lt.data(), C.tloss.p, nt * sizeof(float), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    ctx->prof.harvest();
    double L = 0;
    for (int t = 0; t < nt; t++) L += lt[t];
    if (loss) *loss = L / nt;
    return HDD_OK;
}

template <typename R> InnerWork<R> &work(hdd_ctx *ctx);
template <> InnerWork<float> &work<float>(hdd_ctx *ctx) { return ctx->w32; }
template <> InnerWork<double> &work<double>(hdd_ctx *ctx) { return ctx->w64; }

template <typename R> hdd_status ensure_inner(hdd_ctx *ctx, int R_) {
    InnerWork<R> &W = work<R>(ctx);
    const size_t cs = sizeof(c2<R>);
    const long long ld = ctx->ld, ldc = ctx->ldc, nt = (long long)ctx->h_tasks.size();
    const long long nft = (long long)ctx->h_ftiles.size();
    CK(W.f.ensure(ld * cs)); CK(W.u.ensure(ld * cs)); CK(W.x.ensure(ld * cs)); CK(W.t.ensure(ld * cs));
    CK(W.V.ensure((size_t)(R_ + 1) * ld * cs));
    CK(W.y.ensure(ldc * sizeof(double2))); CK(W.s.ensure((size_t)(R_ + 2) * ldc * sizeof(double2)));
    CK(W.y2.ensure(2 * ldc * sizeof(double2))); CK(W.s2.ensure(2 * ldc * sizeof(double2)));
    CK(W.p1.ensure(nft * LOCAL_LDP * cs)); CK(W.p2.ensure(nft * LOCAL_LDP * cs)); CK(W.p3.ensure(nft * LOCAL_LDP * cs));
    CK(W.H.ensure((size_t)nt * (R_ + 1) * R_ * cs));
    CK(W.cs.ensure((size_t)nt * R_ * sizeof(R)));
    CK(W.sn.ensure((size_t)nt * R_ * cs));
    CK(W.g.ensure((size_t)nt * (R_ + 1) * cs));
    CK(W.ref.ensure(nt * sizeof(R)));
    CK(W.its.ensure(nt * sizeof(int))); CK(W.kcols.ensure(nt * sizeof(int)));
    CK(W.conv.ensure(nt * sizeof(int))); CK(W.rsf.ensure(nt * sizeof(int)));
    CK(W.act0.ensure(nt * sizeof(int))); CK(W.act1.ensure(nt * sizeof(int)));
    CK(W.flagA.ensure(nt * sizeof(int))); CK(W.flagB.ensure(nt * sizeof(int)));
    W.restart = R_;
    size_t smem = local_max_dynamic_smem(ctx->max_nx, (int)cs, ctx->frows, ctx->crows);
    if (smem > 48 * 1024) CK(set_local_smem_limits<R>(smem));
    return HDD_OK;
}

template <typename R> InnerState<R> inner_state(InnerWork<R> &W) {
    InnerState<R> S;
    S.H = W.H.template as<c2<R>>(); S.cs = W.cs.template as<R>(); S.sn = W.sn.template as<c2<R>>();
    S.g = W.g.template as<c2<R>>(); S.ref = W.ref.template as<R>(); S.its = W.its.template as<int>();
    S.kcols = W.kcols.template as<int>(); S.conv = W.conv.template as<int>(); S.restart = W.rsf.template as<int>();
    return S;
}

// Cluster size of the one-launch Arnoldi step for the current task layout: the smallest power of
// two C <= 8 with ceil(ny/C)·nx <= STEP_ROWS_MAX nodes per CTA for every box, raised (up to 8)
// while the device can still hold the clusters of every task at once (more SMs per task, one
// wave); 0 (the separate kernels serve) if no C fits or the device cannot co-schedule a cluster.
template <typename R> int step_plan(hdd_ctx *ctx) {
    const int pi = sizeof(R) == 4 ? 0 : 1;
    if (ctx->step_C[pi] >= 0) return ctx->step_C[pi];
    int max_ny = 0;
    for (const SubBox &b : ctx->subs) max_ny = std::max(max_ny, b.ny);
    int C = 0;
    for (int c = 1; c <= 8; c *= 2) {
        bool ok = true;
        for (const SubBox &b : ctx->subs)
            if ((long long)((b.ny + c - 1) / c) * b.nx > STEP_ROWS_MAX) { ok = false; break; }
        if (ok) { C = c; break; }
    }
    size_t sm = 0;
    if (C > 0) {
        sm = step_smem_bytes(ctx->max_nx, max_ny, C, (int)sizeof(c2<R>));
        if (sm > 160 * 1024 || arnoldi_step_max_cluster<R>(sm, C) < 1) C = 0;
    }
    if (C > 0) {
        const long long nt = (long long)ctx->h_tasks.size();
        while (C < 8) {
            const size_t sm2 = step_smem_bytes(ctx->max_nx, max_ny, 2 * C, (int)sizeof(c2<R>));
            if (sm2 > 160 * 1024 || arnoldi_step_max_cluster<R>(sm2, 2 * C) < nt) break;
            C *= 2;
            sm = sm2;
        }
        arnoldi_step_max_cluster<R>(sm, C);          // leaves the kernels' smem limit at the plan's
    }
    ctx->step_smem[pi] = sm;
    ctx->step_C[pi] = C;
    return C;
}

// All local solves of one RAS application (Eq. 3): z = Σ_j R_jᵀ D_j ũ_j, ũ_j from deflated
// GMRES on P_j A_j ũ = P_j R_j v (Eq. 4), then completed by ũ += Q_j (f̃ - A_j ũ).
// mask (may be null = every task): tasks whose RHS takes part; the others are left untouched.
template <typename R>
hdd_status inner_ras(hdd_ctx *ctx, const double2 *v, double2 *z, const hdd_solve_params *prm,
                     cudaStream_t s, long long *its_total, int *its_max, long long *hits,
                     int *its_out, const int *mask) {
    const int RST = prm->inner_restart;
    hdd_status st = ensure_inner<R>(ctx, RST);
    if (st != HDD_OK) return st;
    if (prm->warm_start && ctx->cnn.ready && (st = cnn_buffers(ctx)) != HDD_OK) return st;
    InnerWork<R> &W = work<R>(ctx);
    InnerState<R> S = inner_state<R>(W);
    LocalArgs<R> a = local_args<R>(ctx);
    const long long ld = ctx->ld, ldc = ctx->ldc;
    const double cs = (double)sizeof(c2<R>);
    const int nt = (int)ctx->h_tasks.size();
    c2<R> *f = W.f.template as<c2<R>>(), *u = W.u.template as<c2<R>>(), *x = W.x.template as<c2<R>>();
    c2<R> *t = W.t.template as<c2<R>>(), *V = W.V.template as<c2<R>>();
    double2 *y = W.y.template as<double2>(), *sc = W.s.template as<double2>();
    c2<R> *p1 = W.p1.template as<c2<R>>(), *p2 = W.p2.template as<c2<R>>(), *p3 = W.p3.template as<c2<R>>();
    int *act[2] = {W.act0.template as<int>(), W.act1.template as<int>()};
    int *cyc = W.flagA.template as<int>(), *rs = W.flagB.template as<int>();
    int *cnt = ctx->d_counter.as<int>();
    const int *ones = ctx->d_ones.as<int>();
    const R tol = (R)prm->inner_tol;
    const int maxit = prm->inner_maxit;
    // the complex64 inner iteration takes its coarse solves in double-FP32 (HDD_OPT_COARSE_DF)
    const bool cdf = sizeof(R) == 4 && ctx->coarse_df;

    const int *all = mask ? mask : ones;
    KL(F_LMISC, ld * (16 + cs), 0, launch_restrict<R>(a, v, ctx->nglob, f, mask, s));
    CK(cudaMemsetAsync(W.its.p, 0, nt * sizeof(int), s));
    CK(cudaMemsetAsync(W.conv.p, 0, nt * sizeof(int), s));
    CK(cudaMemsetAsync(W.kcols.p, 0, nt * sizeof(int), s));
    CK(cudaMemsetAsync(act[0], 0, nt * sizeof(int), s));
    CK(cudaMemsetAsync(act[1], 0, nt * sizeof(int), s));
    const bool warm = prm->warm_start && ctx->cnn.ready;
    if (!warm) {
        CK(cudaMemsetAsync(u, 0, ld * sizeof(c2<R>), s));
        // first cycle from ũ = 0: r0 = P f̃ = f̃ - A Z E⁻¹ Zᵀ f̃, and ref = ||P f̃||
        KL(F_ZT, ld * cs + ldc * 16, 0, launch_zt<R>(a, f, y, 0, mask, s));
        band_solve(ctx, ctx->E, y, sc, false, mask, s, -1, cdf);
        KL(F_PS, 2 * ld * cs + ldc * 16, 0, launch_prolong_stencil<R>(a, 1, f, sc, V, nullptr, 0, p3, mask, s));
    } else {
        // learned initial guess ũ₀ = σ·CNN(f̃/σ) (tensor-core inference); ref = ||P f̃|| and
        // r0 = P(f̃ - A ũ₀)
        if ((st = cnn_infer<R>(ctx, f, s)) != HDD_OK) return st;
        KL(F_CNN, 0, 0, launch_cnn_output<R>(ctx->d_tasks.as<Task>(), ctx->d_ftiles.as<Tile>(),
                                               (int)ctx->h_ftiles.size(), ctx->cnn.sigma.as<float>(),
                                               ctx->cnn.A4.as<float>(), u, mask, s));
        // E⁻¹ Zᵀ f̃ (for ||P f̃||) and E⁻¹ Zᵀ (f̃ - A ũ₀) (for r0) are independent: one launch solves
        // both, the second into slot 0 of sc (kept for the completion)
        double2 *yy = W.y2.template as<double2>(), *ss = W.s2.template as<double2>();
        const int *m2 = nullptr;
        if (mask) {
            int *dm2 = ctx->d_mask2.as<int>();
            CK(cudaMemcpyAsync(dm2, mask, nt * sizeof(int), cudaMemcpyDeviceToDevice, s));
            CK(cudaMemcpyAsync(dm2 + nt, mask, nt * sizeof(int), cudaMemcpyDeviceToDevice, s));
            m2 = dm2;
        }
        KL(F_LMISC, 3 * ld * cs, 0, launch_local_A<R>(a, u, t, f, mask, s));
        KL(F_ZT, ld * cs + ldc * 16, 0, launch_zt<R>(a, f, yy, 0, mask, s));
        KL(F_ZT, ld * cs + ldc * 16, 0, launch_zt<R>(a, t, yy + ldc, 0, mask, s));
        band_solve2(ctx, ctx->E, yy, ss, m2, s, cdf);
        CK(cudaMemcpyAsync(sc, ss + ldc, ldc * sizeof(double2), cudaMemcpyDeviceToDevice, s));
        KL(F_PS, 2 * ld * cs + ldc * 16, 0, launch_prolong_stencil<R>(a, 1, f, ss, x, nullptr, 0, p3, mask, s));
        KL(F_LMISC, 0, 0, launch_set_ref<R>(a, S, p3, mask, s));
        KL(F_PS, 2 * ld * cs + ldc * 16, 0, launch_prolong_stencil<R>(a, 1, t, sc, V, nullptr, 0, p3, mask, s));
    }
    CK(cudaMemsetAsync(cnt, 0, sizeof(int), s));
    KL(F_LMISC, 2 * ld * cs, 0, launch_init_cycle<R>(a, S, RST, V, p3, all, act[0], cnt, tol, maxit, warm ? 0 : 1, s));
    CKL();
    CK(cudaMemcpyAsync(cyc, all, nt * sizeof(int), cudaMemcpyDeviceToDevice, s));
    int cur = 0, nact = 0;
    st = read_counter(ctx, s, &nact);
    if (st != HDD_OK) return st;
    // one launch per Arnoldi step between the coarse solves (cluster per task), or the separate
    // stencil, CGS and Givens kernels
    const int stepC = ctx->fused_inner ? step_plan<R>(ctx) : 0;
    const size_t step_sm = ctx->step_smem[sizeof(R) == 4 ? 0 : 1];
    for (;;) {
        if (stepC > 0 && nact > 0)                        // y = Zᵀ A v_0 of this cycle's tasks
            KL(F_ZT, (double)nact / nt * (ld * cs + ldc * 16), 0, launch_zt<R>(a, V, y, 1, act[cur], s));
        for (int i = 0; i < RST && nact > 0; i++) {
            const int *ain = act[cur];
            int *aout = act[cur ^ 1];
            c2<R> *vi = V + (long long)i * ld, *vn = V + (long long)(i + 1) * ld;
            const double fa = (double)nact / nt;            // fraction of tasks still iterating
            double2 *si = sc + (long long)(i + 1) * ldc;  // E⁻¹ Zᵀ A v_i, kept for the completion
            if (stepC > 0) {
                band_solve(ctx, ctx->E, y, si, false, ain, s, nact, cdf);
                CK(cudaMemsetAsync(aout, 0, nt * sizeof(int), s));
                CK(cudaMemsetAsync(cnt, 0, sizeof(int), s));
                // algorithmic bytes of the fused schedule: 3 passes over V_0..V_i, v_i, v_{i+1}
                // written and read back for the next Zᵀ A, s read and y written
                KL(F_STEP, fa * ((3.0 * i + 7) * ld * cs + 2.0 * ldc * 16), fa * 40.0 * (i + 1) * ld,
                   CK(launch_arnoldi_step<R>(a, stepC, i, RST, V, si, y, S, ain, aout, cnt, tol, maxit, step_sm, s)));
            } else {
                KL(F_ZT, fa * (ld * cs + ldc * 16), 0, launch_zt<R>(a, vi, y, 1, ain, s));
                band_solve(ctx, ctx->E, y, si, false, ain, s, nact, cdf);
                KL(F_PS, fa * ((i + 3) * ld * cs + ldc * 16), fa * 8.0 * (i + 1) * ld,
                   launch_prolong_stencil<R>(a, 0, vi, si, vn, V, i + 1, p1, ain, s));
                KL(F_CGS, fa * (i + 3) * ld * cs, fa * 16.0 * (i + 1) * ld,
                   launch_cgs_update<R>(a, 2, vn, V, i + 1, p1, p2, ain, s));
                KL(F_CGS, fa * (i + 3) * ld * cs, fa * 8.0 * (i + 1) * ld,
                   launch_cgs_update<R>(a, 3, vn, V, i + 1, p2, p3, ain, s));
                CK(cudaMemsetAsync(aout, 0, nt * sizeof(int), s));
                CK(cudaMemsetAsync(cnt, 0, sizeof(int), s));
                KL(F_GIVENS, fa * 2 * ld * cs, 0,
                   launch_givens_normalize<R>(a, S, RST, i, vn, p1, p2, p3, ain, aout, cnt, tol, maxit, s));
            }
            CKL();
            cur ^= 1;
            st = read_counter(ctx, s, &nact);
            if (st != HDD_OK) return st;
        }
        // end of cycle: ũ += V y for the tasks of this cycle; flag the ones needing a restart
        CK(cudaMemsetAsync(cnt, 0, sizeof(int), s));
        CK(cudaMemsetAsync(rs, 0, nt * sizeof(int), s));
        KL(F_LMISC, 0, 0, launch_update_u<R>(a, S, RST, u, V, cyc, rs, cnt, maxit, s));
        CKL();
        int nrs = 0;
        st = read_counter(ctx, s, &nrs);
        if (st != HDD_OK) return st;
        if (nrs == 0) break;
        // restart: r = P(f̃ - A ũ) → v0
        KL(F_LMISC, 0, 0, launch_local_A<R>(a, u, t, f, rs, s));
        KL(F_ZT, 0, 0, launch_zt<R>(a, t, y, 0, rs, s));
        band_solve(ctx, ctx->E, y, sc, false, rs, s, nrs, cdf);
        KL(F_PS, 0, 0, launch_prolong_stencil<R>(a, 1, t, sc, V, nullptr, 0, p3, rs, s));
        CK(cudaMemsetAsync(act[cur], 0, nt * sizeof(int), s));
        CK(cudaMemsetAsync(cnt, 0, sizeof(int), s));
        KL(F_LMISC, 0, 0, launch_init_cycle<R>(a, S, RST, V, p3, rs, act[cur], cnt, tol, maxit, 0, s));
        CKL();
        std::swap(cyc, rs);
        st = read_counter(ctx, s, &nact);
        if (st != HDD_OK) return st;
    }
    // completion x = ũ + Z E⁻¹ Zᵀ (f̃ - A ũ) with E⁻¹ Zᵀ (f̃ - A ũ) = s₀ - Σ y_i s_{i+1}
    // (linearity; every term was solved during the last cycle), then z = Σ R_jᵀ D_j x_j
    double2 *scomp = sc + (long long)(RST + 1) * ldc;
    KL(F_LMISC, (RST + 2) * ldc * 16.0, 0, launch_coarse_combine<R>(a, S, RST, sc, scomp, mask, s));
    KL(F_LMISC, 2 * ld * cs + ldc * 16, 0, launch_z<R>(a, scomp, u, x, mask, s));
    KL(F_LMISC, ld * (cs + 16), 0, launch_scatter<R>(a, x, z, ctx->nglob, mask, s));
    CKL();
    ctx->h_its.resize(nt);
    CK(cudaMemcpyAsync(ctx->h_its.data(), W.its.p, nt * sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    ctx->prof.harvest();
    long long tot = 0, nh = 0;
    int mx = 0;
    for (int q = 0; q < nt; q++) {
        tot += ctx->h_its[q];
        mx = std::max(mx, ctx->h_its[q]);
        if (ctx->h_its[q] >= maxit) nh++;
    }
    if (its_total) *its_total = tot;
    if (its_max) *its_max = mx;
    if (hits) *hits = nh;
    if (its_out) std::copy(ctx->h_its.begin(), ctx->h_its.end(), its_out);
    return HDD_OK;
}

hdd_status exact_ras(hdd_ctx *ctx, const double2 *v, double2 *z, cudaStream_t s, const int *mask) {
    if (!ctx->Aex.ready) FAIL(HDD_ERR_STATE, "direct local solves need hdd_setup_exact");
    hdd_status st = ensure_inner<double>(ctx, 1);
    if (st != HDD_OK) return st;
    InnerWork<double> &W = ctx->w64;
    LocalArgs<double> a = local_args<double>(ctx);
    KL(F_LMISC, ctx->ld * 32, 0, launch_restrict<double>(a, v, ctx->nglob, W.f.as<double2>(), mask, s));
    band_solve(ctx, ctx->Aex, W.f.as<double2>(), W.x.as<double2>(), true, mask, s);
    KL(F_LMISC, ctx->ld * 32, 0, launch_scatter<double>(a, W.x.as<double2>(), z, ctx->nglob, mask, s));
    CKL();
    return HDD_OK;
}

hdd_status ras_apply(hdd_ctx *ctx, const double2 *v, double2 *z, const hdd_solve_params *prm,
                     cudaStream_t s, long long *tot, int *mx, long long *hits, int *its_out,
                     const int *mask = nullptr) {
    if (prm->inner_tol <= 0) {
        if (tot) *tot = 0;
        if (mx) *mx = 0;
        if (hits) *hits = 0;
        return exact_ras(ctx, v, z, s, mask);
    }
    if (!ctx->E.ready) FAIL(HDD_ERR_STATE, "inexact local solves need hdd_setup_deflation");
    if (prm->inner_prec == 64) return inner_ras<float>(ctx, v, z, prm, s, tot, mx, hits, its_out, mask);
    return inner_ras<double>(ctx, v, z, prm, s, tot, mx, hits, its_out, mask);
}

// Rows of A = K - k²M - ik B and of M at a node of each class (node_class) of the impedance
// problem, in the slots of stencil_offset.  Every triangle of the mesh is right-angled with legs
// h, so its element matrices are: stiffness 1 at the right-angle vertex, 1/2 at the other two,
// -1/2 along a leg, 0 along the hypotenuse; mass h²/12 on the diagonal and h²/24 off it.  A row
// sums the triangles around the node that lie in the square; each boundary edge at the node
// (1D P1 mass of length h) adds h/3 to the centre and h/6 to the neighbour along it.
void boundary_rows(int N, double k, int diag, double2 *bcoef, double *bmass) {
    const double h = 1.0 / N;
    for (int cls = 0; cls < 9; cls++) {
        const int cx = cls % 3, cy = cls / 3;
        const int px = cx == 0 ? 0 : (cx == 2 ? N : 1), py = cy == 0 ? 0 : (cy == 2 ? N : 1);
        double K[7] = {}, M[7] = {}, B[7] = {};
        for (int cj = py - 1; cj <= py; cj++)
            for (int ci = px - 1; ci <= px; ci++) {
                if (ci < 0 || ci >= N || cj < 0 || cj >= N) continue;
                // the two triangles of cell (ci, cj) and their right-angle vertices
                int tri[2][3][2], ra[2];
                if (diag == 0) {
                    const int t[2][3][2] = {{{ci, cj}, {ci + 1, cj}, {ci + 1, cj + 1}},
                                            {{ci, cj}, {ci + 1, cj + 1}, {ci, cj + 1}}};
                    std::memcpy(tri, t, sizeof(t));
                    ra[0] = 1; ra[1] = 2;
                } else {
                    const int t[2][3][2] = {{{ci, cj}, {ci + 1, cj}, {ci, cj + 1}},
                                            {{ci + 1, cj}, {ci + 1, cj + 1}, {ci, cj + 1}}};
                    std::memcpy(tri, t, sizeof(t));
                    ra[0] = 0; ra[1] = 1;
                }
                for (int t = 0; t < 2; t++) {
                    int me = -1;
                    for (int v = 0; v < 3; v++)
                        if (tri[t][v][0] == px && tri[t][v][1] == py) me = v;
                    if (me < 0) continue;
                    for (int v = 0; v < 3; v++) {
                        const int dx = tri[t][v][0] - px, dy = tri[t][v][1] - py;
                        const int q = stencil_slot(diag, dx, dy);   // a triangle's vertices are stencil neighbours
                        if (q < 0) continue;
                        if (v == me) {
                            K[q] += (v == ra[t]) ? 1.0 : 0.5;
                            M[q] += h * h / 12.0;
                        } else {
                            K[q] += (dx == 0 || dy == 0) ? -0.5 : 0.0;
                            M[q] += h * h / 24.0;
                        }
                    }
                }
            }
        for (int q = 1; q <= 4; q++) {          // E, W, N, S
            int dx, dy;
            stencil_offset(diag, q, dx, dy);
            const int qx = px + dx, qy = py + dy;
            if (qx < 0 || qx > N || qy < 0 || qy > N) continue;
            const bool on_side = (py == 0 && qy == 0) || (py == N && qy == N) || (px == 0 && qx == 0) ||
                                 (px == N && qx == N);
            if (!on_side) continue;
            B[0] += h / 3.0;
            B[q] += h / 6.0;
        }
        for (int q = 0; q < 7; q++) {
            bcoef[cls * 7 + q] = make_double2(K[q] - k * k * M[q], -k * B[q]);
            bmass[cls * 7 + q] = M[q];
        }
    }
}

hdd_status check_solve_params(hdd_ctx *ctx, const hdd_solve_params *p) {
    if (!p) FAIL(HDD_ERR_INVALID_ARG, "params is NULL");
    if (!(p->outer_tol > 0) || p->outer_maxit < 1 || p->outer_restart < 1)
        FAIL(HDD_ERR_INVALID_ARG, "outer_tol must be > 0, outer_maxit and outer_restart >= 1");
    if (p->inner_tol > 0 && (p->inner_restart < 1 || p->inner_restart > MAX_RESTART || p->inner_maxit < 1))
        FAIL(HDD_ERR_INVALID_ARG, "inner_restart must be in 1..%d and inner_maxit >= 1", MAX_RESTART);
    if (p->inner_prec != 64 && p->inner_prec != 128)
        FAIL(HDD_ERR_INVALID_ARG, "inner_prec must be 64 or 128");
    if (p->two_level != 0 && p->two_level != 1) FAIL(HDD_ERR_INVALID_ARG, "two_level must be 0 or 1");
    if (p->two_level && !ctx->cg.ready) FAIL(HDD_ERR_STATE, "two_level needs hdd_setup_coarse_grid");
    return HDD_OK;
}

// Stages of Q = P A_H⁻¹ Pᵀ (HDD_CG_* bits, applied in the order restrict, solve, prolong) on the
// nrhs vectors of `in`; `active` (per RHS, may be null) skips vectors.  Fine vectors complex128;
// coarse ones in the work precision T inside, complex128 at the boundary.  The last coarse
// result stays in bufA (the hybrid step prolongs it a second time).
template <typename T>
hdd_status cg_stages(hdd_ctx *ctx, int stages, const void *in, void *out, const int *active, cudaStream_t s) {
    auto &G = ctx->cg;
    const long long n = ctx->nglob, mm = (long long)G.m * G.m;
    const int nr = ctx->nrhs;
    CK(G.bufA.ensure((size_t)nr * mm * sizeof(double2)));
    CK(G.bufB.ensure((size_t)nr * mm * sizeof(double2)));
    c2<T> *a = G.bufA.as<c2<T>>(), *b = G.bufB.as<c2<T>>();
    const CGrid g{ctx->N, G.c, G.Nc, G.m, ctx->diag};
    const bool f32 = sizeof(T) == 4;
    const T *S = f32 ? reinterpret_cast<const T *>(G.S32.p) : reinterpret_cast<const T *>(G.S64.p);
    const T *Dinv = f32 ? reinterpret_cast<const T *>(G.D32.p) : reinterpret_cast<const T *>(G.D64.p);
    const double cs = (double)sizeof(c2<T>);
    const c2<T> *cur = nullptr;
    auto coarse_input = [&]() -> hdd_status {      // complex128 coarse input in the work precision
        if (f32) {
            KL(F_CGRID, nr * mm * (16 + cs), 0,
               launch_cg_narrow(nr * mm, (const double2 *)in, reinterpret_cast<float2 *>(a), s));
            cur = a;
        } else {
            cur = reinterpret_cast<const c2<T> *>(in);
        }
        return HDD_OK;
    };
    if (stages & HDD_CG_RESTRICT) {
        KL(F_CGRID, nr * (n * 16.0 + mm * cs), 2.0 * nr * mm * (2 * G.c - 1) * (2 * G.c - 1),
           launch_cg_restrict<T>(g, (const double2 *)in, a, nr, n, mm, active, s));
        cur = a;
    }
    if (stages & HDD_CG_SOLVE) {
        if (!cur) coarse_input();
        // four passes of m³ complex-by-real products each: S Y S, scaled by D⁻¹, then S · S
        const double fl = 4.0 * nr * mm * (double)G.m;
        KL(F_CGRID, 2.0 * nr * mm * cs, fl, launch_dst_pass<T>(G.m, S, nullptr, cur, b, nr, mm, active, s));
        KL(F_CGRID, 2.0 * nr * mm * cs, fl, launch_dst_pass<T>(G.m, S, Dinv, b, a, nr, mm, active, s));
        KL(F_CGRID, 2.0 * nr * mm * cs, fl, launch_dst_pass<T>(G.m, S, nullptr, a, b, nr, mm, active, s));
        KL(F_CGRID, 2.0 * nr * mm * cs, fl, launch_dst_pass<T>(G.m, S, nullptr, b, a, nr, mm, active, s));
        cur = a;
    }
    if (stages & HDD_CG_PROLONG) {
        if (!cur) coarse_input();
        KL(F_CGRID, nr * (n * 16.0 + mm * cs), 0,
           launch_cg_prolong<T>(g, cur, (double2 *)out, 0, nr, n, mm, active, s));
    } else if (f32) {
        KL(F_CGRID, nr * mm * (16 + cs), 0,
           launch_cg_widen(nr * mm, reinterpret_cast<const float2 *>(cur), (double2 *)out, s));
    } else {
        CK(cudaMemcpyAsync(out, cur, (size_t)nr * mm * sizeof(double2), cudaMemcpyDeviceToDevice, s));
    }
    CKL();
    return HDD_OK;
}

// The preconditioner of the outer FGMRES: one-level RAS (Eq. 3), or with two_level the hybrid
// two-level form z = Q v + M_RAS⁻¹(v - A Q v) with Q = P A_H⁻¹ Pᵀ.  The coarse solve runs in
// FP32 with the complex64 inner solves, in FP64 otherwise.  mask: per task, ract: per RHS
// (either may be null = all).
hdd_status precond_apply(hdd_ctx *ctx, const double2 *v, double2 *z, const hdd_solve_params *prm,
                         cudaStream_t s, long long *tot, int *mx, long long *hits, int *its_out,
                         const int *mask, const int *ract) {
    if (!prm->two_level) return ras_apply(ctx, v, z, prm, s, tot, mx, hits, its_out, mask);
    auto &G = ctx->cg;
    if (!G.ready) FAIL(HDD_ERR_STATE, "two_level needs hdd_setup_coarse_grid");
    const long long n = ctx->nglob, mm = (long long)G.m * G.m;
    const int nr = ctx->nrhs;
    CK(G.z0.ensure((size_t)nr * n * sizeof(double2)));
    CK(G.t.ensure((size_t)nr * n * sizeof(double2)));
    double2 *z0 = G.z0.as<double2>(), *t = G.t.as<double2>();
    const bool f32 = prm->inner_tol > 0 && prm->inner_prec == 64;
    const int all = HDD_CG_RESTRICT | HDD_CG_SOLVE | HDD_CG_PROLONG;
    hdd_status st = f32 ? cg_stages<float>(ctx, all, v, z0, ract, s) : cg_stages<double>(ctx, all, v, z0, ract, s);
    if (st != HDD_OK) return st;
    KL(F_CGRID, 3.0 * nr * n * 16, 0, launch_gstencil(ctx->st, ctx->N, z0, t, v, nr, ract, s));  // t = v - A Q v
    CKL();
    if ((st = ras_apply(ctx, t, z, prm, s, tot, mx, hits, its_out, mask)) != HDD_OK) return st;
    // z += Q v, interpolated again from the coarse solution kept in bufA
    const CGrid g{ctx->N, G.c, G.Nc, G.m, ctx->diag};
    if (f32)
        KL(F_CGRID, nr * (2.0 * n * 16 + mm * 8), 0,
           launch_cg_prolong<float>(g, G.bufA.as<float2>(), z, 1, nr, n, mm, ract, s));
    else
        KL(F_CGRID, nr * (2.0 * n * 16 + mm * 16), 0,
           launch_cg_prolong<double>(g, G.bufA.as<double2>(), z, 1, nr, n, mm, ract, s));
    CKL();
    return HDD_OK;
}

}  // namespace

// ===========================================================================================
// Fixed scratch for hdd_apply_PA_noalloc: two complex128 coarse vectors (y = Zᵀ A v and
// s = E⁻¹ y) of at most HDD_NOALLOC_MAX_COARSE entries each, 16 MiB held by every GPU that
// loads the library for the life of the process.  Host code cannot use the symbol itself as a
// device address; the address is looked up with the device current (noalloc_scratch below) and
// cached per device together with the ID of the context it was resolved in.  Each CUDA context
// holds its own copy of the array, and a context created after cudaDeviceReset reloads the
// module at a new address, so a call from a context other than the cached one looks it up again.
// ===========================================================================================
#define HDD_NOALLOC_MAX_COARSE (1 << 19)
#define HDD_NOALLOC_MAX_DEVICES 64
static __device__ __align__(256) double2 g_noalloc_scratch[2 * HDD_NOALLOC_MAX_COARSE];
static double2 *g_noalloc_ptr[HDD_NOALLOC_MAX_DEVICES];
static unsigned long long g_noalloc_ctx[HDD_NOALLOC_MAX_DEVICES];

namespace {
// Unique ID (never reused within the process) of the calling thread's current CUDA context.  The
// driver's cuCtxGetCurrent / cuCtxGetId are reached through the runtime's entry-point query, so
// the library keeps no link-time dependency on libcuda.
cudaError_t current_context_id(unsigned long long *id) {
    using GetCur = int (*)(void **);
    using GetId = int (*)(void *, unsigned long long *);
    static GetCur get_cur = nullptr;
    static GetId get_id = nullptr;
    if (!get_cur || !get_id) {
        void *f1 = nullptr, *f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1);
        if (e != cudaSuccess) return e;
        e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2);
        if (e != cudaSuccess) return e;
        if (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
            return cudaErrorNotSupported;
        get_cur = reinterpret_cast<GetCur>(f1);
        get_id = reinterpret_cast<GetId>(f2);
    }
    void *c = nullptr;
    if (get_cur(&c) != 0 || !c) return cudaErrorDeviceUninitialized;
    if (get_id(c, id) != 0) return cudaErrorDeviceUninitialized;
    return cudaSuccess;
}

// Device address of g_noalloc_scratch in the current context of `device` (looked up on the first
// call from that context).
cudaError_t noalloc_scratch(int device, double2 **out) {
    if (device < 0 || device >= HDD_NOALLOC_MAX_DEVICES) return cudaErrorInvalidDevice;
    unsigned long long cid = 0;
    cudaError_t e = current_context_id(&cid);
    if (e != cudaSuccess) return e;
    if (!g_noalloc_ptr[device] || g_noalloc_ctx[device] != cid) {
        void *p = nullptr;
        if ((e = cudaGetSymbolAddress(&p, g_noalloc_scratch)) != cudaSuccess) return e;
        g_noalloc_ptr[device] = reinterpret_cast<double2 *>(p);
        g_noalloc_ctx[device] = cid;
    }
    *out = g_noalloc_ptr[device];
    return cudaSuccess;
}
}  // namespace

namespace {
// Task and tile tables for nrhs right-hand sides: task t = r·nsub + s solves subdomain s for
// RHS r; fine tiles of ctx->frows box rows, coarse tiles of ctx->crows coarse rows.
hdd_status build_tasks(hdd_ctx *ctx, int nrhs) {
    const int ns = (int)ctx->subs.size();
    // a fine tile holds at most LOCAL_THREADS·FINE_EPT nodes (one register slot per thread each)
    while (ctx->frows > 1 && ctx->frows * ctx->max_nx > LOCAL_THREADS * FINE_EPT) ctx->frows--;
    ctx->h_tasks.clear(); ctx->h_ftiles.clear(); ctx->h_ctiles.clear(); ctx->h_tct.clear();
    ctx->step_C[0] = ctx->step_C[1] = -1;
    ctx->foffs.assign(1, 0); ctx->coffs.assign(1, 0);
    long long fo = 0, co = 0, po = 0;
    int wmx = 0;
    for (int r = 0; r < nrhs; r++)
        for (int q = 0; q < ns; q++) {
            const SubBox &b = ctx->subs[q];
            const int t = r * ns + q;
            Task T{};
            T.nx = b.nx; T.ny = b.ny; T.mx = b.mx; T.my = b.my;
            T.ix0 = b.ix0; T.iy0 = b.iy0; T.ox0 = b.ox0; T.ox1 = b.ox1; T.oy0 = b.oy0; T.oy1 = b.oy1;
            T.shape = ctx->sub_shape[q]; T.sub = q; T.rhs = r;
            T.foff = fo; T.coff = co;
            T.tile0 = (int)ctx->h_ftiles.size();
            for (int y = 0; y < b.ny; y += ctx->frows)
                ctx->h_ftiles.push_back(Tile{t, y, std::min(ctx->frows, b.ny - y)});
            T.ntiles = (int)ctx->h_ftiles.size() - T.tile0;
            for (int y = 0; y < b.my; y += ctx->crows)
                ctx->h_ctiles.push_back(Tile{t, y, std::min(ctx->crows, b.my - y)});
            T.poff = po;
            const int nxp = b.nx + 2;
            for (long long q0 = nxp; q0 < (long long)(b.ny + 1) * nxp; q0 += 128)
                ctx->h_tct.push_back(make_int2(t, (int)q0));
            po += (long long)(b.ny + 2) * nxp;
            wmx = std::max(wmx, b.nx);
            fo += (long long)b.nx * b.ny;
            co += (long long)b.mx * b.my;
            if (r == 0) { ctx->foffs.push_back(fo); ctx->coffs.push_back(co); }
            ctx->h_tasks.push_back(T);
        }
    ctx->ld = fo; ctx->ldc = co;
    ctx->ptot = po;
    ctx->tc_wmax = 128 + 2 * (wmx + 2) + 2;
    ctx->cnn.pad_ready = false;
    const int nt = (int)ctx->h_tasks.size();
    CK(ctx->d_tct.ensure(ctx->h_tct.size() * sizeof(int2)));
    CK(cudaMemcpy(ctx->d_tct.p, ctx->h_tct.data(), ctx->h_tct.size() * sizeof(int2), cudaMemcpyHostToDevice));
    CK(ctx->d_tasks.ensure(nt * sizeof(Task)));
    CK(ctx->d_ftiles.ensure(ctx->h_ftiles.size() * sizeof(Tile)));
    CK(ctx->d_ctiles.ensure(ctx->h_ctiles.size() * sizeof(Tile)));
    CK(ctx->d_ones.ensure(nt * sizeof(int)));
    CK(ctx->d_mask.ensure(nt * sizeof(int)));
    std::vector<int> ones(nt, 1);
    CK(cudaMemcpy(ctx->d_tasks.p, ctx->h_tasks.data(), nt * sizeof(Task), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->d_ftiles.p, ctx->h_ftiles.data(), ctx->h_ftiles.size() * sizeof(Tile), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->d_ctiles.p, ctx->h_ctiles.data(), ctx->h_ctiles.size() * sizeof(Tile), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->d_ones.p, ones.data(), nt * sizeof(int), cudaMemcpyHostToDevice));
    std::vector<Task> t2(ctx->h_tasks);
    t2.insert(t2.end(), ctx->h_tasks.begin(), ctx->h_tasks.end());
    for (int q = nt; q < 2 * nt; q++) t2[q].coff += ctx->ldc;
    CK(ctx->d_tasks2.ensure(2 * (size_t)nt * sizeof(Task)));
    CK(ctx->d_mask2.ensure(2 * (size_t)nt * sizeof(int)));
    CK(cudaMemcpy(ctx->d_tasks2.p, t2.data(), 2 * (size_t)nt * sizeof(Task), cudaMemcpyHostToDevice));
    ctx->nrhs = nrhs;
    return HDD_OK;
}
}  // namespace

namespace {
// Parameter files of the warm-start network: "HDDCNN01", the count n (u32), the CRC-32 of the
// payload (u32), then n FP32 values; integers and floats little-endian.  The CRC is the IEEE
// 802.3 / zlib one (reflected polynomial 0xEDB88320, initial value and final XOR 0xFFFFFFFF),
// computed bit by bit.
const char kWsMagic[8] = {'H', 'D', 'D', 'C', 'N', 'N', '0', '1'};
uint32_t crc32_ieee(const unsigned char *p, size_t n) {
    uint32_t c = 0xFFFFFFFFu;
    for (size_t i = 0; i < n; i++) {
        c ^= p[i];
        for (int k = 0; k < 8; k++) c = (c >> 1) ^ (0xEDB88320u & (0u - (c & 1u)));
    }
    return c ^ 0xFFFFFFFFu;
}
uint32_t rd_le32(const unsigned char *p) {
    return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}
void wr_le32(unsigned char *p, uint32_t v) {
    p[0] = (unsigned char)v; p[1] = (unsigned char)(v >> 8); p[2] = (unsigned char)(v >> 16); p[3] = (unsigned char)(v >> 24);
}
}  // namespace

// ===========================================================================================
// C ABI
// ===========================================================================================
extern "C" {

const char *hdd_status_str(hdd_status s) {
    switch (s) {
        case HDD_OK: return "HDD_OK";
        case HDD_ERR_INVALID_ARG: return "HDD_ERR_INVALID_ARG";
        case HDD_ERR_STATE: return "HDD_ERR_STATE";
        case HDD_ERR_OOM: return "HDD_ERR_OOM";
        case HDD_ERR_CUDA: return "HDD_ERR_CUDA";
        case HDD_ERR_SINGULAR_COARSE: return "HDD_ERR_SINGULAR_COARSE";
        case HDD_ERR_SINGULAR_LOCAL: return "HDD_ERR_SINGULAR_LOCAL";
        case HDD_ERR_NO_CONVERGENCE: return "HDD_ERR_NO_CONVERGENCE";
        case HDD_ERR_BREAKDOWN: return "HDD_ERR_BREAKDOWN";
        case HDD_ERR_NONFINITE: return "HDD_ERR_NONFINITE";
        case HDD_ERR_TIMEOUT: return "HDD_ERR_TIMEOUT";
    }
    return "HDD_UNKNOWN";
}

const char *hdd_last_error(const hdd_ctx *ctx) { return ctx ? ctx->err.c_str() : ""; }

hdd_status hdd_create(hdd_ctx **out, int device) {
    if (!out) return HDD_ERR_INVALID_ARG;
    *out = nullptr;
    int nd = 0;
    if (cudaGetDeviceCount(&nd) != cudaSuccess || device < 0 || device >= nd) return HDD_ERR_CUDA;
    if (cudaSetDevice(device) != cudaSuccess) return HDD_ERR_CUDA;
    hdd_ctx *ctx = new hdd_ctx();
    ctx->device = device;
    if (cudaDeviceGetAttribute(&ctx->nsm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || ctx->nsm < 1)
        ctx->nsm = 152;
    if (cudaMallocHost(&ctx->h_counter, sizeof(int)) != cudaSuccess || ctx->d_counter.ensure(sizeof(int)) != cudaSuccess) {
        delete ctx;
        return HDD_ERR_OOM;
    }
    *out = ctx;
    return HDD_OK;
}

void hdd_destroy(hdd_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    delete ctx;
}

hdd_status hdd_assemble(hdd_ctx *ctx, const hdd_assemble_params *p) {
    if (!ctx) return HDD_ERR_INVALID_ARG;
    if (ctx->poisoned) FAIL(HDD_ERR_TIMEOUT, "context lost: a device wait and its drain timed out earlier");
    if (!p) FAIL(HDD_ERR_INVALID_ARG, "params is NULL");
    if (p->N < 4 || p->N > 65536) FAIL(HDD_ERR_INVALID_ARG, "N must be in 4..65536");
    if (!std::isfinite(p->k) || p->k < 0) FAIL(HDD_ERR_INVALID_ARG, "k must be finite and >= 0");
    if (p->diag != 0 && p->diag != 1) FAIL(HDD_ERR_INVALID_ARG, "diag must be 0 or 1");
    if (p->bc != 0 && p->bc != 1) FAIL(HDD_ERR_INVALID_ARG, "bc must be 0 (Dirichlet) or 1 (impedance)");
    CK(cudaSetDevice(ctx->device));
    ctx->N = p->N; ctx->k = p->k; ctx->diag = p->diag; ctx->h = 1.0 / p->N; ctx->bc = p->bc;
    ctx->nglob = p->bc ? (long long)(p->N + 1) * (p->N + 1) : (long long)(p->N - 1) * (p->N - 1);
    const double kh2 = p->k * p->k * ctx->h * ctx->h;
    // element-by-element P1 assembly on the uniform mesh reduces to this 7-point stencil
    // (stiffness [4; -1 x4], consistent mass h²/12 [6; 1 x6]); see the header comment.
    ctx->st.c0 = 4.0 - kh2 / 2.0;
    ctx->st.c1 = -1.0 - kh2 / 12.0;
    ctx->st.c2 = -kh2 / 12.0;
    ctx->st.diag = p->diag;
    ctx->st.bc = p->bc;
    ctx->st.N = p->N;
    ctx->st.bcoef = nullptr;
    ctx->st.bmass = nullptr;
    if (p->bc) {
        double2 bco[63];
        double bma[63];
        boundary_rows(p->N, p->k, p->diag, bco, bma);
        CK(ctx->d_bcoef.ensure(sizeof(bco)));
        CK(ctx->d_bmass.ensure(sizeof(bma)));
        CK(cudaMemcpy(ctx->d_bcoef.p, bco, sizeof(bco), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(ctx->d_bmass.p, bma, sizeof(bma), cudaMemcpyHostToDevice));
        ctx->st.bcoef = ctx->d_bcoef.as<double2>();
        ctx->st.bmass = ctx->d_bmass.as<double>();
        ctx->cnn.ready = false;               // the warm start serves the Dirichlet problem only
    }
    ctx->assembled = true;
    ctx->dd = false;
    ctx->E.clear(); ctx->Aex.clear();
    ctx->cg.ready = false;
    return HDD_OK;
}

hdd_status hdd_stencil_rows(int N, double k, int diag, double *coef_c128, double *mass) {
    if (N < 4 || N > 65536 || (diag != 0 && diag != 1) || !std::isfinite(k) || k < 0 || !coef_c128)
        return HDD_ERR_INVALID_ARG;
    double2 bco[63];
    double bma[63];
    boundary_rows(N, k, diag, bco, bma);
    for (int i = 0; i < 63; i++) { coef_c128[2 * i] = bco[i].x; coef_c128[2 * i + 1] = bco[i].y; }
    if (mass) std::memcpy(mass, bma, sizeof(bma));
    return HDD_OK;
}

hdd_status hdd_build_rhs(hdd_ctx *ctx, int npoints, const double *points, int nbumps,
                         const double *bumps, void *f_dev, void *stream) {
    if (!ctx) return HDD_ERR_INVALID_ARG;
    if (ctx->poisoned) FAIL(HDD_ERR_TIMEOUT, "context lost: a device wait and its drain timed out earlier");
    if (!ctx->assembled) FAIL(HDD_ERR_STATE, "hdd_assemble first");
    if (!f_dev || !aligned16(f_dev) || npoints < 0 || nbumps < 0 || (npoints && !points) || (nbumps && !bumps))
        FAIL(HDD_ERR_INVALID_ARG, "bad rhs arguments");
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaSetDevice(ctx->device));
    std::vector<double> buf(3 * npoints + 4 * nbumps + 1);
    for (int q = 0; q < 3 * npoints; q++) buf[q] = points[q];
    for (int q = 0; q < 4 * nbumps; q++) buf[3 * npoints + q] = bumps[q];
    CK(ctx->tmp_c.ensure(buf.size() * sizeof(double)));
    CK(cudaMemcpyAsync(ctx->tmp_c.p, buf.data(), buf.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    launch_build_rhs(ctx->st, ctx->N, ctx->h, npoints, ctx->tmp_c.as<double>(), nbumps,
                     ctx->tmp_c.as<double>() + 3 * npoints, (double2 *)f_dev, s);
    CKL();
    CK(cudaStreamSynchronize(s));
    return HDD_OK;
}

hdd_status hdd_apply_A(hdd_ctx *ctx, const void *x_dev, void *y_dev, int nrhs, void *stream) {
    if (!ctx) return HDD_ERR_INVALID_ARG;
    if (ctx->poisoned) FAIL(HDD_ERR_TIMEOUT, "context lost: a device wait and its drain timed out earlier");
    if (!ctx->assembled) FAIL(HDD_ERR_STATE, "hdd_assemble first");
    if (!x_dev || !y_dev || nrhs < 1 || x_dev == y_dev || !aligned16(x_dev) || !aligned16(y_dev))
        FAIL(HDD_ERR_INVALID_ARG, "bad apply_A arguments");
    CK(cudaSetDevice(ctx->device));
    launch_gstencil(ctx->st, ctx->N, (const double2 *)x_dev, (double2 *)y_dev, nullptr, nrhs, nullptr,
                    (cudaStream_t)stream);
    CKL();
    return HDD_OK;
}

hdd_status hdd_setup_dd(hdd_ctx *ctx, const hdd_dd_params *p) {
    if (!ctx) return HDD_ERR_INVALID_ARG;
    if (ctx->poisoned) FAIL(HDD_ERR_TIMEOUT, "context lost: a device wait and its drain timed out earlier");
    if (!ctx->assembled) FAIL(HDD_ERR_STATE, "hdd_assemble first");
    if (!p) FAIL(HDD_ERR_INVALID_ARG, "params is NULL");
    if (p->Sx < 1 || p->Sy < 1 || p->Sx > 4096 || p->Sy > 4096 || p->overlap < 1)
        FAIL(HDD_ERR_INVALID_ARG, "need 1 <= Sx, Sy <= 4096 and overlap >= 1");
    CK(cudaSetDevice(ctx->device));
    const int N = ctx->N;
    auto interfaces = [&](int S, const int *given, std::vector<int> &a) -> bool {
        a.resize(S + 1);
        for (int q = 0; q <= S; q++) a[q] = given ? given[q] : (int)std::floor((double)q * N / S + 0.5);
        if (a[0] != 0 || a[S] != N) return false;
        for (int q = 0; q < S; q++) if (a[q + 1] - a[q] < 2) return false;
        return true;
    };
    std::vector<int> ax, ay;
    if (!interfaces(p->Sx, p->ifx, ax) || !interfaces(p->Sy, p->ify, ay))
        FAIL(HDD_ERR_INVALID_ARG, "interfaces must run 0 = a_0 < ... < a_S = N with gaps >= 2");
    ctx->Sx = p->Sx; ctx->Sy = p->Sy; ctx->overlap = p->overlap;
    ctx->subs.clear(); ctx->shapes.clear(); ctx->sub_shape.clear(); ctx->shape_org.clear();
    // boxes and factors share a shape when (nx, ny) agree and, under the impedance condition,
    // the same sides of the box lie on the boundary of the square (those rows differ)
    std::map<std::pair<std::pair<int, int>, int>, int> shape_id;
    const int d = p->overlap;
    const int lo = ctx->bc ? 0 : 1, hi = ctx->bc ? N : N - 1;   // mesh range of the unknowns
    for (int qy = 0; qy < p->Sy; qy++)
        for (int qx = 0; qx < p->Sx; qx++) {
            SubBox b;
            b.ix0 = std::max(lo, ax[qx] - d + 1); b.ix1 = std::min(hi, ax[qx + 1] + d - 1);
            b.iy0 = std::max(lo, ay[qy] - d + 1); b.iy1 = std::min(hi, ay[qy + 1] + d - 1);
            // owned a_p <= i < a_{p+1}; the last subdomain in each direction also owns hi
            b.ox0 = std::max(lo, ax[qx]); b.ox1 = qx == p->Sx - 1 ? hi : ax[qx + 1] - 1;
            b.oy0 = std::max(lo, ay[qy]); b.oy1 = qy == p->Sy - 1 ? hi : ay[qy + 1] - 1;
            b.nx = b.ix1 - b.ix0 + 1; b.ny = b.iy1 - b.iy0 + 1;
            b.mx = b.nx / 2; b.my = b.ny / 2;
            if (b.nx > 256) FAIL(HDD_ERR_INVALID_ARG, "subdomain box %d nodes wide exceeds 256", b.nx);
            const int sides = ctx->bc ? (b.ix0 == 0) | (b.ix1 == N) << 1 | (b.iy0 == 0) << 2 | (b.iy1 == N) << 3 : 0;
            auto key = std::make_pair(std::make_pair(b.nx, b.ny), sides);
            auto it = shape_id.find(key);
            int sid;
            if (it == shape_id.end()) {
                sid = (int)ctx->shapes.size();
                shape_id[key] = sid;
                ctx->shapes.push_back(key.first);
                ctx->shape_org.push_back(std::make_pair(b.ix0, b.iy0));
            } else {
                sid = it->second;
            }
            ctx->subs.push_back(b);
            ctx->sub_shape.push_back(sid);
        }
    ctx->max_nx = 0; ctx->max_n = 0;
    for (const SubBox &b : ctx->subs) {
        ctx->max_nx = std::max(ctx->max_nx, b.nx);
        ctx->max_n = std::max(ctx->max_n, b.nx * b.ny);
    }
    hdd_status bst = build_tasks(ctx, 1);
    if (bst != HDD_OK) return bst;
    ctx->E.clear(); ctx->Aex.clear();
    ctx->dd = true;
    return HDD_OK;
}

int hdd_num_subdomains(const hdd_ctx *ctx) { return ctx && ctx->dd ? (int)ctx->subs.size() : 0; }

hdd_status hdd_get_subdomain(const hdd_ctx *ctx_, int s, int *info) {
    hdd_ctx *ctx = const_cast<hdd_ctx *>(ctx_);
    if (!ctx) return HDD_ERR_INVALID_ARG;
    if (ctx->poisoned) FAIL(HDD_ERR_TIMEOUT, "context lost: a device wait and its drain timed out earlier");
    if (!ctx->dd) FAIL(HDD_ERR_STATE, "hdd_setup_dd first");
    if (s < 0 || s >= (int)ctx->subs.size() || !info) FAIL(HDD_ERR_INVALID_ARG, "bad subdomain index");
    const SubBox &b = ctx->subs[s];
    int v[12] = {b.ix0, b.ix1, b.iy0, b.iy1, b.ox0, b.ox1, b.oy0, b.oy1, b.nx, b.ny, b.mx, b.my};
    std::memcpy(info, v, sizeof(v));
    return HDD_OK;
}

hdd_status hdd_get_offsets(const hdd_ctx *ctx_, long long *fine_off, long long *coarse_off) {
    hdd_ctx *ctx = const_cast<hdd_ctx *>(ctx_);
    if (!ctx) return HDD_ERR_INVALID_ARG;
    if (ctx->poisoned) FAIL(HDD_ERR_TIMEOUT, "context lost: a device wait and its drain timed out earlier");
    if (!ctx->dd) FAIL(HDD_ERR_STATE, "hdd_setup_dd first");
    if (fine_off) std::copy(ctx->foffs.begin(), ctx->foffs.end(), fine_off);
    if (coarse_off) std::copy(ctx->coffs.begin(), ctx->coffs.end(), coarse_off);
    return HDD_OK;
}

hdd_status hdd_setup_deflation(hdd_ctx *ctx, void *stream) {
    if (!ctx) return HDD_ERR_INVALID_ARG;
    if (ctx->poisoned) FAIL(HDD_ERR_TIMEOUT, "context lost: a device wait and its drain timed out earlier");
    if (!ctx->dd) FAIL(HDD_ERR_STATE, "hdd_setup_dd first");
    CK(cudaSetDevice(ctx->device));
    return build_factors(ctx, ctx->E, true, (cudaStream_t)stream);
}

hdd_status hdd_setup_exact(hdd_ctx *ctx, void *stream) {
    if (!ctx) return HDD_ERR_INVALID_ARG;
    if (ctx->poisoned) FAIL(HDD_ERR_TIMEOUT, "context lost: a device wait and its drain timed out earlier");
    if (!ctx->dd) FAIL(HDD_ERR_STATE, "hdd_setup_dd first");
    CK(cudaSetDevice(ctx->device));
    return build_factors(ctx, ctx->Aex, false, (cudaStream_t)stream);
}

hdd_status hdd_setup_coarse_grid(hdd_ctx *ctx, int c, void *stream) {
    if (!ctx) return HDD_ERR_INVALID_ARG;
    if (ctx->poisoned) FAIL(HDD_ERR_TIMEOUT, "context lost: a device wait and its drain timed out earlier");
    if (!ctx->assembled) FAIL(HDD_ERR_STATE, "hdd_assemble first");
    if (ctx->bc != 0) FAIL(HDD_ERR_INVALID_ARG, "the grid coarse space serves the Dirichlet problem only");
    if (c < 2 || ctx->N % c != 0 || ctx->N / c < 2)
        FAIL(HDD_ERR_INVALID_ARG, "coarsening factor %d must be >= 2 and divide N = %d with N/c >= 2", c, ctx->N);
    CK(cudaSetDevice(ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    auto &G = ctx->cg;
    G.ready = false;
    const int Nc = ctx->N / c, m = Nc - 1;
    const double H = 1.0 / Nc, kH2 = ctx->k * ctx->k * H * H, sc = std::sqrt(2.0 / Nc), pi = 3.141592653589793;
    const size_t mm = (size_t)m * m;
    // orthonormal DST-I: S_ij = sqrt(2/Nc) sin(π (i+1)(j+1) / Nc), the argument reduced modulo 2π
    // exactly in integers; eigenvalues of tridiag(-1, 2, -1): λ_p = 4 sin²(pπ / 2Nc)
    std::vector<double> S(mm), D(mm), lam(m);
    std::vector<float> S32(mm), D32(mm);
    for (int p = 1; p <= m; p++) {
        const double sn = std::sin(pi * p / (2.0 * Nc));
        lam[p - 1] = 4.0 * sn * sn;
    }
    for (int i = 0; i < m; i++)
        for (int j = 0; j < m; j++) {
            const long long t = ((long long)(i + 1) * (j + 1)) % (2LL * Nc);
            S[(size_t)i * m + j] = sc * std::sin(pi * (double)t / Nc);
        }
    double dmin = 1e300, dmax = 0.0;
    for (int q = 0; q < m; q++)
        for (int p = 0; p < m; p++) {
            const double d = lam[p] + lam[q] - kH2;
            dmin = std::min(dmin, std::fabs(d));
            dmax = std::max(dmax, std::fabs(d));
            D[(size_t)q * m + p] = 1.0 / d;
        }
    if (!(dmin > 1e-13 * dmax))
        FAIL(HDD_ERR_SINGULAR_COARSE, "coarse operator singular: min |D| = %.3e (k H on a coarse resonance)", dmin);
    for (size_t e = 0; e < mm; e++) { S32[e] = (float)S[e]; D32[e] = (float)D[e]; }
    CK(G.S64.ensure(mm * sizeof(double))); CK(G.D64.ensure(mm * sizeof(double)));
    CK(G.S32.ensure(mm * sizeof(float))); CK(G.D32.ensure(mm * sizeof(float)));
    CK(cudaMemcpyAsync(G.S64.p, S.data(), mm * sizeof(double), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(G.D64.p, D.data(), mm * sizeof(double), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(G.S32.p, S32.data(), mm * sizeof(float), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(G.D32.p, D32.data(), mm * sizeof(float), cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
    G.c = c; G.Nc = Nc; G.m = m;
    G.ready = true;
    return HDD_OK;
}

long long hdd_coarse_grid_size(const hdd_ctx *ctx) {
    if (!ctx || !ctx->cg.ready) return 0;
    return (long long)ctx->cg.m * ctx->cg.m;
}

hdd_status hdd_coarse_grid_op(hdd_ctx *ctx, int stages, int prec, const void *in_dev, void *out_dev,
                              void *stream) {
    if (!ctx) return HDD_ERR_INVALID_ARG;
    if (ctx->poisoned) FAIL(HDD_ERR_TIMEOUT, "context lost: a device wait and its drain timed out earlier");
    if (!ctx->cg.ready) FAIL(HDD_ERR_STATE, "hdd_setup_coarse_grid first");
    if (stages < 1 || stages > 7)
        FAIL(HDD_ERR_INVALID_ARG, "stages must be a non-empty set of HDD_CG_* bits");
    if (prec != 64 && prec != 128) FAIL(HDD_ERR_INVALID_ARG, "prec must be 64 or 128");
    if (!in_dev || !out_dev || in_dev == out_dev || !aligned16(in_dev) || !aligned16(out_dev))
        FAIL(HDD_ERR_INVALID_ARG, "bad vector arguments");
    CK(cudaSetDevice(ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    hdd_status st = prec == 64 ? cg_stages<float>(ctx, stages, in_dev, out_dev, nullptr, s)
                               : cg_stages<double>(ctx, stages, in_dev, out_dev, nullptr, s);
    if (st != HDD_OK) return st;
    CK(cudaStreamSynchronize(s));
    return HDD_OK;
}

hdd_status hdd_ras_apply(hdd_ctx *ctx, const void *v_dev, void *z_dev, const hdd_solve_params *prm,
                         int *inner_its, void *stream) {
    if (!ctx) return HDD_ERR_INVALID_ARG;
    if (ctx->poisoned) FAIL(HDD_ERR_TIMEOUT, "context lost: a device wait and its drain timed out earlier");
    if (!ctx->dd) FAIL(HDD_ERR_STATE, "hdd_setup_dd first");
    if (!v_dev || !z_dev || v_dev == z_dev || !aligned16(v_dev) || !aligned16(z_dev))
        FAIL(HDD_ERR_INVALID_ARG, "bad vector arguments");
    hdd_status st = check_solve_params(ctx, prm);
    if (st != HDD_OK) return st;
    CK(cudaSetDevice(ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaMemsetAsync(z_dev, 0, (size_t)ctx->nrhs * ctx->nglob * sizeof(double2), s));
    st = precond_apply(ctx, (const double2 *)v_dev, (double2 *)z_dev, prm, s, nullptr, nullptr, nullptr, inner_its,
                       nullptr, nullptr);
    if (st != HDD_OK) return st;
    CK(cudaStreamSynchronize(s));
    return HDD_OK;
}

hdd_status hdd_solve(hdd_ctx *ctx, const void *f_dev, void *x_dev, const hdd_solve_params *prm,
                     hdd_solve_stats *stats, void *stream) {
    if (!ctx) return HDD_ERR_INVALID_ARG;
    if (ctx->poisoned) FAIL(HDD_ERR_TIMEOUT, "context lost: a device wait and its drain timed out earlier");
    if (!ctx->dd) FAIL(HDD_ERR_STATE, "hdd_setup_dd first");
    if (!f_dev || !x_dev || f_dev == x_dev || !aligned16(f_dev) || !aligned16(x_dev))
        FAIL(HDD_ERR_INVALID_ARG, "bad vector arguments");
    hdd_status st = check_solve_params(ctx, prm);
    if (st != HDD_OK) return st;
    if (prm->inner_tol > 0 && !ctx->E.ready) FAIL(HDD_ERR_STATE, "hdd_setup_deflation first");
    if (prm->inner_tol <= 0 && !ctx->Aex.ready) FAIL(HDD_ERR_STATE, "hdd_setup_exact first");
    CK(cudaSetDevice(ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    auto t0 = std::chrono::steady_clock::now();
    const long long n = ctx->nglob;
    const int nr = ctx->nrhs, ns = (int)ctx->subs.size();
    const int R = std::min(prm->outer_restart, prm->outer_maxit);
    OuterWork &O = ctx->ow;
    const int G = outer_grid(n);
    const int ldp = R + 1;
    OuterBatch B{nr, n, (long long)nr * n, ldp, G, R, nullptr};
    B.n32 = n + (n & 1);
    B.ld32 = (long long)nr * B.n32;
    CK(O.D.ensure((size_t)(R + 1) * nr * n * sizeof(double)));
    B.D = O.D.as<double>();
    CK(O.V.ensure((size_t)(R + 1) * nr * n * sizeof(double2)));
    CK(O.Z.ensure((size_t)R * nr * n * sizeof(double2)));
    CK(O.w.ensure((size_t)nr * n * sizeof(double2))); CK(O.r.ensure((size_t)nr * n * sizeof(double2)));
    CK(O.H.ensure((size_t)nr * (R + 1) * R * sizeof(double2)));
    CK(O.cs.ensure((size_t)nr * R * sizeof(double))); CK(O.sn.ensure((size_t)nr * R * sizeof(double2)));
    CK(O.g.ensure((size_t)nr * (R + 1) * sizeof(double2)));
    CK(O.Wq.ensure((size_t)nr * (R + 1) * sizeof(double2)));
    CK(O.h1.ensure((size_t)nr * ldp * sizeof(double2))); CK(O.h2.ensure((size_t)nr * ldp * sizeof(double2)));
    CK(O.y.ensure((size_t)nr * ldp * sizeof(double2)));
    // the double-FP32 first pass runs on a grid of its own, three CTAs per SM (its register
    // budget), at least as many CTAs as the other kernels: more of the basis in flight per SM;
    // its partials share the buffer
    OuterBatch Bd = B;
    Bd.G = std::max(G, 3 * ctx->nsm);
    CK(O.part.ensure((size_t)nr * Bd.G * ldp * sizeof(double2)));
    CK(O.npart.ensure((size_t)nr * G * sizeof(double)));
    const int Gu = oupdate_df_grid(n);          // partials of the double-FP32 first-pass update
    CK(O.npart1.ensure((size_t)nr * std::max(G, Gu) * sizeof(double)));
    const bool r32 = prm->outer_reorth32 != 0;
    // the double-FP32 first pass pairs with the guarded FP32 second pass (its coefficients are
    // what that guard tests); with the FP64 second pass both passes stay FP64
    const bool df = r32 && ctx->outer_df;
    if (r32) CK(O.V32.ensure((size_t)(R + 1) * B.ld32 * sizeof(float2)));
    if (df) CK(O.V32L.ensure((size_t)(R + 1) * B.ld32 * sizeof(float2)));
    float2 *V32 = r32 ? O.V32.as<float2>() : nullptr;
    float2 *V32L = df ? O.V32L.as<float2>() : nullptr;
    // delayed CGS2 (two passes over the basis per step) with the double-FP32 dots and update
    const bool dc = df && ctx->outer_udf && ctx->outer_dcgs;
    const int Gc = oupdate_dcgs_grid(n);        // partials of its update
    if (dc) {
        CK(O.part2.ensure((size_t)nr * G * ldp * sizeof(double2)));
        CK(O.invs.ensure(nr * sizeof(double)));
        CK(O.vmax.ensure((size_t)nr * ldp * sizeof(unsigned)));
        CK(O.err.ensure(sizeof(int)));
        CK(O.close.ensure(nr * sizeof(int)));
        CK(O.npart1.ensure((size_t)nr * std::max(std::max(G, Gu), Gc) * sizeof(double)));
        CK(cudaMemsetAsync(O.err.p, 0, sizeof(int), s));
    }
    CK(O.fallbacks.ensure(sizeof(int)));
    CK(cudaMemsetAsync(O.fallbacks.p, 0, sizeof(int), s));
    CK(O.hn.ensure(nr * sizeof(double))); CK(O.flag.ensure(nr * sizeof(int))); CK(O.beta.ensure(nr * sizeof(double)));
    CK(O.fnorm.ensure(nr * sizeof(double))); CK(O.act.ensure(nr * sizeof(int))); CK(O.kcols.ensure(nr * sizeof(int)));
    CK(O.hist.ensure((size_t)nr * (prm->outer_maxit + 1) * sizeof(double)));
    const size_t osm = (size_t)(R + 1) * 3 * sizeof(double);   // dynamic: h (update), y (axpy, trisolve)
    if (osm + 40 * 1024 > 227 * 1024) FAIL(HDD_ERR_INVALID_ARG, "outer restart %d too long", R);
    CK(set_outer_smem_limits(osm));
    double2 *V = O.V.as<double2>(), *Zb = O.Z.as<double2>(), *w = O.w.as<double2>(), *rv = O.r.as<double2>();
    const double2 *f = (const double2 *)f_dev;
    double2 *x = (double2 *)x_dev;
    const int hstride = prm->outer_maxit + 1;
    hdd_solve_stats loc{};
    hdd_solve_stats &S = stats ? *stats : loc;
    std::memset(&S, 0, sizeof(S));
    ctx->hist.clear();
    CK(cudaMemsetAsync(x, 0, (size_t)nr * n * sizeof(double2), s));
    // ||f_r|| for every RHS (host sums the per-CTA partials in CTA order)
    std::vector<double> fn(nr), part((size_t)nr * G), beta(nr);
    KL(F_OMISC, (double)nr * n * 16, 0, launch_onorm(B, f, O.npart.as<double>(), s));
    CKL();
    CK(cudaMemcpyAsync(part.data(), O.npart.p, part.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    ctx->prof.harvest();
    for (int r = 0; r < nr; r++) {
        double a = 0;
        for (int q = 0; q < G; q++) a += part[(size_t)r * G + q];
        fn[r] = std::sqrt(a);
        if (!std::isfinite(fn[r])) FAIL(HDD_ERR_NONFINITE, "right-hand side %d is not finite", r);
    }
    CK(cudaMemcpyAsync(O.fnorm.p, fn.data(), nr * sizeof(double), cudaMemcpyHostToDevice, s));
    // per-RHS state: done[r] once its true residual meets the tolerance (zero RHS: at once)
    std::vector<int> done(nr), act(nr), kcols(nr), its(nr, 0), tmask((size_t)nr * ns);
    std::vector<double> relres(nr, 0.0);
    for (int r = 0; r < nr; r++) done[r] = fn[r] == 0.0;
    int total = 0;
    long long inner_tot = 0, hits = 0;
    int inner_mx = 0;
    hdd_status result = HDD_OK;
    const int *dact = O.act.as<int>();
    auto push_active = [&]() -> hdd_status {
        for (int r = 0; r < nr; r++)
            for (int q = 0; q < ns; q++) tmask[(size_t)r * ns + q] = act[r];
        CK(cudaMemcpyAsync(O.act.p, act.data(), nr * sizeof(int), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(ctx->d_mask.p, tmask.data(), tmask.size() * sizeof(int), cudaMemcpyHostToDevice, s));
        return HDD_OK;
    };
    for (;;) {
        // true residuals r = f - A x of the RHS still running, β_r, v_{r,0}, g_r
        for (int r = 0; r < nr; r++) act[r] = !done[r];
        if ((st = push_active()) != HDD_OK) return st;
        B.active = dact;
        Bd.active = dact;
        KL(F_OMISC, 3.0 * nr * n * 16, 0, launch_gstencil(ctx->st, ctx->N, x, rv, f, nr, dact, s));
        KL(F_OMISC, (double)nr * n * 16, 0, launch_onorm(B, rv, O.npart.as<double>(), s));
        KL(F_OMISC, 2.0 * nr * n * 16 + (r32 ? nr * n * 8.0 : 0.0) + (df ? nr * n * 8.0 : 0.0), 0,
           launch_oinit(B, rv, O.npart.as<double>(), V, V32, V32L, O.D.as<double>(), O.g.as<double2>(),
                        O.Wq.as<double2>(), O.beta.as<double>(), s));
        CKL();
        CK(cudaMemcpyAsync(beta.data(), O.beta.p, nr * sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        ctx->prof.harvest();
        bool any = false;
        for (int r = 0; r < nr; r++) {
            if (done[r]) continue;
            if (!std::isfinite(beta[r])) { result = HDD_ERR_NONFINITE; ctx->err = "non-finite outer residual"; done[r] = 1; continue; }
            relres[r] = beta[r] / fn[r];
            if (relres[r] <= prm->outer_tol) { done[r] = 1; continue; }
            any = true;
        }
        if (!any) break;
        if (total >= prm->outer_maxit) { result = HDD_ERR_NO_CONVERGENCE; ctx->err = "outer_maxit reached"; break; }
        for (int r = 0; r < nr; r++) { act[r] = !done[r]; kcols[r] = 0; }
        if ((st = push_active()) != HDD_OK) return st;
        for (int j = 0; j < R; j++) {
            double2 *vj = V + (long long)j * B.ld, *zj = Zb + (long long)j * B.ld;
            long long it_tot = 0, it_hits = 0;
            int it_mx = 0;
            st = precond_apply(ctx, vj, zj, prm, s, &it_tot, &it_mx, &it_hits, nullptr, ctx->d_mask.as<int>(), dact);
            if (st != HDD_OK) return st;
            inner_tot += it_tot; hits += it_hits; inner_mx = std::max(inner_mx, it_mx);
            int nact = 0;
            for (int r = 0; r < nr; r++) nact += act[r];
            const double nv = j + 1, fa = nact;
            KL(F_OMISC, 2.0 * fa * n * 16, 0, launch_gstencil(ctx->st, ctx->N, zj, w, nullptr, nr, dact, s));  // w = A z_j
            if (dc) {
                // delayed CGS2: one double-FP32 pass for V^H ṽ_j and V^H w (slots 0..j), the
                // per-RHS completion of column j-1, one pass writing v_j and w', the tentative
                // stopping test of column j, then ṽ_{j+1} = w'/ν_{j+1} into slot j+1
                double2 *P1 = O.h2.as<double2>(), *P2 = O.h1.as<double2>();
                if (j == 0) {
                    KL(F_ODF, fa * 32.0 * n, fa * 48.0 * n,
                       launch_odots_df(Bd, V32, V32L, 1, w, O.part.as<double2>(), s));
                    KL(F_OMISC, 0, 0, launch_oreduce(Bd, O.part.as<double2>(), 1, P2, s));
                } else {
                    // two compensated complex dot products per basis vector and element: 96 FP32
                    // instructions with the two-sum, 72 with the first pass's biased accumulators
                    KL(F_ODF, fa * (nv * 16 + 32) * n, fa * (ctx->outer_bias ? 72 : 96) * nv * n,
                       CK(launch_odots2_df(B, V32, V32L, j + 1, V32 + (long long)j * B.ld32,
                                           V32L + (long long)j * B.ld32, w, O.part.as<double2>(),
                                           O.part2.as<double2>(), O.vmax.as<unsigned>(), ctx->outer_bias, s)));
                    KL(F_OMISC, 0, 0, launch_oreduce(B, O.part.as<double2>(), j + 1, P1, s));
                    KL(F_OMISC, 0, 0, launch_oreduce(B, O.part2.as<double2>(), j + 1, P2, s));
                }
                KL(F_OMISC, 0, 0,
                   launch_dcgs_col(B, O.H.as<double2>(), O.cs.as<double>(), O.sn.as<double2>(), O.g.as<double2>(),
                                   O.Wq.as<double2>(), j, P1, P2, O.hn.as<double>(), O.invs.as<double>(),
                                   O.fnorm.as<double>(), O.hist.as<double>(), hstride, total, O.err.as<int>(),
                                   O.vmax.as<unsigned>(), s));
                // bytes: hi/lo of slots 0..j-1, slot j read and rewritten (FP64, Re - Im, hi/lo), w
                // read and written; ≈ 56 FP32 instructions per basis vector and element
                KL(F_OUDF, fa * ((nv - 1) * 16 + 16 + 40 + 32) * n, fa * 56 * (nv - 1) * n,
                   launch_oupdate_dcgs(B, V32, V32L, j, j > 0 ? 1 : 0, V + (long long)j * B.ld,
                                       O.D.as<double>() + (long long)j * B.ld, V32 + (long long)j * B.ld32,
                                       V32L + (long long)j * B.ld32, P1, P2, O.invs.as<double>(), w,
                                       O.npart1.as<double>(), O.vmax.as<unsigned>(), s));
                KL(F_OMISC, 0, 0,
                   launch_dcgs_tent(B, O.H.as<double2>(), O.g.as<double2>(), O.Wq.as<double2>(), j,
                                    O.npart1.as<double>(), Gc, O.fnorm.as<double>(), prm->outer_tol,
                                    O.hn.as<double>(), O.flag.as<int>(), O.hist.as<double>(), hstride, total, s));
                KL(F_OMISC, 2.0 * fa * n * 16 + fa * n * 16.0, 0,
                   launch_oscale(B, V + (long long)(j + 1) * B.ld, V32 + (long long)(j + 1) * B.ld32,
                                 V32L + (long long)(j + 1) * B.ld32, O.D.as<double>() + (long long)(j + 1) * B.ld, w,
                                 O.hn.as<double>(), s));
            } else {
                // CGS2 flops as executed: dots and update 6 per (vector, element) each (three FMAs,
                // Gauss form); bytes: V (16 B) and d (8 B) per vector and element for each pass over
                // the basis (k_oupdate with dots makes two: the update, then the dots of the updated
                // w), and w
                if (df) {     // 16 B (hi + lo FP32) per vector and element; 4 real products of ~12 FP32 ops
                    KL(F_ODF, fa * (nv * 16 + 16) * n, fa * 48 * nv * n,
                       launch_odots_df(Bd, V32, V32L, j + 1, w, O.part.as<double2>(), s));             // h1 = V^H w
                    KL(F_OMISC, 0, 0, launch_oreduce(Bd, O.part.as<double2>(), j + 1, O.h1.as<double2>(), s));
                } else {
                    KL(F_OCGS, fa * (nv * 24 + 16) * n, fa * 6 * nv * n,
                       launch_odots(B, V, j + 1, w, O.part.as<double2>(), s));                          // h1 = V^H w
                    KL(F_OMISC, 0, 0, launch_oreduce(B, O.part.as<double2>(), j + 1, O.h1.as<double2>(), s));
                }
                int g1 = G;   // norm partials of w' = w - V h1
                if (df) {     // update w' = w - V h1, then h2 = V^H w' in double-FP32 (16 B)
                    if (ctx->outer_udf) {   // double-FP32 update from the hi/lo copies: 16 B, ≈ 48 FP32 instructions
                        g1 = Gu;
                        KL(F_OUDF, fa * (nv * 16 + 32) * n, fa * 48 * nv * n,
                           launch_oupdate_df(B, V32, V32L, j + 1, O.h1.as<double2>(), w, O.npart1.as<double>(), s));
                    } else {                // FP64 Gauss form: 24 B, 3 FMAs
                        KL(F_OCGS, fa * (nv * 24 + 32) * n, fa * 6 * nv * n,
                           launch_oupdate(B, V, j + 1, O.h1.as<double2>(), w, nullptr, O.npart1.as<double>(), s));
                    }
                    KL(F_ODF, fa * (nv * 16 + 16) * n, fa * 48 * nv * n,
                       launch_odots_df(Bd, V32, V32L, j + 1, w, O.part.as<double2>(), s));
                    KL(F_OMISC, 0, 0, launch_oreduce(Bd, O.part.as<double2>(), j + 1, O.h2.as<double2>(), s));
                } else {
                    KL(F_OCGS, fa * (nv * 48 + 32) * n, fa * 12 * nv * n,
                       launch_oupdate(B, V, j + 1, O.h1.as<double2>(), w, O.part.as<double2>(), O.npart1.as<double>(), s));
                    KL(F_OMISC, 0, 0, launch_oreduce(B, O.part.as<double2>(), j + 1, O.h2.as<double2>(), s));
                }
                if (r32)   // FP32 correction from the FP32 basis copy (guarded; FP64 fallback inside)
                    KL(F_OREORTH, fa * (nv * 8 + 2 * 16) * n, fa * 8 * nv * n,
                       launch_oupdate2(B, V, V32, j + 1, O.h2.as<double2>(), w, O.npart1.as<double>(), g1,
                                       O.npart.as<double>(), 1, O.fallbacks.as<int>(), s));
                else
                    KL(F_OCGS, fa * (nv * 24 + 32) * n, fa * 6 * nv * n,
                       launch_oupdate(B, V, j + 1, O.h2.as<double2>(), w, nullptr, O.npart.as<double>(), s));
                KL(F_OMISC, 0, 0,
                   launch_ogivens(B, O.H.as<double2>(), O.cs.as<double>(), O.sn.as<double2>(), O.g.as<double2>(),
                                  O.Wq.as<double2>(), j,
                                  O.h1.as<double2>(), O.h2.as<double2>(), O.npart.as<double>(), O.fnorm.as<double>(),
                                  prm->outer_tol, O.hn.as<double>(), O.flag.as<int>(), O.hist.as<double>(), hstride,
                                  total, s));
                KL(F_OMISC, 2.0 * fa * n * 16 + (r32 ? fa * n * 8.0 : 0.0) + (df ? fa * n * 8.0 : 0.0), 0,
                   launch_oscale(B, V + (long long)(j + 1) * B.ld, r32 ? V32 + (long long)(j + 1) * B.ld32 : nullptr,
                                 df ? V32L + (long long)(j + 1) * B.ld32 : nullptr,
                                 O.D.as<double>() + (long long)(j + 1) * B.ld, w, O.hn.as<double>(), s));
            }
            CKL();
            total++;
            std::vector<int> flags(nr);
            int berr = 0;
            CK(cudaMemcpyAsync(flags.data(), O.flag.p, nr * sizeof(int), cudaMemcpyDeviceToHost, s));
            if (dc) CK(cudaMemcpyAsync(&berr, O.err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            ctx->prof.harvest();
            if (berr) FAIL(HDD_ERR_NONFINITE, "outer orthogonalisation: a pending basis vector lost half its norm");
            bool changed = false, more = false;
            std::vector<int> closev(nr, 0);
            for (int r = 0; r < nr; r++) {
                if (!act[r]) continue;
                its[r]++;
                kcols[r] = j + 1;
                if (!flags[r]) { act[r] = 0; changed = true; closev[r] = 1; } else more = true;
            }
            const bool stop = !more || total >= prm->outer_maxit || j == R - 1;
            if (dc) {   // the cycle ends for these RHS: commit the rotation of their tentative column j
                bool anyc = false;
                for (int r = 0; r < nr; r++) {
                    if (stop && act[r]) closev[r] = 1;
                    anyc = anyc || closev[r];
                }
                if (anyc) {
                    CK(cudaMemcpyAsync(O.close.p, closev.data(), nr * sizeof(int), cudaMemcpyHostToDevice, s));
                    KL(F_OMISC, 0, 0, launch_dcgs_close(B, O.H.as<double2>(), O.cs.as<double>(), O.sn.as<double2>(),
                                                        O.g.as<double2>(), O.Wq.as<double2>(), j, O.close.as<int>(), s));
                    CKL();
                }
            }
            if (stop) break;
            if (changed && (st = push_active()) != HDD_OK) return st;
        }
        // x_r += Z_r y_r, y_r = H_r⁻¹ g_r, for every RHS that ran in this cycle
        int kmax = 0;
        for (int r = 0; r < nr; r++) kmax = std::max(kmax, kcols[r]);
        CK(cudaMemcpyAsync(O.kcols.p, kcols.data(), nr * sizeof(int), cudaMemcpyHostToDevice, s));
        if (kmax > 0) {
            KL(F_OMISC, 0, 0, launch_orotate(B, O.H.as<double2>(), O.cs.as<double>(), O.sn.as<double2>(),
                                             O.kcols.as<int>(), kmax, s));
            KL(F_OMISC, 0, 0, launch_otrisolve(B, O.H.as<double2>(), O.g.as<double2>(), O.kcols.as<int>(), kmax,
                                               O.y.as<double2>(), s));
            KL(F_OMISC, (kmax + 2.0) * nr * n * 16, 8.0 * kmax * nr * n,
               launch_oaxpy(B, O.y.as<double2>(), O.kcols.as<int>(), kmax, Zb, x, s));
            CKL();
        }
    }
    CK(cudaStreamSynchronize(s));
    ctx->prof.harvest();
    auto t1 = std::chrono::steady_clock::now();
    // residual history of the first RHS (per-RHS histories stay on the device)
    const int n0 = its[0];
    ctx->hist.resize(n0);
    if (n0) CK(cudaMemcpy(ctx->hist.data(), O.hist.p, n0 * sizeof(double), cudaMemcpyDeviceToHost));
    int fb = 0;
    CK(cudaMemcpy(&fb, O.fallbacks.p, sizeof(int), cudaMemcpyDeviceToHost));
    if (prm->warm_start && ctx->cnn.ready && (st = cnn_check_err(ctx, s)) != HDD_OK) return st;
    double worst = 0;
    for (int r = 0; r < nr; r++) worst = std::max(worst, relres[r]);
    S.outer_its = total;
    S.status = result;
    S.rel_res_true = worst;
    S.inner_its_total = inner_tot;
    long long solves = 0;
    for (int r = 0; r < nr; r++) solves += (long long)its[r] * ns;
    S.inner_its_avg = solves ? (double)inner_tot / (double)solves : 0.0;
    S.inner_its_max = inner_mx;
    S.inner_maxit_hits = hits;
    S.t_solve_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
    S.n_history = n0;
    S.res_history = ctx->hist.data();
    S.outer_reorth_fp64 = fb;
    return result;
}

hdd_status hdd_autotune(hdd_ctx *ctx, const hdd_solve_params *prm, void *stream, int *fine_rows,
                        int *coarse_rows, double *best_ms) {
    if (!ctx) return HDD_ERR_INVALID_ARG;
    if (ctx->poisoned) FAIL(HDD_ERR_TIMEOUT, "context lost: a device wait and its drain timed out earlier");
    if (!ctx->dd) FAIL(HDD_ERR_STATE, "hdd_setup_dd first");
    hdd_status st = check_solve_params(ctx, prm);
    if (st != HDD_OK) return st;
    if (prm->inner_tol > 0 && !ctx->E.ready) FAIL(HDD_ERR_STATE, "hdd_setup_deflation first");
    if (prm->inner_tol <= 0 && !ctx->Aex.ready) FAIL(HDD_ERR_STATE, "hdd_setup_exact first");
    CK(cudaSetDevice(ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    const long long nv = (long long)ctx->nrhs * ctx->nglob;
    DevMem v, z;
    CK(v.ensure((size_t)nv * sizeof(double2)));
    CK(z.ensure((size_t)nv * sizeof(double2)));
    launch_fill_test(nv, 0x9e3779b97f4a7c15ULL, v.as<double2>(), s);
    CKL();
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); FAIL(HDD_ERR_CUDA, "cudaEventCreate"); }
    const int f0 = ctx->frows, c0 = ctx->crows;
    int bf = f0, bc = c0;
    float best = 3.0e38f;
    const int Fc[] = {4, 6, 8, 12, 16, 24}, Cc[] = {2, 4, 8};
    for (int f : Fc) {
        if (f * ctx->max_nx > LOCAL_THREADS * FINE_EPT) continue;
        for (int c : Cc) {
            if (local_max_dynamic_smem(ctx->max_nx, (int)sizeof(double2), f, c) > 227 * 1024) continue;
            ctx->frows = f; ctx->crows = c;
            if ((st = build_tasks(ctx, ctx->nrhs)) != HDD_OK) break;
            float t = 3.0e38f;
            for (int rep = 0; rep < 3 && st == HDD_OK; rep++) {      // rep 0: buffers, attributes
                if (cudaMemsetAsync(z.p, 0, (size_t)nv * sizeof(double2), s) != cudaSuccess ||
                    cudaEventRecord(e0, s) != cudaSuccess) { st = HDD_ERR_CUDA; break; }
                st = ras_apply(ctx, v.as<double2>(), z.as<double2>(), prm, s, nullptr, nullptr, nullptr, nullptr);
                if (st != HDD_OK) break;
                float ms = 0.f;
                if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                    cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) { st = HDD_ERR_CUDA; break; }
                if (rep > 0) t = std::min(t, ms);
            }
            if (st != HDD_OK) break;
            if (t < best) { best = t; bf = f; bc = c; }
        }
        if (st != HDD_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->prof.harvest();
    if (st != HDD_OK) { bf = f0; bc = c0; }
    ctx->frows = bf; ctx->crows = bc;
    const hdd_status st2 = build_tasks(ctx, ctx->nrhs);
    if (st != HDD_OK) return st;
    if (st2 != HDD_OK) return st2;
    if (fine_rows) *fine_rows = bf;
    if (coarse_rows) *coarse_rows = bc;
    if (best_ms) *best_ms = best;
    return HDD_OK;
}

hdd_status hdd_setup_batch(hdd_ctx *ctx, int nrhs) {
    if (!ctx) return HDD_ERR_INVALID_ARG;
    if (ctx->poisoned) FAIL(HDD_ERR_TIMEOUT, "context lost: a device wait and its drain timed out earlier");
    if (!ctx->dd) FAIL(HDD_ERR_STATE, "hdd_setup_dd first");
    if (nrhs < 1 || nrhs > 4096) FAIL(HDD_ERR_INVALID_ARG, "nrhs must be in 1..4096");
    CK(cudaSetDevice(ctx->device));
    return build_tasks(ctx, nrhs);
}

int hdd_num_rhs(const hdd_ctx *ctx) { return ctx && ctx->dd ? ctx->nrhs : 0; }

hdd_status hdd_profile(hdd_ctx *ctx, int enable) {
    if (!ctx) return HDD_ERR_INVALID_ARG;
    if (ctx->poisoned) FAIL(HDD_ERR_TIMEOUT, "context lost: a device wait and its drain timed out earlier");
    CK(cudaSetDevice(ctx->device));
    CK(cudaDeviceSynchronize());
    ctx->prof.harvest();
    ctx->prof.reset();
    ctx->prof.on = enable != 0;
    return HDD_OK;
}

int hdd_profile_count(const hdd_ctx *ctx) { return ctx ? (int)NFAM : 0; }

hdd_status hdd_profile_get(hdd_ctx *ctx, int i, hdd_kernel_stat *out) {
    if (!ctx) return HDD_ERR_INVALID_ARG;
    if (ctx->poisoned) FAIL(HDD_ERR_TIMEOUT, "context lost: a device wait and its drain timed out earlier");
    if (i < 0 || i >= NFAM || !out) FAIL(HDD_ERR_INVALID_ARG, "bad profile index");
    CK(cudaSetDevice(ctx->device));
    CK(cudaDeviceSynchronize());
    ctx->prof.harvest();
    std::memset(out, 0, sizeof(*out));
    std::snprintf(out->name, sizeof(out->name), "%s", kFamName[i]);
    out->launches = ctx->prof.cnt[i];
    out->ms = ctx->prof.ms[i];
    out->bytes = ctx->prof.bytes[i];
    out->flops = ctx->prof.flops[i];
    out->bound = kFamBound[i];
    return HDD_OK;
}

long long hdd_launch_count(const hdd_ctx *ctx) { return ctx ? ctx->prof.launches : 0; }

int hdd_cnn_num_params(void) { return CNN_NPARAM; }

hdd_status hdd_cnn_set_params(hdd_ctx *ctx, const float *params) {
    if (!ctx) return HDD_ERR_INVALID_ARG;
    if (ctx->poisoned) FAIL(HDD_ERR_TIMEOUT, "context lost: a device wait and its drain timed out earlier");
    if (!ctx->dd) FAIL(HDD_ERR_STATE, "hdd_setup_dd first");
    if (ctx->bc) FAIL(HDD_ERR_INVALID_ARG, "the learned warm start serves the Dirichlet problem only");
    if (!params) FAIL(HDD_ERR_INVALID_ARG, "params is NULL");
    for (int i = 0; i < CNN_NPARAM; i++)
        if (!std::isfinite(params[i])) FAIL(HDD_ERR_NONFINITE, "parameter %d is not finite", i);
    CK(cudaSetDevice(ctx->device));
    hdd_status st = cnn_buffers(ctx);
    if (st != HDD_OK) return st;
    CnnState &C = ctx->cnn;
    CK(cudaMemcpy(C.P.p, params, CNN_NPARAM * sizeof(float), cudaMemcpyHostToDevice));
    CK(cudaMemset(C.M.p, 0, CNN_NPARAM * sizeof(float)));
    CK(cudaMemset(C.Vm.p, 0, CNN_NPARAM * sizeof(float)));
    launch_to_bf16(CNN_NPARAM, C.P.as<float>(), C.Pb.as<__nv_bfloat16>(), 0);
    C.tc_dirty = true;
    CKL();
    CK(cudaDeviceSynchronize());
    C.step = 0;
    C.ready = true;
    return HDD_OK;
}

hdd_status hdd_warmstart_load(hdd_ctx *ctx, const char *path) {
    if (!ctx) return HDD_ERR_INVALID_ARG;
    if (ctx->poisoned) FAIL(HDD_ERR_TIMEOUT, "context lost: a device wait and its drain timed out earlier");
    if (!path) FAIL(HDD_ERR_INVALID_ARG, "path is NULL");
    FILE *fh = std::fopen(path, "rb");
    if (!fh) FAIL(HDD_ERR_INVALID_ARG, "cannot open %s", path);
    std::vector<unsigned char> buf;
    unsigned char tmp[65536];
    size_t got;
    while ((got = std::fread(tmp, 1, sizeof(tmp), fh)) > 0) buf.insert(buf.end(), tmp, tmp + got);
    const bool rerr = std::ferror(fh) != 0;
    std::fclose(fh);
    if (rerr) FAIL(HDD_ERR_INVALID_ARG, "cannot read %s", path);
    if (buf.size() < 16 || std::memcmp(buf.data(), kWsMagic, 8) != 0)
        FAIL(HDD_ERR_INVALID_ARG, "%s is not a warm-start parameter file", path);
    const uint32_t n = rd_le32(buf.data() + 8), crc = rd_le32(buf.data() + 12);
    if (n != (uint32_t)CNN_NPARAM || buf.size() != 16 + 4 * (size_t)n)
        FAIL(HDD_ERR_INVALID_ARG, "%s holds %u parameters, the network has %d", path, n, CNN_NPARAM);
    if (crc32_ieee(buf.data() + 16, 4 * (size_t)n) != crc) FAIL(HDD_ERR_INVALID_ARG, "%s is corrupt (CRC-32)", path);
    std::vector<float> prm(n);
    for (uint32_t i = 0; i < n; i++) {
        const uint32_t b = rd_le32(buf.data() + 16 + 4 * (size_t)i);
        std::memcpy(&prm[i], &b, 4);
    }
    return hdd_cnn_set_params(ctx, prm.data());
}

hdd_status hdd_warmstart_save(hdd_ctx *ctx, const char *path) {
    if (!ctx) return HDD_ERR_INVALID_ARG;
    if (ctx->poisoned) FAIL(HDD_ERR_TIMEOUT, "context lost: a device wait and its drain timed out earlier");
    if (!path) FAIL(HDD_ERR_INVALID_ARG, "path is NULL");
    std::vector<float> prm(CNN_NPARAM);
    hdd_status st = hdd_cnn_get_params(ctx, prm.data());
    if (st != HDD_OK) return st;
    std::vector<unsigned char> buf(16 + 4 * (size_t)CNN_NPARAM);
    std::memcpy(buf.data(), kWsMagic, 8);
    for (int i = 0; i < CNN_NPARAM; i++) {
        uint32_t b;
        std::memcpy(&b, &prm[i], 4);
        wr_le32(buf.data() + 16 + 4 * (size_t)i, b);
    }
    wr_le32(buf.data() + 8, (uint32_t)CNN_NPARAM);
    wr_le32(buf.data() + 12, crc32_ieee(buf.data() + 16, 4 * (size_t)CNN_NPARAM));
    FILE *fh = std::fopen(path, "wb");
    if (!fh) FAIL(HDD_ERR_INVALID_ARG, "cannot create %s", path);
    const bool ok = std::fwrite(buf.data(), 1, buf.size(), fh) == buf.size();
    if (std::fclose(fh) != 0 || !ok) FAIL(HDD_ERR_INVALID_ARG, "cannot write %s", path);
    return HDD_OK;
}

hdd_status hdd_cnn_get_params(hdd_ctx *ctx, float *params) {
    if (!ctx) return HDD_ERR_INVALID_ARG;
    if (ctx->poisoned) FAIL(HDD_ERR_TIMEOUT, "context lost: a device wait and its drain timed out earlier");
    if (!ctx->cnn.ready) FAIL(HDD_ERR_STATE, "hdd_cnn_set_params first");
    if (!params) FAIL(HDD_ERR_INVALID_ARG, "params is NULL");
    CK(cudaSetDevice(ctx->device));
    CK(cudaMemcpy(params, ctx->cnn.P.p, CNN_NPARAM * sizeof(float), cudaMemcpyDeviceToHost));
    return HDD_OK;
}

hdd_status hdd_cnn_forward(hdd_ctx *ctx, const void *f_dev, void *x0_dev, void *stream) {
    if (!ctx) return HDD_ERR_INVALID_ARG;
    if (ctx->poisoned) FAIL(HDD_ERR_TIMEOUT, "context lost: a device wait and its drain timed out earlier");
    if (!ctx->cnn.ready) FAIL(HDD_ERR_STATE, "hdd_cnn_set_params first");
    if (!f_dev || !x0_dev || f_dev == x0_dev || !aligned16(f_dev) || !aligned16(x0_dev))
        FAIL(HDD_ERR_INVALID_ARG, "bad vector arguments");
    CK(cudaSetDevice(ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    hdd_status st = cnn_buffers(ctx);
    if (st != HDD_OK) return st;
    cnn_forward<double>(ctx, (const double2 *)f_dev, s);
    KL(F_CNN, 0, 0, launch_cnn_output<double>(ctx->d_tasks.as<Task>(), ctx->d_ftiles.as<Tile>(),
                                                (int)ctx->h_ftiles.size(), ctx->cnn.sigma.as<float>(),
                                                ctx->cnn.A4.as<float>(), (double2 *)x0_dev, nullptr, s));
    CKL();
    return HDD_OK;
}

hdd_status hdd_cnn_infer(hdd_ctx *ctx, const void *f_dev, void *x0_dev, void *stream) {
    if (!ctx) return HDD_ERR_INVALID_ARG;
    if (ctx->poisoned) FAIL(HDD_ERR_TIMEOUT, "context lost: a device wait and its drain timed out earlier");
    if (!ctx->cnn.ready) FAIL(HDD_ERR_STATE, "hdd_cnn_set_params first");
    if (!f_dev || !x0_dev || f_dev == x0_dev || !aligned16(f_dev) || !aligned16(x0_dev))
        FAIL(HDD_ERR_INVALID_ARG, "bad vector arguments");
    CK(cudaSetDevice(ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    hdd_status st = cnn_buffers(ctx);
    if (st != HDD_OK) return st;
    if ((st = cnn_infer<double>(ctx, (const double2 *)f_dev, s)) != HDD_OK) return st;
    KL(F_CNN, 0, 0, launch_cnn_output<double>(ctx->d_tasks.as<Task>(), ctx->d_ftiles.as<Tile>(),
                                                (int)ctx->h_ftiles.size(), ctx->cnn.sigma.as<float>(),
                                                ctx->cnn.A4.as<float>(), (double2 *)x0_dev, nullptr, s));
    CKL();
    return cnn_check_err(ctx, s);
}

hdd_status hdd_cnn_loss_grad(hdd_ctx *ctx, const void *f_dev, double *loss, float *grad) {
    if (!ctx) return HDD_ERR_INVALID_ARG;
    if (ctx->poisoned) FAIL(HDD_ERR_TIMEOUT, "context lost: a device wait and its drain timed out earlier");
    if (!ctx->cnn.ready) FAIL(HDD_ERR_STATE, "hdd_cnn_set_params first");
    if (!f_dev || !aligned16(f_dev)) FAIL(HDD_ERR_INVALID_ARG, "bad vector argument");
    CK(cudaSetDevice(ctx->device));
    cudaStream_t s = 0;
    hdd_status st = cnn_loss_grad<double>(ctx, (const double2 *)f_dev, loss, s);
    if (st != HDD_OK) return st;
    if (grad) CK(cudaMemcpy(grad, ctx->cnn.G.p, CNN_NPARAM * sizeof(float), cudaMemcpyDeviceToHost));
    return HDD_OK;
}

hdd_status hdd_cnn_train_step(hdd_ctx *ctx, const void *f_dev, float lr, double *loss, void *stream) {
    if (!ctx) return HDD_ERR_INVALID_ARG;
    if (ctx->poisoned) FAIL(HDD_ERR_TIMEOUT, "context lost: a device wait and its drain timed out earlier");
    if (!ctx->cnn.ready) FAIL(HDD_ERR_STATE, "hdd_cnn_set_params first");
    if (!f_dev || !aligned16(f_dev) || !(lr > 0)) FAIL(HDD_ERR_INVALID_ARG, "bad arguments");
    CK(cudaSetDevice(ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    hdd_status st = cnn_loss_grad<double>(ctx, (const double2 *)f_dev, loss, s);
    if (st != HDD_OK) return st;
    CnnState &C = ctx->cnn;
    C.step++;
    C.tc_dirty = true;
    KL(F_CNN, 0, 0, launch_adam(CNN_NPARAM, C.P.as<float>(), C.G.as<float>(), C.M.as<float>(), C.Vm.as<float>(),
                                  C.Pb.as<__nv_bfloat16>(), lr, 0.9f, 0.999f, 1e-8f, C.step, s));
    CKL();
    return HDD_OK;
}

hdd_status hdd_get_outer_vector(hdd_ctx *ctx, int j, void *v_dev, void *stream) {
    if (!ctx) return HDD_ERR_INVALID_ARG;
    if (ctx->poisoned) FAIL(HDD_ERR_TIMEOUT, "context lost: a device wait and its drain timed out earlier");
    if (!ctx->ow.V.p) FAIL(HDD_ERR_STATE, "no solve has run");
    if (j < 0 || !v_dev || !aligned16(v_dev)) FAIL(HDD_ERR_INVALID_ARG, "bad arguments");
    const size_t bytes = (size_t)ctx->nrhs * ctx->nglob * sizeof(double2);
    if ((size_t)(j + 1) * bytes > ctx->ow.V.bytes) FAIL(HDD_ERR_INVALID_ARG, "basis vector %d not stored", j);
    CK(cudaSetDevice(ctx->device));
    CK(cudaMemcpyAsync(v_dev, ctx->ow.V.as<char>() + (size_t)j * bytes, bytes, cudaMemcpyDeviceToDevice,
                       (cudaStream_t)stream));
    return HDD_OK;
}

hdd_status hdd_set_option(hdd_ctx *ctx, int key, int value) {
    if (!ctx) return HDD_ERR_INVALID_ARG;
    if (value != 0 && value != 1) FAIL(HDD_ERR_INVALID_ARG, "option values are 0 or 1");
    if (key == HDD_OPT_COARSE_LOOKAHEAD) ctx->coarse_la = value;
    else if (key == HDD_OPT_FUSED_INNER) ctx->fused_inner = value;
    else if (key == HDD_OPT_OUTER_DOTS_DF) ctx->outer_df = value;
    else if (key == HDD_OPT_OUTER_UPDATE_DF) ctx->outer_udf = value;
    else if (key == HDD_OPT_OUTER_DCGS2) ctx->outer_dcgs = value;
    else if (key == HDD_OPT_COARSE_DF) ctx->coarse_df = value;
    else if (key == HDD_OPT_COARSE_SPIKE) ctx->coarse_spike = value;
    else if (key == HDD_OPT_OUTER_DOTS_BIASED) ctx->outer_bias = value;
    else FAIL(HDD_ERR_INVALID_ARG, "unknown option %d", key);
    return HDD_OK;
}

hdd_status hdd_apply_PA_noalloc(hdd_ctx *ctx, const void *in_dev, void *out_dev, void *stream) {
    if (!ctx) return HDD_ERR_INVALID_ARG;
    if (ctx->poisoned) FAIL(HDD_ERR_TIMEOUT, "context lost: a device wait and its drain timed out earlier");
    if (!ctx->dd) FAIL(HDD_ERR_STATE, "hdd_setup_dd first");
    if (!ctx->E.ready) FAIL(HDD_ERR_STATE, "hdd_setup_deflation first");
    if (!in_dev || !out_dev || in_dev == out_dev || !aligned16(in_dev) || !aligned16(out_dev))
        FAIL(HDD_ERR_INVALID_ARG, "bad vector arguments");
    if (ctx->ldc > HDD_NOALLOC_MAX_COARSE)
        FAIL(HDD_ERR_INVALID_ARG, "packed coarse length %lld exceeds the no-allocation limit %d",
             ctx->ldc, HDD_NOALLOC_MAX_COARSE);
    CK(cudaSetDevice(ctx->device));
    double2 *scratch = nullptr;
    CK(noalloc_scratch(ctx->device, &scratch));
    cudaStream_t s = (cudaStream_t)stream;
    LocalArgs<double> a = local_args<double>(ctx);
    const size_t smem = local_max_dynamic_smem(ctx->max_nx, (int)sizeof(double2), ctx->frows, ctx->crows);
    if (smem > 48 * 1024) CK(set_local_smem_limits<double>(smem));
    double2 *y = scratch, *sc = scratch + HDD_NOALLOC_MAX_COARSE;
    const double2 *in = (const double2 *)in_dev;
    double2 *out = (double2 *)out_dev;
    const FactorSet &F = ctx->E;
    // every coarse entry of y and s is written before it is read: nothing needs clearing
    launch_zt<double>(a, in, y, 1, nullptr, s);                                        // y = Zᵀ A v
    launch_block_solve(ctx->d_tasks.as<Task>(), (int)ctx->h_tasks.size(), F.table.as<BlockFactor>(),
                       F.M.as<double>(), F.P.as<int>(), F.Meta.as<int4>(), y, sc, 0, nullptr,
                       F.cfg, F.re2 ? 1 : 0, s);                                        // s = E⁻¹ y
    launch_prolong_stencil<double>(a, 0, in, sc, out, nullptr, 0, scratch, nullptr, s); // A(v - Z s)
    ctx->prof.launches += 3;
    CKL();
    return HDD_OK;
}

hdd_status hdd_local_op(hdd_ctx *ctx, int op, int prec, const void *in_dev, void *out_dev, void *stream) {
    if (!ctx) return HDD_ERR_INVALID_ARG;
    if (ctx->poisoned) FAIL(HDD_ERR_TIMEOUT, "context lost: a device wait and its drain timed out earlier");
    if (!ctx->dd) FAIL(HDD_ERR_STATE, "hdd_setup_dd first");
    if (op < 0 || op > 6 || (prec != 64 && prec != 128) || !in_dev || !out_dev || in_dev == out_dev ||
        !aligned16(in_dev) || !aligned16(out_dev))
        FAIL(HDD_ERR_INVALID_ARG, "bad local_op arguments");
    if ((op == 3 || op == 4) && !ctx->E.ready) FAIL(HDD_ERR_STATE, "hdd_setup_deflation first");
    if (op == 6 && !ctx->Aex.ready) FAIL(HDD_ERR_STATE, "hdd_setup_exact first");
    CK(cudaSetDevice(ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    const long long ld = ctx->ld, ldc = ctx->ldc;
    const double2 *in = (const double2 *)in_dev;
    double2 *out = (double2 *)out_dev;
    if (op == 3) {
        band_solve(ctx, ctx->E, in, out, false, nullptr, s, -1, prec == 64);
        CKL(); CK(cudaStreamSynchronize(s)); return HDD_OK;
    }
    if (op == 6) {
        band_solve(ctx, ctx->Aex, in, out, true, nullptr, s, -1, prec == 64);
        CKL(); CK(cudaStreamSynchronize(s)); return HDD_OK;
    }
    auto run = [&](auto tag) -> hdd_status {
        using R = decltype(tag);
        LocalArgs<R> a = local_args<R>(ctx);
        size_t smem = local_max_dynamic_smem(ctx->max_nx, (int)sizeof(c2<R>), ctx->frows, ctx->crows);
        if (smem > 48 * 1024) CK(set_local_smem_limits<R>(smem));
        CK(ctx->tmp_a.ensure(std::max(ld, ldc) * sizeof(c2<R>)));
        CK(ctx->tmp_b.ensure(std::max(ld, ldc) * sizeof(c2<R>)));
        CK(ctx->tmp_c.ensure((std::max(ld, ldc) + 64) * sizeof(double2)));
        c2<R> *ta = ctx->tmp_a.as<c2<R>>(), *tb = ctx->tmp_b.as<c2<R>>();
        const int is_d = sizeof(R) == 8;
        switch (op) {
            case 0:
                launch_cast(ld, in, 1, ta, is_d, s);
                launch_local_A<R>(a, ta, tb, nullptr, nullptr, s);
                launch_cast(ld, tb, is_d, out, 1, s);
                break;
            case 1:
                launch_z<R>(a, in, nullptr, tb, nullptr, s);
                launch_cast(ld, tb, is_d, out, 1, s);
                break;
            case 2:
                launch_cast(ld, in, 1, ta, is_d, s);
                launch_zt<R>(a, ta, out, 0, nullptr, s);
                break;
            case 4: {                                   // P A v = A (v - Z E⁻¹ Zᵀ A v)
                double2 *y = ctx->tmp_c.as<double2>();      // ld + 64 >= 2·ldc + 32 entries
                double2 *s2 = y + ldc + 32;
                launch_cast(ld, in, 1, ta, is_d, s);
                launch_zt<R>(a, ta, y, 1, nullptr, s);
                band_solve(ctx, ctx->E, y, s2, false, nullptr, s);
                launch_prolong_stencil<R>(a, 0, ta, s2, tb, nullptr, 0, ta /*unused: nv = 0*/, nullptr, s);
                launch_cast(ld, tb, is_d, out, 1, s);
                break;
            }
            case 5:
                launch_restrict<R>(a, in, ctx->nglob, tb, nullptr, s);
                launch_cast(ld, tb, is_d, out, 1, s);
                break;
        }
        CKL();
        CK(cudaStreamSynchronize(s));
        return HDD_OK;
    };
    return prec == 64 ? run(float{}) : run(double{});
}

}  // extern "C"
