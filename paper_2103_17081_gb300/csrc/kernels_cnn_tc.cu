// kernels_cnn_tc.cu — inference of the warm-start network on the 5th-generation tensor cores.
//
// Activations between layers are BF16 in a padded planar layout: task t's nx x ny image sits in
// a (ny+2) x (nx+2) frame whose border positions are zero; frame position q = (y+1)(nx+2)+(x+1)
// holds channels 8c..8c+7 of pixel (x, y) as 16 bytes at uint4 index c·ptot + poff_t + q
// (4 planes of 8 channels, ptot positions per plane over all tasks).
//
// A 3x3 convolution with 32 input channels is then a GEMM per tile of 128 consecutive frame
// positions: D[i][co] = Σ_tap Σ_ci X[q0 + i + s_tap][ci] W[co][tap][ci], s_tap = dy·(nx+2) + dx.
// The 128 x 16 operand block of one tap and 16 input channels is the window of the staged planes
// that starts s_tap positions later: rows are 16-byte position records (stride 16 B, 8-row core
// matrices 128 B apart) and the two 8-channel halves one plane apart, which is a K-major,
// unswizzled shared-memory operand for tcgen05.mma at any start position.  So the tile's input
// window (128 + 2(nx+3) positions of each plane, fetched with four 1D bulk copies) is staged once
// and the 18 MMAs (9 taps x 2 halves of K = 32) read it in place: no im2col copy.  The zero frame
// border supplies the zero padding; outputs at border positions are discarded.
#include "hdd_common.cuh"
#include "umma.cuh"

#include <cuda_bf16.h>

namespace hdd {

constexpr int TCM = 128;                  // output positions per tile (MMA M)
constexpr int TC_THREADS = 128;           // 4 warps: TMEM lanes 32w..32w+31 each
constexpr int TC_WAIT = 1 << 22;          // mbarrier polls before a wait gives up

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
    __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&v);
}

// Layer 1 (4 → 32, ReLU) on the CUDA cores from the FP32 input image X0 (float4 per pixel, packed
// layout), written as BF16 to the padded planar buffer X1.  One pixel per thread step.
__global__ void __launch_bounds__(256)
k_cnn_l1_bf16(const Task *__restrict__ tasks, const Tile *__restrict__ tiles,
              const __nv_bfloat16 *__restrict__ Wb, const float *__restrict__ bias,
              const float *__restrict__ X0, uint4 *__restrict__ X1, long long ptot) {
    __shared__ float Ws[32 * 9 * 4];
    __shared__ float Bs[32];
    for (int i = threadIdx.x; i < 32 * 9 * 4; i += blockDim.x) Ws[i] = __bfloat162float(Wb[i]);
    for (int i = threadIdx.x; i < 32; i += blockDim.x) Bs[i] = bias[i];
    __syncthreads();
    const Tile tl = tiles[blockIdx.x];
    const Task T = tasks[tl.task];
    const int nx = T.nx, ny = T.ny, nxp = nx + 2;
    for (int e = threadIdx.x; e < tl.nr * nx; e += blockDim.x) {
        const int y = tl.r0 + e / nx, x = e % nx;
        float acc[32];
#pragma unroll
        for (int c = 0; c < 32; c++) acc[c] = Bs[c];
#pragma unroll
        for (int k = 0; k < 9; k++) {
            const int yy = y + k / 3 - 1, xx = x + k % 3 - 1;
            if (yy < 0 || yy >= ny || xx < 0 || xx >= nx) continue;
            const float4 v = reinterpret_cast<const float4 *>(X0)[T.foff + (long long)yy * nx + xx];
#pragma unroll
            for (int co = 0; co < 32; co++) {
                const float *w = Ws + (co * 9 + k) * 4;
                acc[co] = fmaf(w[0], v.x, fmaf(w[1], v.y, fmaf(w[2], v.z, fmaf(w[3], v.w, acc[co]))));
            }
        }
        const long long q = T.poff + (long long)(y + 1) * nxp + (x + 1);
#pragma unroll
        for (int c = 0; c < 4; c++) {
            uint4 o;
            o.x = pack_bf16x2(fmaxf(acc[8 * c + 0], 0.f), fmaxf(acc[8 * c + 1], 0.f));
            o.y = pack_bf16x2(fmaxf(acc[8 * c + 2], 0.f), fmaxf(acc[8 * c + 3], 0.f));
            o.z = pack_bf16x2(fmaxf(acc[8 * c + 4], 0.f), fmaxf(acc[8 * c + 5], 0.f));
            o.w = pack_bf16x2(fmaxf(acc[8 * c + 6], 0.f), fmaxf(acc[8 * c + 7], 0.f));
            X1[c * ptot + q] = o;
        }
    }
}

// Weight images of the three 32-input layers in the B-operand layout of the MMA: for tap k and
// 8-channel input chunk c, rows co = 0..NCO-1 of 16 bytes (W[co][k][8c..8c+7]), i.e. element
// ((k·4 + c)·NCO + co)·8 + e.  NCO = 32 for layers 2, 3; 16 for layer 4 (rows 2..15 zero).
__global__ void k_cnn_tc_weights(const __nv_bfloat16 *__restrict__ W2, const __nv_bfloat16 *__restrict__ W3,
                                 const __nv_bfloat16 *__restrict__ W4, __nv_bfloat16 *__restrict__ img2,
                                 __nv_bfloat16 *__restrict__ img3, __nv_bfloat16 *__restrict__ img4) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int n32 = 9 * 4 * 32 * 8, n16 = 9 * 4 * 16 * 8;
    if (i < 2 * n32) {
        const int l = i / n32, j = i % n32;             // l = 0: layer 2, 1: layer 3
        const int e = j % 8, co = (j / 8) % 32, c = (j / 256) % 4, k = j / 1024;
        (l == 0 ? img2 : img3)[j] = (l == 0 ? W2 : W3)[(co * 9 + k) * 32 + 8 * c + e];
    } else if (i < 2 * n32 + n16) {
        const int j = i - 2 * n32;
        const int e = j % 8, co = (j / 8) % 16, c = (j / 128) % 4, k = j / 512;
        img4[j] = co < 2 ? W4[(co * 9 + k) * 32 + 8 * c + e] : __float2bfloat16(0.f);
    }
}

// One 32-input 3x3 convolution layer on the tensor cores (see the file comment).  Persistent:
// CTA b handles tiles b, b + gridDim.x, ...; tile = (task, q0), 128 frame positions from q0.
// NCO = 32: bias + ReLU, BF16 to the padded planar Y.  NCO = 16 (last layer): output channels
// 0, 1 + bias in FP32 to A4 (packed layout, float2 per pixel).  Every mbarrier wait is bounded;
// on a timeout the CTA sets *err, waits (bounded) for its copies and MMAs, frees TMEM, returns.
template <int NCO>
__global__ void __launch_bounds__(TC_THREADS)
k_conv_tc(const Task *__restrict__ tasks, const int2 *__restrict__ tct, int ntct, const uint4 *__restrict__ X,
          long long ptot, const uint4 *__restrict__ Wimg, const float *__restrict__ bias, uint4 *__restrict__ Y,
          float2 *__restrict__ A4, int wmax, int *__restrict__ err) {
    extern __shared__ __align__(128) uint8_t sm[];
    __shared__ uint64_t bar_ld, bar_mma;
    __shared__ uint32_t tbase;
    __shared__ float bs[32];
    constexpr uint32_t WB = 9 * 4 * NCO * 16;           // weight image bytes
    uint8_t *sB = sm, *sA = sm + WB;
    const uint32_t plane = (uint32_t)wmax * 16;         // bytes per staged plane
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 0) umma::tmem_alloc(&tbase, 32);
    if (threadIdx.x == 0) { umma::mbar_init(&bar_ld, 1); umma::mbar_init(&bar_mma, 1); }
    if (threadIdx.x < 32) bs[threadIdx.x] = threadIdx.x < (NCO == 32 ? 32 : 2) ? bias[threadIdx.x] : 0.f;
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t td = tbase;
    // phase bookkeeping (uniform over the CTA): parity of the next phase of each barrier and
    // whether copies / MMAs of that phase were issued and not yet seen complete
    uint32_t ldpar = 0, mmapar = 0;
    bool ld_pending = true, mma_pending = false;
    if (threadIdx.x == 0) {
        umma::mbar_expect_tx(&bar_ld, WB);
        umma::bulk_g2s(sB, Wimg, WB, &bar_ld);
    }
    bool ok = __syncthreads_and(umma::mbar_wait(&bar_ld, ldpar, TC_WAIT));
    if (ok) { ld_pending = false; ldpar ^= 1u; }
    constexpr uint32_t idesc = umma::idesc_bf16_f32(TCM, NCO);
    for (int tix = blockIdx.x; ok && tix < ntct; tix += gridDim.x) {
        const int2 tc = tct[tix];
        const Task T = tasks[tc.x];
        const int nxp = T.nx + 2;
        const long long P = (long long)(T.ny + 2) * nxp;
        const long long lo = (long long)tc.y - nxp - 1, hi = lo + TCM + 2 * nxp + 2;
        const long long a = lo < 0 ? 0 : lo, b = hi > P ? P : hi;
        // clipped window ends (outside the frame; read only for discarded outputs): zeros
        for (int c = 0; c < 4; c++) {
            uint4 *pl = reinterpret_cast<uint4 *>(sA + c * plane);
            for (long long q = lo + threadIdx.x; q < a; q += blockDim.x) pl[q - lo] = make_uint4(0, 0, 0, 0);
            for (long long q = b + threadIdx.x; q < hi; q += blockDim.x) pl[q - lo] = make_uint4(0, 0, 0, 0);
        }
        umma::fence_async_smem();
        if (threadIdx.x == 0) {
            const uint32_t bytes = (uint32_t)(b - a) * 16;
            umma::mbar_expect_tx(&bar_ld, 4 * bytes);
            for (int c = 0; c < 4; c++)
                umma::bulk_g2s(sA + c * plane + (a - lo) * 16, X + c * ptot + T.poff + a, bytes, &bar_ld);
        }
        ld_pending = true;
        ok = __syncthreads_and(umma::mbar_wait(&bar_ld, ldpar, TC_WAIT));
        if (!ok) break;
        ld_pending = false;
        ldpar ^= 1u;
        if (threadIdx.x == 0) {
            umma::fence_after_sync();
#pragma unroll
            for (int k = 0; k < 9; k++) {
                const uint32_t off = (uint32_t)((k / 3) * nxp + (k % 3)) * 16;
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    const uint64_t ad = umma::desc_kmajor(umma::smem_u32(sA + 2 * h * plane + off), plane, 128);
                    const uint64_t bd = umma::desc_kmajor(umma::smem_u32(sB + (k * 4 + 2 * h) * NCO * 16), NCO * 16, 128);
                    umma::mma_bf16(td, ad, bd, idesc, (k | h) != 0);
                }
            }
            umma::commit(&bar_mma);
        }
        mma_pending = true;
        ok = __syncthreads_and(umma::mbar_wait(&bar_mma, mmapar, TC_WAIT));
        if (!ok) break;
        mma_pending = false;
        mmapar ^= 1u;
        umma::fence_after_sync();
        const long long q = (long long)tc.y + 32 * warp + lane;
        const int py = (int)(q / nxp), px = (int)(q - (long long)py * nxp);
        const bool valid = py >= 1 && py <= T.ny && px >= 1 && px <= T.nx;
        const uint32_t ta = td + ((uint32_t)(32 * warp) << 16);
        if constexpr (NCO == 32) {
            float v[32];
            umma::tmem_ld32(ta, v);
            if (valid) {
#pragma unroll
                for (int c = 0; c < 4; c++) {
                    uint4 o;
                    o.x = pack_bf16x2(fmaxf(v[8 * c + 0] + bs[8 * c + 0], 0.f), fmaxf(v[8 * c + 1] + bs[8 * c + 1], 0.f));
                    o.y = pack_bf16x2(fmaxf(v[8 * c + 2] + bs[8 * c + 2], 0.f), fmaxf(v[8 * c + 3] + bs[8 * c + 3], 0.f));
                    o.z = pack_bf16x2(fmaxf(v[8 * c + 4] + bs[8 * c + 4], 0.f), fmaxf(v[8 * c + 5] + bs[8 * c + 5], 0.f));
                    o.w = pack_bf16x2(fmaxf(v[8 * c + 6] + bs[8 * c + 6], 0.f), fmaxf(v[8 * c + 7] + bs[8 * c + 7], 0.f));
                    Y[c * ptot + T.poff + q] = o;
                }
            }
        } else {
            float v0, v1;
            umma::tmem_ld2(ta, v0, v1);
            if (valid) A4[T.foff + (long long)(py - 1) * T.nx + (px - 1)] = make_float2(v0 + bs[0], v1 + bs[1]);
        }
        umma::fence_before_sync();
        __syncthreads();            // TMEM read and window consumed before the next tile reuses them
    }
    if (!ok) {
        // drain: copies and a committed MMA not yet seen complete, each with a bounded wait.
        // Flag 1: a wait gave up and the drain then saw everything in flight complete (the
        // context stays usable).  Flag 2: the drain gave up as well, so a bulk copy or an MMA may
        // still be writing this CTA's shared memory or TMEM after the CTA frees them and exits;
        // nothing bounds what that write reaches, so the host treats flag 2 as fatal for the CUDA
        // context (the library refuses further work on it, the caller must discard the context).
        bool drained = true;
        if (ld_pending) drained &= umma::mbar_wait(&bar_ld, ldpar, TC_WAIT);
        if (mma_pending) drained &= umma::mbar_wait(&bar_mma, mmapar, TC_WAIT);
        drained = __syncthreads_and(drained);
        if (threadIdx.x == 0) atomicMax(err, drained ? 1 : 2);
    }
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    if (warp == 0) umma::tmem_dealloc(td, 32);
}

size_t conv_tc_smem(int nco, int wmax) { return (size_t)9 * 4 * nco * 16 + (size_t)4 * wmax * 16; }

void launch_cnn_l1_bf16(const Task *tasks, const Tile *tiles, int ntiles, const __nv_bfloat16 *W, const float *b,
                        const float *X0, uint4 *X1, long long ptot, cudaStream_t s) {
    k_cnn_l1_bf16<<<ntiles, 256, 0, s>>>(tasks, tiles, W, b, X0, X1, ptot);
}

void launch_cnn_tc_weights(const __nv_bfloat16 *Wb, __nv_bfloat16 *img2, __nv_bfloat16 *img3,
                           __nv_bfloat16 *img4, cudaStream_t s) {
    const int n = 2 * 9 * 4 * 32 * 8 + 9 * 4 * 16 * 8;
    k_cnn_tc_weights<<<(n + 255) / 256, 256, 0, s>>>(Wb + CNN_OFF[1], Wb + CNN_OFF[2], Wb + CNN_OFF[3], img2, img3,
                                                     img4);
}

cudaError_t set_conv_tc_smem(int wmax) {
    cudaError_t e = cudaFuncSetAttribute(k_conv_tc<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)conv_tc_smem(32, wmax));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_conv_tc<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)conv_tc_smem(16, wmax));
}

void launch_conv_tc(int nco, int grid, const Task *tasks, const int2 *tct, int ntct, const uint4 *X, long long ptot,
                    const uint4 *Wimg, const float *bias, uint4 *Y, float2 *A4, int wmax, int *err, cudaStream_t s) {
    if (nco == 32)
        k_conv_tc<32><<<grid, TC_THREADS, conv_tc_smem(32, wmax), s>>>(tasks, tct, ntct, X, ptot, Wimg, bias, Y, A4,
                                                                        wmax, err);
    else
        k_conv_tc<16><<<grid, TC_THREADS, conv_tc_smem(16, wmax), s>>>(tasks, tct, ntct, X, ptot, Wimg, bias, Y, A4,
                                                                        wmax, err);
}

}  // namespace hdd
