// The proposal network's 3 x 3 circular convolutions as implicit GEMMs on the
// sm_103a tensor cores (tcgen05.mma, accumulators in TMEM).
//
//   forward      Y[b][o][s] = bias[o] + sum_{t, c} W[o][c][t] X[b][c][nb_t(s)]
//                D[s][o] (M = pixels, N = output channels, K = taps x input
//                channels), BF16 operands (kind::f16), FP32 accumulation;
//   input grad   dX[b][c][s] = [act > 0] sum_{t, o} W[o][c][t] dY[b][o][nb'_t(s)]
//                D[s][c] (K = taps x output channels), TF32 operands
//                (kind::tf32: dY is FP32, rounded to TF32 once);
//   weight grad  dW[o][c][t] = sum_{b, s} X[b][c][nb_t(s)] dY[b][o][s]
//                D[(t, c)][o] (K = pixels of the CTA's samples), TF32,
//                partial sums of the CTAs added atomically.
// nb_t(s) is pixel s shifted by tap t = 3 ky + kx, (ky - 1, kx - 1), on the
// torus; nb'_t(s) the opposite shift (the output pixel whose tap t read s).
//
// One CTA of 256 threads: every thread builds one row of the im2col operand
// tile per K step (the gather from global memory, which stays in L2), one
// thread issues the MMAs, and two operand buffers alternate so the gather of
// step k + 1 overlaps the MMAs of step k.  Mbarrier waits are bounded; on
// expiry the CTA stops, raises the network's error word and frees its TMEM.
#include <cuda_bf16.h>
#include "ggf_ctx.h"
#include "ggf_tc.cuh"

namespace {

typedef __nv_bfloat16 bf16;
constexpr int CT = 256;                 // threads per CTA = im2col rows built per K step

__device__ __forceinline__ unsigned char* align1k(unsigned char* p) {
    return (unsigned char*)(((uintptr_t)p + 1023) & ~(uintptr_t)1023);
}

__device__ __forceinline__ int shifted(int L, int s, int t, int sign) {
    const int x = s % L, y = s / L, ky = t / 3 - 1, kx = t % 3 - 1;
    return ((y + sign * ky + L) % L) * L + (x + sign * kx + L) % L;
}

// TMEM allocation by one whole warp; the column address lands in *slot
__device__ __forceinline__ void tmem_alloc_warp(uint32_t* slot, int ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::smem_u32(slot)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}

// Operand-buffer bookkeeping shared by the three kernels: before a buffer is
// rewritten, the MMAs that read it (one commit) must have completed.  Every
// thread tracks the same state and takes the same waits; the outcome is
// agreed with __syncthreads_or so that no thread leaves a loop alone.
struct Bufs {
    uint32_t bar[2];
    uint32_t phase[2] = {0u, 0u};
    bool pending[2] = {false, false};
    __device__ bool wait(int b) {
        bool ok = true;
        if (pending[b]) {
            ok = tc::mbar_wait(bar[b], phase[b]);
            phase[b] ^= 1u;
            pending[b] = false;
        }
        return !__syncthreads_or(!ok);
    }
    __device__ bool drain() { return wait(0) && wait(1); }
};

__device__ __forceinline__ void fence_to_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// ---------------------------------------------------------------------------
// forward: two M tiles of 128 pixels per pass, N = CO_PAD output channels
template <int CI_PAD, int CO_PAD, bool RELU, bool OUT_F32>
__global__ void __launch_bounds__(CT, 1)
conv_fwd_tc(int n, int L, int ci, int co, const bf16* X, const bf16* W, const float* bias, void* Y, int* err) {
    constexpr int KT = 9 * CI_PAD, KS = KT / 16;
    constexpr int TCOLS = 2 * CO_PAD < 32 ? 32 : 2 * CO_PAD;
    constexpr uint32_t SBO_B = (KT / 8) * 128;
    extern __shared__ unsigned char smraw[];
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ uint32_t tslot;
    unsigned char* Bs = align1k(smraw);                       // CO_PAD x KT, k = t * CI_PAD + c
    unsigned char* As = Bs + CO_PAD * KT * 2;                 // 2 buffers x 2 tiles x 128 rows x 32 B
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int V = L * L;
    for (int e = tid; e < CO_PAD * KT; e += CT) {
        const int o = e / KT, k = e % KT, t = k / CI_PAD, c = k % CI_PAD;
        const bf16 v = (o < co && c < ci) ? W[((size_t)o * ci + c) * 9 + t] : __float2bfloat16(0.f);
        *(bf16*)(Bs + (o >> 3) * SBO_B + (k >> 3) * 128 + (o & 7) * 16 + (k & 7) * 2) = v;
    }
    if (warp == 0) tmem_alloc_warp(&tslot, TCOLS);
    Bufs bf;
    bf.bar[0] = tc::smem_u32(&bars[0]);
    bf.bar[1] = tc::smem_u32(&bars[1]);
    if (tid == 0) {
        tc::mbar_init(bf.bar[0], 1);
        tc::mbar_init(bf.bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    fence_to_async();
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tbase = tslot;
    bool ok = true;
    for (int b = blockIdx.x; b < n && ok; b += gridDim.x) {
        const bf16* Xb = X + (size_t)b * ci * V;
        for (int p0 = 0; p0 < V && ok; p0 += 2 * 128) {
            const int s = p0 + tid;
            for (int ks = 0; ks < KS && ok; ++ks) {
                const int buf = ks & 1;
                if (!(ok = bf.wait(buf))) break;
                const int t = ks / (CI_PAD / 16), c0 = (ks % (CI_PAD / 16)) * 16;
                uint32_t pk[8];
                const int nb = s < V ? shifted(L, s, t, 1) : 0;
#pragma unroll
                for (int h = 0; h < 8; ++h) {
                    const int c = c0 + 2 * h;
                    const bf16 lo = (s < V && c < ci) ? Xb[(size_t)c * V + nb] : __float2bfloat16(0.f);
                    const bf16 hi = (s < V && c + 1 < ci) ? Xb[(size_t)(c + 1) * V + nb] : __float2bfloat16(0.f);
                    pk[h] = (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
                }
                unsigned char* Ab = As + buf * 8192 + (tid >> 7) * 4096;
                const int r = tid & 127;
                *(uint4*)(Ab + tc::cm32(r, 0, 2)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                *(uint4*)(Ab + tc::cm32(r, 8, 2)) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
                fence_to_async();
                __syncthreads();
                if (tid == 0) {
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    const uint64_t bd = tc::desc(tc::smem_u32(Bs + ks * 256), 128, SBO_B);
#pragma unroll
                    for (int m = 0; m < 2; ++m) {
                        const uint64_t ad = tc::desc(tc::smem_u32(As + buf * 8192 + m * 4096), 128, 256);
                        tc::mma_bf16(tbase + m * CO_PAD, ad, bd, tc::idesc_bf16(128, CO_PAD), ks > 0 ? 1u : 0u);
                    }
                    tc::commit(bf.bar[buf]);
                }
                bf.pending[buf] = true;
            }
            if (!ok || !(ok = bf.drain())) break;
            asm volatile("tcgen05.fence::after_thread_sync;");
            // epilogue: warp -> TMEM lane quarter q of tile m
            const int q = warp & 3, m = warp >> 2;
            const int sp = p0 + m * 128 + q * 32 + lane;
#pragma unroll
            for (int j = 0; j < CO_PAD; j += 16) {
                float v[16];
                tc::ld16(tbase + ((uint32_t)(q * 32) << 16) + (uint32_t)(m * CO_PAD + j), v);
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    const int o = j + k;
                    if (o < co && sp < V) {
                        float a = v[k] + bias[o];
                        if (RELU) a = fmaxf(a, 0.f);
                        const size_t oi = ((size_t)b * co + o) * V + sp;
                        if (OUT_F32) ((float*)Y)[oi] = a;
                        else ((bf16*)Y)[oi] = __float2bfloat16(a);
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncthreads();
        }
    }
    bf.drain();
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(TCOLS));
    }
    if (!ok && tid == 0) atomicExch(err, 1);
}

// ---------------------------------------------------------------------------
// input gradient: D[s][c], N = 64 input channels, K = 9 x CO_PAD (TF32 steps of 8)
template <int CO_PAD>
__global__ void __launch_bounds__(CT, 1)
conv_bwd_data_tc(int n, int L, int ci, int co, const bf16* W, const float* dY, const bf16* act, float* dX,
                 int* err) {
    constexpr int NC = 64, KT = 9 * CO_PAD, KS = KT / 8, TCOLS = 2 * NC;
    constexpr uint32_t SBO_B = (KT / 4) * 128;
    extern __shared__ unsigned char smraw[];
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ uint32_t tslot;
    unsigned char* Bs = align1k(smraw);                       // NC x KT floats, k = t * CO_PAD + o
    unsigned char* As = Bs + NC * KT * 4;                     // 2 buffers x 2 tiles x 128 rows x 32 B
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int V = L * L;
    for (int e = tid; e < NC * KT; e += CT) {
        const int c = e / KT, k = e % KT, t = k / CO_PAD, o = k % CO_PAD;
        const float v = (c < ci && o < co) ? __bfloat162float(W[((size_t)o * ci + c) * 9 + t]) : 0.f;
        *(float*)(Bs + (c >> 3) * SBO_B + (k >> 2) * 128 + (c & 7) * 16 + (k & 3) * 4) = v;
    }
    if (warp == 0) tmem_alloc_warp(&tslot, TCOLS);
    Bufs bf;
    bf.bar[0] = tc::smem_u32(&bars[0]);
    bf.bar[1] = tc::smem_u32(&bars[1]);
    if (tid == 0) {
        tc::mbar_init(bf.bar[0], 1);
        tc::mbar_init(bf.bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    fence_to_async();
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tbase = tslot;
    bool ok = true;
    for (int b = blockIdx.x; b < n && ok; b += gridDim.x) {
        const float* dYb = dY + (size_t)b * co * V;
        for (int p0 = 0; p0 < V && ok; p0 += 2 * 128) {
            const int s = p0 + tid;
            for (int ks = 0; ks < KS && ok; ++ks) {
                const int buf = ks & 1;
                if (!(ok = bf.wait(buf))) break;
                const int t = ks / (CO_PAD / 8), o0 = (ks % (CO_PAD / 8)) * 8;
                const int nb = s < V ? shifted(L, s, t, -1) : 0;
                float v[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int o = o0 + k;
                    v[k] = (s < V && o < co) ? tc::tf32_rna(dYb[(size_t)o * V + nb]) : 0.f;
                }
                unsigned char* Ab = As + buf * 8192 + (tid >> 7) * 4096;
                const int r = tid & 127;
                *(float4*)(Ab + tc::cm32(r, 0, 4)) = make_float4(v[0], v[1], v[2], v[3]);
                *(float4*)(Ab + tc::cm32(r, 4, 4)) = make_float4(v[4], v[5], v[6], v[7]);
                fence_to_async();
                __syncthreads();
                if (tid == 0) {
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    const uint64_t bd = tc::desc(tc::smem_u32(Bs + ks * 256), 128, SBO_B);
#pragma unroll
                    for (int m = 0; m < 2; ++m) {
                        const uint64_t ad = tc::desc(tc::smem_u32(As + buf * 8192 + m * 4096), 128, 256);
                        tc::mma_tf32(tbase + m * NC, ad, bd, tc::idesc_tf32(128, NC), ks > 0 ? 1u : 0u);
                    }
                    tc::commit(bf.bar[buf]);
                }
                bf.pending[buf] = true;
            }
            if (!ok || !(ok = bf.drain())) break;
            asm volatile("tcgen05.fence::after_thread_sync;");
            const int q = warp & 3, m = warp >> 2;
            const int sp = p0 + m * 128 + q * 32 + lane;
#pragma unroll
            for (int j = 0; j < NC; j += 16) {
                float v[16];
                tc::ld16(tbase + ((uint32_t)(q * 32) << 16) + (uint32_t)(m * NC + j), v);
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    const int c = j + k;
                    if (c < ci && sp < V) {
                        const size_t xi = ((size_t)b * ci + c) * V + sp;
                        dX[xi] = (act && !(__bfloat162float(act[xi]) > 0.f)) ? 0.f : v[k];
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncthreads();
        }
    }
    bf.drain();
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(TCOLS));
    }
    if (!ok && tid == 0) atomicExch(err, 1);
}

// ---------------------------------------------------------------------------
// weight gradient: D[(t, c)][o], MT tiles of 128 rows (t, c), N = CO_PAD,
// K = pixels (TF32 steps of 8); the CTA's partial sums are added to dW
// (zeroed by the caller).
template <int MT, int CO_PAD>
__global__ void __launch_bounds__(CT, 1)
conv_bwd_weight_tc(int n, int L, int ci, int co, const bf16* X, const float* dY, float* dW, int* err) {
    constexpr int TC_ = MT * CO_PAD <= 32 ? 32 : MT * CO_PAD <= 64 ? 64 : MT * CO_PAD <= 128 ? 128
                        : MT * CO_PAD <= 256 ? 256 : 512;
    constexpr int ABYTES = MT * 128 * 32;                     // one buffer of A
    constexpr int BBYTES = CO_PAD * 32;                       // one buffer of B
    extern __shared__ unsigned char smraw[];
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ uint32_t tslot;
    unsigned char* As = align1k(smraw);
    unsigned char* Bsm = As + 2 * ABYTES;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int V = L * L, R = 9 * ci;                          // rows (t, c) = t * ci + c
    if (warp == 0) tmem_alloc_warp(&tslot, TC_);
    Bufs bf;
    bf.bar[0] = tc::smem_u32(&bars[0]);
    bf.bar[1] = tc::smem_u32(&bars[1]);
    if (tid == 0) {
        tc::mbar_init(bf.bar[0], 1);
        tc::mbar_init(bf.bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tbase = tslot;
    bool ok = true;
    int step = 0;
    for (int b = blockIdx.x; b < n && ok; b += gridDim.x) {
        const bf16* Xb = X + (size_t)b * ci * V;
        const float* dYb = dY + (size_t)b * co * V;
        for (int s0 = 0; s0 < V && ok; s0 += 8, ++step) {
            const int buf = step & 1;
            if (!(ok = bf.wait(buf))) break;
            unsigned char* Ab = As + buf * ABYTES;
            // A: rows (t, c), 8 pixels; 4-wide groups of k per store
            for (int e = tid; e < MT * 128 * 2; e += CT) {
                const int row = e >> 1, kg = (e & 1) * 4;
                const int t = row / ci, c = row - t * ci;
                float v[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int s = s0 + kg + k;
                    v[k] = (row < R && s < V) ? __bfloat162float(Xb[(size_t)c * V + shifted(L, s, t, 1)]) : 0.f;
                }
                *(float4*)(Ab + (row >> 7) * 4096 + tc::cm32(row & 127, kg, 4)) = make_float4(v[0], v[1], v[2], v[3]);
            }
            unsigned char* Bb = Bsm + buf * BBYTES;
            for (int e = tid; e < CO_PAD * 2; e += CT) {
                const int o = e >> 1, kg = (e & 1) * 4;
                float v[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int s = s0 + kg + k;
                    v[k] = (o < co && s < V) ? tc::tf32_rna(dYb[(size_t)o * V + s]) : 0.f;
                }
                *(float4*)(Bb + tc::cm32(o, kg, 4)) = make_float4(v[0], v[1], v[2], v[3]);
            }
            fence_to_async();
            __syncthreads();
            if (tid == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint64_t bd = tc::desc(tc::smem_u32(Bb), 128, 256);
#pragma unroll
                for (int m = 0; m < MT; ++m) {
                    const uint64_t ad = tc::desc(tc::smem_u32(Ab + m * 4096), 128, 256);
                    tc::mma_tf32(tbase + m * CO_PAD, ad, bd, tc::idesc_tf32(128, CO_PAD), step > 0 ? 1u : 0u);
                }
                tc::commit(bf.bar[buf]);
            }
            bf.pending[buf] = true;
        }
    }
    if (ok) ok = bf.drain();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (ok && step > 0) {
        // warp -> lane quarter q; the tiles are shared out over the two warp halves
        const int q = warp & 3;
        for (int m = warp >> 2; m < MT; m += 2) {
            const int row = m * 128 + q * 32 + lane;
            const int t = row / ci, c = row - t * ci;
#pragma unroll
            for (int j = 0; j < CO_PAD; j += 16) {
                float v[16];
                tc::ld16(tbase + ((uint32_t)(q * 32) << 16) + (uint32_t)(m * CO_PAD + j), v);
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    const int o = j + k;
                    if (o < co && row < R) atomicAdd(&dW[((size_t)o * ci + c) * 9 + t], v[k]);
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(TC_));
    }
    if (!ok && tid == 0) atomicExch(err, 1);
}

// db[o] = sum_{b, s} dY[b][o][s]
__global__ void conv_bias_grad(int n, int V, int co, const float* dY, float* db) {
    const int o = blockIdx.x;
    float acc = 0.f;
    for (int e = threadIdx.x; e < n * V; e += blockDim.x) {
        const int b = e / V, s = e - b * V;
        acc += dY[((size_t)b * co + o) * V + s];
    }
    __shared__ float red[32];
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float v = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[w];
        db[o] = v;
    }
}

}  // namespace

// Dynamic shared memory of a launch: at least what the kernel uses, and at
// least enough that the CTAs resident on one SM never ask for more than the
// 512 TMEM columns together (a tcgen05.alloc beyond them would wait for a
// neighbour to finish): 60 KB (at most three CTAs) for up to 128 columns,
// 120 KB (one CTA) for 512.
static size_t launch_smem(size_t need, int tmem_cols) {
    const size_t floor_ = tmem_cols > 128 ? (size_t)120 << 10 : (size_t)60 << 10;
    return need > floor_ ? need : floor_;
}

// Host launchers (the kernels stride over samples; grid at most one CTA per
// SM).  ci, co: the layer's real channel counts (8 -> 64 -> 64 -> 64 -> 6).
ggf_status ggf_conv_fwd_tc(int n, int L, int ci, int co, bool relu, const void* X, const void* W, const float* bias,
                           void* Y, bool out_f32, int* err, int sms, cudaStream_t st) {
    const int grid = n < sms ? n : sms;
    if (grid == 0) return GGF_OK;
    cudaError_t e = cudaSuccess;
#define GGF_FWD(CIP, COP, RL, OF)                                                                              \
    do {                                                                                                       \
        const size_t sm = launch_smem(1024 + (size_t)(COP) * 9 * (CIP) * 2 + 2 * 8192, 2 * (COP));            \
        e = cudaFuncSetAttribute(conv_fwd_tc<CIP, COP, RL, OF>, cudaFuncAttributeMaxDynamicSharedMemorySize,   \
                                 (int)sm);                                                                     \
        if (e == cudaSuccess)                                                                                  \
            conv_fwd_tc<CIP, COP, RL, OF><<<grid, CT, sm, st>>>(n, L, ci, co, (const bf16*)X, (const bf16*)W, \
                                                                 bias, Y, err);                                 \
    } while (0)
    if (ci <= 16 && co <= 64 && relu && !out_f32) GGF_FWD(16, 64, true, false);
    else if (ci <= 64 && co <= 64 && co > 16 && relu && !out_f32) GGF_FWD(64, 64, true, false);
    else if (ci <= 64 && co <= 16 && !relu && out_f32) GGF_FWD(64, 16, false, true);
    else return GGF_EINVAL;
#undef GGF_FWD
    if (e != cudaSuccess) return GGF_ECUDA;
    return cudaGetLastError() == cudaSuccess ? GGF_OK : GGF_ECUDA;
}

ggf_status ggf_conv_bwd_data_tc(int n, int L, int ci, int co, const void* W, const float* dY, const void* act,
                                float* dX, int* err, int sms, cudaStream_t st) {
    const int grid = n < sms ? n : sms;
    if (grid == 0) return GGF_OK;
    if (ci > 64) return GGF_EINVAL;
    cudaError_t e = cudaSuccess;
#define GGF_BWD(COP)                                                                                           \
    do {                                                                                                       \
        const size_t sm = launch_smem(1024 + (size_t)64 * 9 * (COP) * 4 + 2 * 8192, 128);                     \
        e = cudaFuncSetAttribute(conv_bwd_data_tc<COP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm); \
        if (e == cudaSuccess)                                                                                  \
            conv_bwd_data_tc<COP><<<grid, CT, sm, st>>>(n, L, ci, co, (const bf16*)W, dY, (const bf16*)act,  \
                                                        dX, err);                                              \
    } while (0)
    if (co <= 8) GGF_BWD(8);
    else if (co <= 64) GGF_BWD(64);
    else return GGF_EINVAL;
#undef GGF_BWD
    if (e != cudaSuccess) return GGF_ECUDA;
    return cudaGetLastError() == cudaSuccess ? GGF_OK : GGF_ECUDA;
}

ggf_status ggf_conv_bwd_weight_tc(int n, int L, int ci, int co, const void* X, const float* dY, float* dW,
                                  float* db, int* err, int sms, cudaStream_t st) {
    const int grid = n < sms ? n : sms;
    if (grid == 0) return GGF_OK;
    if (cudaMemsetAsync(dW, 0, (size_t)co * ci * 9 * sizeof(float), st) != cudaSuccess) return GGF_ECUDA;
    cudaError_t e = cudaSuccess;
#define GGF_BWW(MT, COP)                                                                                       \
    do {                                                                                                       \
        const size_t sm = launch_smem(1024 + 2 * ((size_t)(MT) * 128 * 32 + (size_t)(COP) * 32), (MT) * (COP));  \
        e = cudaFuncSetAttribute(conv_bwd_weight_tc<MT, COP>, cudaFuncAttributeMaxDynamicSharedMemorySize,     \
                                 (int)sm);                                                                     \
        if (e == cudaSuccess)                                                                                  \
            conv_bwd_weight_tc<MT, COP><<<grid, CT, sm, st>>>(n, L, ci, co, (const bf16*)X, dY, dW, err);      \
    } while (0)
    const int rows = 9 * ci;
    if (rows <= 128 && co <= 64) GGF_BWW(1, 64);
    else if (rows <= 640 && co <= 16) GGF_BWW(5, 16);
    else if (rows <= 640 && co <= 64) GGF_BWW(5, 64);
    else return GGF_EINVAL;
#undef GGF_BWW
    if (e != cudaSuccess) return GGF_ECUDA;
    conv_bias_grad<<<co, 256, 0, st>>>(n, L * L, co, dY, db);
    return cudaGetLastError() == cudaSuccess ? GGF_OK : GGF_ECUDA;
}
