// The X product of the batched updates, V^T <- V^T X^T, for FP32 chains on
// the sm_103a tensor cores (tcgen05.mma kind::tf32, accumulators in TMEM).
//
// Per (chain, pair) the batch leaves Y^T = W[T, :]^T (N x kr) in the V^T
// panel and the kr x kr matrix X in the small-matrix store; the flush then
// needs V^T = Y^T X^T.  As a GEMM: D[i][a] = sum_b Vt[i][b] X[a][b], M = 128
// panel rows i per tile, N = the output columns a (128 per block, zero-padded;
// complex pairs 256: re in columns 0..127, im in 128..255), K = b in steps of
// 8.  FP32 accuracy from the TF32 split x = hi + lo (a b ~ a_hi b_hi +
// a_hi b_lo + a_lo b_hi), as in the flush.  Complex pairs use the flush's
// composite B operand: rows [-X_i ; X_r ; X_i], so that
//   D[:, 0:256] += V_r [X_r ; X_i]^T + V_i [-X_i ; X_r]^T.
//
// A CTA (256 threads) owns 128 panel rows of one (chain, pair) at a time:
// every thread loads one 16-byte piece of A and of each B block per K step
// (one step ahead, into registers) and splits it into the no-swizzle K-major
// core-matrix layout, one thread issues the MMAs, and two operand buffers
// alternate.  All NBLK output blocks (kr <= 128 NBLK) sit in TMEM together, so
// the rows are rewritten in place only after every K step has read them.
//
// Accuracy: the K steps are dealt round-robin to NACC accumulators per block
// (4 for real pairs, 2 for complex ones, what 512 TMEM columns hold), summed
// in FP32 by the epilogue.  With one accumulator over the 16 steps of a
// rank-128 batch, the tracked log-weight of FP32 16x16 Z2 chains drifted
// 3.3e-6 per accepted flip against 1.7e-6 with the FP32 FMA version of this
// product; with four, 2.3e-6.  Neither the fourth split product
// (a_lo b_lo) nor rounding the lo part to TF32 changed it: the length of
// the tensor-core accumulation is what matters.  The sampler therefore keeps
// Z2 chains on the FMA-pipe product and uses this kernel for U(1) and SU(2)
// chains, whose small moves drift ~1e-8 per accept either way.
//
// Waits are bounded; on expiry the CTA stops, raises the context's error
// word and frees its TMEM.
#include "ggf_ctx.h"
#include "ggf_tc.cuh"

// Split products per operand pair: 3 (a_hi b_hi + a_hi b_lo + a_lo b_hi) or
// 4 (also a_lo b_lo, the exact product of the split operands).
#ifndef GGF_APPLY_TERMS
#define GGF_APPLY_TERMS 3
#endif
// Accumulators per output block (K steps dealt round-robin, summed in FP32 in
// the epilogue), at most what 512 TMEM columns hold; and 1: the lo part of the
// split is rounded to TF32 (else the MMA drops its low 13 bits).
#ifndef GGF_APPLY_NACC
#define GGF_APPLY_NACC 4
#endif
#ifndef GGF_SPLIT_LO_RNA
#define GGF_SPLIT_LO_RNA 0
#endif

namespace {

constexpr int APPLY_TERMS = GGF_APPLY_TERMS;
constexpr int AT = 256;                       // threads per CTA
constexpr int PLANE = 128 * 8 * 4;            // 4 KB: 128 rows x 8 tf32 (one K step)

__host__ __device__ constexpr int nacc(bool cplx, int nblk) {
    return GGF_APPLY_NACC * (cplx ? 256 : 128) * nblk <= 512 ? GGF_APPLY_NACC : 512 / ((cplx ? 256 : 128) * nblk);
}
__host__ __device__ constexpr int tmem_cols(bool cplx, int nblk) { return (cplx ? 256 : 128) * nblk * nacc(cplx, nblk); }
// one operand buffer: A (hi, lo; complex re and im) and B (hi, lo; complex
// the 384-row composite) of every output block
__host__ __device__ constexpr int buf_bytes(bool cplx, int nblk) {
    return (cplx ? 4 : 2) * PLANE + nblk * (cplx ? 6 : 2) * PLANE;
}

struct Bufs {
    uint32_t bar[2];
    uint32_t phase[2] = {0u, 0u};
    bool pending[2] = {false, false};
    // wait until the MMAs that read buffer b have completed; every thread
    // takes the same waits and agrees on the outcome
    __device__ bool wait(int b) {
        bool ok = true;
        if (pending[b]) {
            ok = tc::mbar_wait(bar[b], phase[b]);
            phase[b] ^= 1u;
            pending[b] = false;
        }
        return !__syncthreads_or(!ok);
    }
};

__device__ __forceinline__ float4 split_hi(float4 x) {
    return make_float4(tc::tf32_rna(x.x), tc::tf32_rna(x.y), tc::tf32_rna(x.z), tc::tf32_rna(x.w));
}
__device__ __forceinline__ float4 sub4(float4 a, float4 b) { return make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w); }
__device__ __forceinline__ float4 neg4(float4 a) { return make_float4(-a.x, -a.y, -a.z, -a.w); }

// write x (4 consecutive k of row `row`, k a multiple of 4) as tf32 hi into
// plane hi and the remainder into plane lo (8-wide K-major core-matrix planes)
__device__ __forceinline__ void put_split(unsigned char* hi, unsigned char* lo, int row, int k, float4 x) {
    const float4 h = split_hi(x);
    const uint32_t cm = tc::cm32(row, k, 4);
    *(float4*)(hi + cm) = h;
    const float4 l = sub4(x, h);
    *(float4*)(lo + cm) = GGF_SPLIT_LO_RNA ? split_hi(l) : l;
}

template <bool CPLX, int NBLK>
__global__ void __launch_bounds__(AT, 1)
apply_tc_kernel(int N, int fam_pairs, int n_chains, int KRM, int kr, float* Pan, const float* Sm, const int* pend,
                int* err) {
    extern __shared__ unsigned char smraw[];
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ uint32_t tslot;
    constexpr int BB = buf_bytes(CPLX, NBLK);
    constexpr int TCOLS = tmem_cols(CPLX, NBLK);
    constexpr int PL = CPLX ? 2 : 1;              // panel planes (re, im)
    constexpr int DCOLS = CPLX ? 256 : 128;       // TMEM columns of one output block
    constexpr int NACC = nacc(CPLX, NBLK);        // accumulators per block
    // an earlier bounded wait of this context ran out: do nothing
    if (*(volatile int*)err) return;
    unsigned char* sb = (unsigned char*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::smem_u32(&tslot)),
                     "r"(TCOLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    Bufs bf;
    bf.bar[0] = tc::smem_u32(&bars[0]);
    bf.bar[1] = tc::smem_u32(&bars[1]);
    if (tid == 0) {
        tc::mbar_init(bf.bar[0], 1);
        tc::mbar_init(bf.bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tbase = tslot;
    const size_t NK = panel_plane(N, KRM);
    const int NP = panel_rows(N);
    const int tiles_i = (N + 127) / 128;
    const long long total = (long long)n_chains * fam_pairs * tiles_i;
    const int nks = (kr + 7) / 8;
    const int row = tid & 127, kq = 4 * (tid >> 7);          // this thread's operand row and 4 K columns
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    bool ok = true;
    for (long long tile = blockIdx.x; tile < total && ok; tile += gridDim.x) {
        const int ti = (int)(tile % tiles_i);
        const long long rest = tile / tiles_i;
        const int p = (int)(rest % fam_pairs), c = (int)(rest / fam_pairs);
        if (pend[c] == 0) continue;                          // no accepted link: V^T stays
        const size_t base = (size_t)c * fam_pairs + p;
        float* Vt = Pan + (base * 2 + 1) * PL * NK;
        const float* Xm = Sm + (base * 2 * KRM * KRM + (size_t)KRM * KRM) * PL;
        const int i0 = ti * 128;
        // one K step's operand values of this thread: A (V^T row i0 + row) and
        // B (X row 128 blk + row), rank columns b .. b + 3.  Loads only where
        // b < kr: kr = links x r with r = 4 n_v, a multiple of 4 (checked by
        // the launcher), so a group of 4 columns that starts inside the matrix
        // ends inside it.
        struct Vals {
            float4 ar, ai, br[NBLK], bi[NBLK];
        };
        auto load = [&](int ks, Vals& x) {
            const int b = ks * 8 + kq, i = i0 + row;
            x.ar = x.ai = zero;
            if (i < N && b < kr) {
                x.ar = *(const float4*)(Vt + pidx(i, b, NP));
                if (CPLX) x.ai = *(const float4*)(Vt + NK + pidx(i, b, NP));
            }
#pragma unroll
            for (int blk = 0; blk < NBLK; ++blk) {
                const int a = blk * 128 + row;
                x.br[blk] = x.bi[blk] = zero;
                if (a < kr && b < kr) {
                    if (!CPLX) {
                        x.br[blk] = *(const float4*)(Xm + (size_t)a * KRM + b);
                    } else {
                        const float4 v0 = *(const float4*)(Xm + 2 * ((size_t)a * KRM + b));
                        const float4 v1 = *(const float4*)(Xm + 2 * ((size_t)a * KRM + b) + 4);
                        x.br[blk] = make_float4(v0.x, v0.z, v1.x, v1.z);
                        x.bi[blk] = make_float4(v0.y, v0.w, v1.y, v1.w);
                    }
                }
            }
        };
        Vals cur, nxt;
        load(0, cur);
        for (int ks = 0; ks < nks && ok; ++ks) {
            const int buf = ks & 1;
            if (!(ok = bf.wait(buf))) break;
            unsigned char* B0 = sb + buf * BB;
            put_split(B0, B0 + PLANE, row, kq, cur.ar);
            if (CPLX) put_split(B0 + 2 * PLANE, B0 + 3 * PLANE, row, kq, cur.ai);
#pragma unroll
            for (int blk = 0; blk < NBLK; ++blk) {
                if (!CPLX) {
                    unsigned char* bh = B0 + 2 * PLANE + blk * 2 * PLANE;
                    put_split(bh, bh + PLANE, row, kq, cur.br[blk]);
                } else {
                    unsigned char* bh = B0 + 4 * PLANE + blk * 6 * PLANE;
                    unsigned char* bl = bh + 3 * PLANE;
                    put_split(bh, bl, row, kq, neg4(cur.bi[blk]));   // composite rows 0 .. 127: -X_i
                    put_split(bh, bl, 128 + row, kq, cur.br[blk]);   // 128 .. 255: X_r
                    put_split(bh, bl, 256 + row, kq, cur.bi[blk]);   // 256 .. 383: X_i
                }
            }
            // the next step's loads are in flight during this step's MMAs
            if (ks + 1 < nks) load(ks + 1, nxt);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
            if (tid == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t s0 = tc::smem_u32(B0);
                const uint32_t acc = ks >= NACC ? 1u : 0u;
#pragma unroll
                for (int blk = 0; blk < NBLK; ++blk) {
                    const uint32_t d = tbase + (uint32_t)(((ks % NACC) * NBLK + blk) * DCOLS);
                    if (!CPLX) {
                        constexpr uint32_t id = tc::idesc_tf32(128, 128);
                        const uint32_t bh = s0 + 2 * PLANE + blk * 2 * PLANE, bl = bh + PLANE;
                        tc::mma_tf32(d, tc::desc(s0, 128, 256), tc::desc(bh, 128, 256), id, acc);
                        tc::mma_tf32(d, tc::desc(s0, 128, 256), tc::desc(bl, 128, 256), id, 1u);
                        tc::mma_tf32(d, tc::desc(s0 + PLANE, 128, 256), tc::desc(bh, 128, 256), id, 1u);
                        if (APPLY_TERMS == 4) tc::mma_tf32(d, tc::desc(s0 + PLANE, 128, 256), tc::desc(bl, 128, 256), id, 1u);
                    } else {
                        constexpr uint32_t id = tc::idesc_tf32(128, 256);
                        const uint32_t arh = s0, arl = s0 + PLANE, aih = s0 + 2 * PLANE, ail = s0 + 3 * PLANE;
                        const uint32_t bh = s0 + 4 * PLANE + blk * 6 * PLANE, bl = bh + 3 * PLANE;
                        // rows 128 .. 383 = [X_r ; X_i] against V_r, rows 0 .. 255 = [-X_i ; X_r] against V_i
                        tc::mma_tf32(d, tc::desc(arh, 128, 256), tc::desc(bh + PLANE, 128, 256), id, acc);
                        tc::mma_tf32(d, tc::desc(arh, 128, 256), tc::desc(bl + PLANE, 128, 256), id, 1u);
                        tc::mma_tf32(d, tc::desc(arl, 128, 256), tc::desc(bh + PLANE, 128, 256), id, 1u);
                        if (APPLY_TERMS == 4)
                            tc::mma_tf32(d, tc::desc(arl, 128, 256), tc::desc(bl + PLANE, 128, 256), id, 1u);
                        tc::mma_tf32(d, tc::desc(aih, 128, 256), tc::desc(bh, 128, 256), id, 1u);
                        tc::mma_tf32(d, tc::desc(aih, 128, 256), tc::desc(bl, 128, 256), id, 1u);
                        tc::mma_tf32(d, tc::desc(ail, 128, 256), tc::desc(bh, 128, 256), id, 1u);
                        if (APPLY_TERMS == 4) tc::mma_tf32(d, tc::desc(ail, 128, 256), tc::desc(bl, 128, 256), id, 1u);
                    }
                }
                tc::commit(bf.bar[buf]);
            }
            bf.pending[buf] = true;
            cur = nxt;
        }
        if (!ok) break;
        // every MMA of the tile has completed before the rows are rewritten
        if (!(ok = bf.wait(0))) break;
        if (!(ok = bf.wait(1))) break;
        asm volatile("tcgen05.fence::after_thread_sync;");
        // epilogue: warp w reads TMEM lanes 32 (w mod 4) .. + 31 (rows), output
        // columns 64 (w / 4) .. + 63 of every block, 16 at a time
        const int q = warp & 3, h = warp >> 2;
        const int i = i0 + q * 32 + lane;
        const uint32_t tl = tbase + ((uint32_t)(q * 32) << 16);
#pragma unroll 1
        for (int blk = 0; blk < NBLK; ++blk) {
#pragma unroll 1
            for (int g = 0; g < 4; ++g) {
                const int al = h * 64 + 16 * g;                     // column inside the block
                float v[16], vi[16];
                tc::ld16(tl + (uint32_t)(blk * DCOLS + al), v);       // whole warp, converged
                if (CPLX) tc::ld16(tl + (uint32_t)(blk * DCOLS + 128 + al), vi);
#pragma unroll 1
                for (int ac = 1; ac < NACC && ac < nks; ++ac) {
                    float w[16];
                    const uint32_t o = (uint32_t)((ac * NBLK + blk) * DCOLS + al);
                    tc::ld16(tl + o, w);
#pragma unroll
                    for (int e = 0; e < 16; ++e) v[e] += w[e];
                    if (CPLX) {
                        tc::ld16(tl + o + 128, w);
#pragma unroll
                        for (int e = 0; e < 16; ++e) vi[e] += w[e];
                    }
                }
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int a = blk * 128 + al + 4 * e;
                    if (i >= N || a >= kr) continue;
                    const size_t o = pidx(i, a, NP);
                    *(float4*)(Vt + o) = make_float4(v[4 * e], v[4 * e + 1], v[4 * e + 2], v[4 * e + 3]);
                    if (CPLX)
                        *(float4*)(Vt + NK + o) = make_float4(vi[4 * e], vi[4 * e + 1], vi[4 * e + 2], vi[4 * e + 3]);
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
    }
    if (!ok && tid == 0) atomicExch(err, 1);
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(TCOLS));
    }
}

// Dynamic shared memory of a launch: the two operand buffers, raised where
// needed so that no more CTAs share an SM than its 512 TMEM columns serve.
template <bool CPLX, int NBLK>
int apply_smem() {
    const int need = 2 * buf_bytes(CPLX, NBLK) + 1024;
    const int per_sm = 512 / tmem_cols(CPLX, NBLK);
    const int floor = 228 * 1024 / (per_sm + 1);
    return need > floor ? need : floor;
}

template <bool CPLX, int NBLK>
ggf_status launch_apply(ggf_ctx* ctx, int fam_pairs, int kr, float* Pan, const float* Sm, cudaStream_t st) {
    static bool attr[64] = {false};
    const int smem = apply_smem<CPLX, NBLK>();
    if (ctx->device < 0 || ctx->device >= 64) return ggf_fail(ctx, GGF_EINVAL, "device ordinal out of range");
    if (!attr[ctx->device]) {
        GGF_CK(cudaFuncSetAttribute(apply_tc_kernel<CPLX, NBLK>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        attr[ctx->device] = true;
    }
    const Chains& ch = ctx->ch;
    const int N = ctx->g.N;
    const long long tiles = (long long)ch.n * fam_pairs * ((N + 127) / 128);
    const int sms = ctx->n_sms > 0 ? ctx->n_sms : 152;
    const long long grid = std::min<long long>(tiles, (long long)sms * (512 / tmem_cols(CPLX, NBLK)));
    apply_tc_kernel<CPLX, NBLK><<<(unsigned)grid, AT, smem, st>>>(N, fam_pairs, ch.n, ch.kmax * ctx->g.r, kr, Pan, Sm,
                                                                  ch.pend, ctx->d_err);
    GGF_CK(cudaGetLastError());
    return GGF_OK;
}

}  // namespace

// V^T <- V^T X^T of one batch for every chain and pair of a family (FP32
// chains, kr <= 256; Sm is the family's small-matrix store).
ggf_status ggf_apply_tc(ggf_ctx* ctx, bool cplx, int fam_pairs, int kr, float* Pan, const float* Sm, cudaStream_t st) {
    if (fam_pairs == 0) return GGF_OK;
    if (kr < 4 || kr > 256 || kr % 4) return ggf_fail(ctx, GGF_EINVAL, "tensor-core X product: rank must be a multiple of 4 in [4, 256]");
    if (cplx) return kr <= 128 ? launch_apply<true, 1>(ctx, fam_pairs, kr, Pan, Sm, st)
                               : launch_apply<true, 2>(ctx, fam_pairs, kr, Pan, Sm, st);
    return kr <= 128 ? launch_apply<false, 1>(ctx, fam_pairs, kr, Pan, Sm, st)
                     : launch_apply<false, 2>(ctx, fam_pairs, kr, Pan, Sm, st);
}
