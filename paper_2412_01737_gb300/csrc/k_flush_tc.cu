// Delayed-update flush on the sm_103a tensor cores (tcgen05 + TMEM).
//
// For FP32 chains, folds the pending rank-(k r) panels into the cached
// inverse: W <- W - U V, with U (N x KR) and V^T (N x KR) stored K-major
// (rank index contiguous), complex pairs as separate real/imaginary planes.
// FP32 accuracy from TF32 tensor cores by the three-product split
// x = hi + lo, hi = rna_tf32(x):  a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi.
//
// The MMA computes the transposed tile D^T = V U^T (A operand: 128 rows of
// V^T, B operand: rows of U), so the TMEM lane is the output column and the
// TMEM column the output row: in the epilogue a warp's 32 lanes hold 32
// consecutive columns of W for every row it reads, and its loads and stores
// of W are coalesced without staging.  Persistent CTAs of 128 threads walk
// tiles of 128 columns x 128 rows
// (real) or 128 complex columns x 64 rows (complex: two 64-column
// accumulators, re and im, in the 128 TMEM columns allocated once); four
// CTAs share an SM (all 512 TMEM columns) so that one CTA's loads overlap
// another's MMAs and stores.  Per 16-wide rank chunk the operands are loaded
// (float4, all loads in flight), split into tf32 hi/lo and written in the
// no-swizzle K-major core-matrix layout (8 rows x 16 bytes per core matrix,
// LBO = 128 B along K, SBO = 512 B between 8-row groups); one thread issues
// the MMAs (M = 128, K = 8 each) and commits them to an mbarrier.  Every wait on the mbarrier is bounded; on
// expiry the kernel raises the device error word and frees its TMEM.
#include <cstring>
#include "ggf_ctx.h"

namespace {

constexpr int TC_THREADS = 128;
constexpr int KCH = 16;                       // rank chunk (tf32 elements)
constexpr int SBO = KCH / 4 * 128;            // bytes between 8-row core-matrix groups
constexpr int TILE_BYTES_128 = 128 * KCH * 4; // 8 KB per 128-row operand plane
constexpr int CTAS_PER_SM = 4;                // 4 x 128 TMEM columns = all 512
constexpr int smem_bytes(bool cplx) { return (cplx ? 48 : 32) * 1024 + 1024; }

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// byte offset of (row, k) inside a K-major no-swizzle operand tile (KCH wide)
__device__ __forceinline__ uint32_t cm_off(int row, int k) {
    return (uint32_t)((row >> 3) * SBO + (k >> 2) * 128 + (row & 7) * 16 + (k & 3) * 4);
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);              // start address
    d |= (uint64_t)((128u >> 4) & 0x3FFFu) << 16;         // leading byte offset (K direction)
    d |= (uint64_t)(((uint32_t)SBO >> 4) & 0x3FFFu) << 32; // stride byte offset (8-row groups)
    d |= (uint64_t)1 << 46;                               // descriptor version for sm_100 family
    return d;                                             // base offset 0, no swizzle
}

// instruction descriptor: D f32, A/B tf32, both K-major
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N, bool negA) {
    return (1u << 4) | (2u << 7) | (2u << 10) | (negA ? (1u << 13) : 0u) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t dt, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dt),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ float tf32_hi(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

__device__ __forceinline__ bool mbar_try(uint32_t addr, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(addr), "r"(phase)
        : "memory");
    return ok != 0;
}

__device__ bool mbar_wait_bounded(uint32_t addr, uint32_t phase) {
    long long t0 = clock64();
    while (!mbar_try(addr, phase))
        if (clock64() - t0 > (1LL << 32)) return false;   // about two seconds
    return true;
}

// Load a 32-wide rank chunk of `ROWS` rows (float4 per thread, all loads in
// flight before any store), split into tf32 hi/lo core-matrix tiles.
template <int ROWS>
__device__ __forceinline__ void stage_plane(const float* src, int KRM, int row0, int row_lim, int k0, int K,
                                            unsigned char* hi, unsigned char* lo) {
    constexpr int PER = ROWS * (KCH / 4) / TC_THREADS;   // float4 per thread
    constexpr int Q4 = KCH / 4;                          // float4 per row
    float4 v[PER];
#pragma unroll
    for (int t = 0; t < PER; ++t) {
        int idx = threadIdx.x + t * TC_THREADS;
        int row = idx / Q4, q4 = idx % Q4;
        int gr = row0 + row, gk = k0 + 4 * q4;
        v[t] = (gr < row_lim && gk < K) ? *(const float4*)(src + (size_t)gr * KRM + gk) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int t = 0; t < PER; ++t) {
        int idx = threadIdx.x + t * TC_THREADS;
        int row = idx / Q4, q4 = idx % Q4;
        float4 h = make_float4(tf32_hi(v[t].x), tf32_hi(v[t].y), tf32_hi(v[t].z), tf32_hi(v[t].w));
        float4 l = make_float4(v[t].x - h.x, v[t].y - h.y, v[t].z - h.z, v[t].w - h.w);
        uint32_t o = cm_off(row, 4 * q4);
        *(float4*)(hi + o) = h;
        *(float4*)(lo + o) = l;
    }
}

template <bool CPLX>
__global__ void __launch_bounds__(TC_THREADS, CTAS_PER_SM)
flush_tc_kernel(int N, int fam_pairs, int n_chains, float* W, const float* Pan, const int* pend, int R, int KRM,
                int* err) {
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ uint64_t mbar;
    __shared__ uint32_t tmem_slot;
    __shared__ int s_fail;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // The MMA computes the transposed tile D^T = V^T-rows x U-rows^T: TMEM lane
    // = output column j (128 per tile), TMEM column = output row i.
    constexpr int NROW = CPLX ? 64 : 128;         // output rows per tile (MMA N)
    const int rowW = CPLX ? 2 * N : N;            // floats per W row
    const int tiles_i = (N + NROW - 1) / NROW, tiles_j = (N + 127) / 128;
    const size_t NK = (size_t)N * KRM;
    const long long total = (long long)n_chains * fam_pairs * tiles_i * tiles_j;
    unsigned char* base = (unsigned char*)(((uintptr_t)sm + 1023) & ~(uintptr_t)1023);
    // MMA A operand: V^T rows (re[, im]) x (hi, lo); B operand: U rows likewise
    unsigned char* A0h = base;
    unsigned char* A0l = A0h + TILE_BYTES_128;
    unsigned char* A1h = A0l + TILE_BYTES_128;       // complex only
    unsigned char* A1l = A1h + TILE_BYTES_128;
    unsigned char* B0h = CPLX ? A1l + TILE_BYTES_128 : A1h;
    unsigned char* B0l = B0h + NROW * KCH * 4;
    unsigned char* B1h = B0l + NROW * KCH * 4;       // complex only
    unsigned char* B1l = B1h + NROW * KCH * 4;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(128));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
        s_fail = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tbase = tmem_slot;
    const uint32_t mb = smem_u32(&mbar);
    uint32_t phase = 0;

    for (long long tile = blockIdx.x; tile < total; tile += gridDim.x) {
        long long rest = tile;
        const int tj = (int)(rest % tiles_j); rest /= tiles_j;
        const int ti = (int)(rest % tiles_i); rest /= tiles_i;
        const int p = (int)(rest % fam_pairs); rest /= fam_pairs;
        const int c = (int)rest;
        const int K = pend[c] * R;
        if (K == 0) continue;
        const size_t blk = ((size_t)c * fam_pairs + p) * (CPLX ? 4 : 2) * NK;
        const float* U0 = Pan + blk;                         // U (re)
        const float* U1 = U0 + NK;                           // U im (complex)
        const float* V0 = Pan + blk + (CPLX ? 2 : 1) * NK;   // V^T (re)
        const float* V1 = V0 + NK;
        const int i0 = ti * NROW, j0 = tj * 128;
        float* Wp = W + ((size_t)c * fam_pairs + p) * (size_t)N * rowW;
        for (int k0 = 0; k0 < K; k0 += KCH) {
            stage_plane<128>(V0, KRM, j0, N, k0, K, A0h, A0l);
            stage_plane<NROW>(U0, KRM, i0, N, k0, K, B0h, B0l);
            if (CPLX) {
                stage_plane<128>(V1, KRM, j0, N, k0, K, A1h, A1l);
                stage_plane<NROW>(U1, KRM, i0, N, k0, K, B1h, B1l);
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
            if (threadIdx.x == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t a0h = smem_u32(A0h), a0l = smem_u32(A0l), b0h = smem_u32(B0h), b0l = smem_u32(B0l);
                const uint32_t a1h = smem_u32(A1h), a1l = smem_u32(A1l), b1h = smem_u32(B1h), b1l = smem_u32(B1l);
#pragma unroll
                for (int kk = 0; kk < KCH / 8; ++kk) {
                    const uint32_t o = kk * 256;             // two core matrices along K per MMA
                    const uint32_t first = (k0 == 0 && kk == 0) ? 0u : 1u;
                    if (!CPLX) {
                        constexpr uint32_t id = idesc_tf32(128, 128, false);
                        mma_tf32(tbase, smem_desc(a0h + o), smem_desc(b0h + o), id, first);
                        mma_tf32(tbase, smem_desc(a0h + o), smem_desc(b0l + o), id, 1u);
                        mma_tf32(tbase, smem_desc(a0l + o), smem_desc(b0h + o), id, 1u);
                    } else {
                        constexpr uint32_t id = idesc_tf32(128, 64, false);
                        constexpr uint32_t idn = idesc_tf32(128, 64, true);
                        const uint32_t dre = tbase, dim = tbase + 64;
                        // re(D^T) = Vr Ur^T - Vi Ui^T
                        mma_tf32(dre, smem_desc(a0h + o), smem_desc(b0h + o), id, first);
                        mma_tf32(dre, smem_desc(a0h + o), smem_desc(b0l + o), id, 1u);
                        mma_tf32(dre, smem_desc(a0l + o), smem_desc(b0h + o), id, 1u);
                        mma_tf32(dre, smem_desc(a1h + o), smem_desc(b1h + o), idn, 1u);
                        mma_tf32(dre, smem_desc(a1h + o), smem_desc(b1l + o), idn, 1u);
                        mma_tf32(dre, smem_desc(a1l + o), smem_desc(b1h + o), idn, 1u);
                        // im(D^T) = Vr Ui^T + Vi Ur^T
                        mma_tf32(dim, smem_desc(a0h + o), smem_desc(b1h + o), id, first);
                        mma_tf32(dim, smem_desc(a0h + o), smem_desc(b1l + o), id, 1u);
                        mma_tf32(dim, smem_desc(a0l + o), smem_desc(b1h + o), id, 1u);
                        mma_tf32(dim, smem_desc(a1h + o), smem_desc(b0h + o), id, 1u);
                        mma_tf32(dim, smem_desc(a1h + o), smem_desc(b0l + o), id, 1u);
                        mma_tf32(dim, smem_desc(a1l + o), smem_desc(b0h + o), id, 1u);
                    }
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb)
                             : "memory");
                if (!mbar_wait_bounded(mb, phase)) {
                    s_fail = 1;
                    atomicExch(err, 1);
                    mbar_wait_bounded(mb, phase);   // second bounded wait for the MMAs in flight
                }
            }
            phase ^= 1u;
            __syncthreads();
            if (s_fail) break;
        }
        if (s_fail) break;
        asm volatile("tcgen05.fence::after_thread_sync;");
        // epilogue: lane = output column j, register k of block cb = output row
        // i0 + 16 cb + k; a warp touches 32 consecutive columns (coalesced)
        {
            const int j = j0 + warp * 32 + lane;
            const uint32_t tl = tbase + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
            for (int cb = 0; cb < NROW / 16; ++cb) {
                uint32_t v[16];
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15},"
                    " [%16];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                      "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                      "=r"(v[15])
                    : "r"(tl + cb * 16));
                if (!CPLX) {
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    float w[16];
#pragma unroll
                    for (int k = 0; k < 16; ++k) {
                        const int i = i0 + cb * 16 + k;
                        w[k] = (i < N && j < N) ? Wp[(size_t)i * N + j] : 0.f;
                    }
#pragma unroll
                    for (int k = 0; k < 16; ++k) {
                        const int i = i0 + cb * 16 + k;
                        if (i < N && j < N) Wp[(size_t)i * N + j] = w[k] - __uint_as_float(v[k]);
                    }
                } else {
                    uint32_t vi[16];
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
                        "%15}, [%16];"
                        : "=r"(vi[0]), "=r"(vi[1]), "=r"(vi[2]), "=r"(vi[3]), "=r"(vi[4]), "=r"(vi[5]), "=r"(vi[6]),
                          "=r"(vi[7]), "=r"(vi[8]), "=r"(vi[9]), "=r"(vi[10]), "=r"(vi[11]), "=r"(vi[12]),
                          "=r"(vi[13]), "=r"(vi[14]), "=r"(vi[15])
                        : "r"(tl + 64 + cb * 16));
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    float2 w[16];
#pragma unroll
                    for (int k = 0; k < 16; ++k) {
                        const int i = i0 + cb * 16 + k;
                        w[k] = (i < N && j < N) ? *(const float2*)(Wp + (size_t)i * rowW + 2 * j) : make_float2(0.f, 0.f);
                    }
#pragma unroll
                    for (int k = 0; k < 16; ++k) {
                        const int i = i0 + cb * 16 + k;
                        if (i < N && j < N)
                            *(float2*)(Wp + (size_t)i * rowW + 2 * j) =
                                make_float2(w[k].x - __uint_as_float(v[k]), w[k].y - __uint_as_float(vi[k]));
                    }
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
    }
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(128));
    }
}

}  // namespace

// Shared-memory attributes of the tensor-core flush, set once per process and
// device ordinal outside any stream capture.
ggf_status ggf_prepare_flush_tc(ggf_ctx* ctx) {
    static bool done[64] = {false};
    if (ctx->device >= 0 && ctx->device < 64 && done[ctx->device]) return GGF_OK;
    GGF_CK(cudaFuncSetAttribute(flush_tc_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes(true)));
    GGF_CK(cudaFuncSetAttribute(flush_tc_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes(false)));
    if (ctx->device >= 0 && ctx->device < 64) done[ctx->device] = true;
    return GGF_OK;
}

namespace {

ggf_status launch_flush_tc(ggf_ctx* ctx, bool cplx, int N, int fam_pairs, int n_chains, float* W, const float* Pan,
                           const int* pend, int R, int KRM, int* err, cudaStream_t st) {
    if (fam_pairs == 0 || n_chains == 0) return GGF_OK;
    const int rowW = cplx ? 2 * N : N;
    const long long total = (long long)n_chains * fam_pairs * ((N + (cplx ? 63 : 127)) / (cplx ? 64 : 128)) *
                            ((N + 127) / 128);
    int sms = ctx->n_sms > 0 ? ctx->n_sms : 152;
    const long long grid = std::min<long long>(total, (long long)sms * CTAS_PER_SM);
    GGF_TRY(ggf_prepare_flush_tc(ctx));
    if (cplx) {
        flush_tc_kernel<true><<<(unsigned)grid, TC_THREADS, smem_bytes(true), st>>>(N, fam_pairs, n_chains, W, Pan,
                                                                                    pend, R, KRM, err);
    } else {
        flush_tc_kernel<false><<<(unsigned)grid, TC_THREADS, smem_bytes(false), st>>>(N, fam_pairs, n_chains, W, Pan,
                                                                                      pend, R, KRM, err);
    }
    GGF_CK(cudaGetLastError());
    return GGF_OK;
}

// ---- self-test: one (chain, pair) against an FP64 reference --------------------
__device__ __forceinline__ float hash_val(uint64_t i, uint64_t salt) {
    uint64_t c[4] = {i, salt, 0, 0}, o[4];
    philox4x64_10(c, 0x1234, 0x5678, o);
    return (float)(u53(o[0]) * 2.0 - 1.0);
}

__global__ void st_fill(float* p, size_t n, uint64_t salt, float scale) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = scale * hash_val(i, salt);
}

__global__ void st_reference(bool cplx, int N, int K, int KRM, const float* W0, const float* Pan, double* ref) {
    const int rowW = cplx ? 2 * N : N;
    size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (size_t)N * rowW) return;
    const size_t NK = (size_t)N * KRM;
    int i = (int)(e / rowW), f = (int)(e % rowW);
    if (!cplx) {
        double s = 0.0;
        for (int q = 0; q < K; ++q) s += (double)Pan[(size_t)i * KRM + q] * (double)Pan[NK + (size_t)f * KRM + q];
        ref[e] = (double)W0[e] - s;
    } else {
        int j = f >> 1, part = f & 1;
        double sr = 0.0, si = 0.0;
        for (int q = 0; q < K; ++q) {
            double ur = Pan[(size_t)i * KRM + q], ui = Pan[NK + (size_t)i * KRM + q];
            double vr = Pan[2 * NK + (size_t)j * KRM + q], vi = Pan[3 * NK + (size_t)j * KRM + q];
            sr += ur * vr - ui * vi;
            si += ur * vi + ui * vr;
        }
        ref[e] = (double)W0[e] - (part ? si : sr);
    }
}

__global__ void st_maxerr(size_t n, const float* got, const double* ref, unsigned long long* out) {
    size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    double d = fabs((double)got[e] - ref[e]);
    double m = fabs(ref[e]);
    atomicMax(&out[0], __double_as_longlong(d));
    atomicMax(&out[1], __double_as_longlong(m));
}

}  // namespace

ggf_status ggf_flush_tc(ggf_ctx* ctx, cudaStream_t st) {
    Chains& ch = ctx->ch;
    const Geometry& g = ctx->g;
    const int KRM = ch.kmax * g.r;
    GGF_TRY(launch_flush_tc(ctx, false, g.N, ctx->K, ch.n, (float*)ch.Wr, (const float*)ch.Pr, ch.pend, g.r, KRM,
                            ctx->d_err, st));
    GGF_TRY(launch_flush_tc(ctx, true, g.N, ctx->Kc, ch.n, (float*)ch.Wc, (const float*)ch.Pc, ch.pend, g.r, KRM,
                            ctx->d_err, st));
    return GGF_OK;
}

extern "C" ggf_status ggf_selftest_flush(ggf_ctx* ctx, int cplx, int N, int rank, double* max_rel_err) {
    if (!ctx || !max_rel_err || N < 1 || N > 8192 || rank < 8 || rank > 128 || rank % 8)
        return ggf_fail(ctx, GGF_EINVAL, "selftest_flush: N in [1, 8192], rank in {8, 16, ..., 128}");
    cudaSetDevice(ctx->device);
    const int R = 8, KRM = rank;
    const int rowW = cplx ? 2 * N : N;
    const size_t NK = (size_t)N * KRM, nW = (size_t)N * rowW, nP = (cplx ? 4 : 2) * NK;
    float *W = nullptr, *Pan = nullptr;
    double* ref = nullptr;
    int* pend = nullptr;
    unsigned long long* mx = nullptr;
    ggf_status rc = GGF_OK;
    auto cleanup = [&]() {
        if (W) cudaFree(W);
        if (Pan) cudaFree(Pan);
        if (ref) cudaFree(ref);
        if (pend) cudaFree(pend);
        if (mx) cudaFree(mx);
    };
    if (cudaMalloc(&W, nW * 4) != cudaSuccess || cudaMalloc(&Pan, nP * 4) != cudaSuccess ||
        cudaMalloc(&ref, nW * 8) != cudaSuccess || cudaMalloc(&pend, 4) != cudaSuccess ||
        cudaMalloc(&mx, 16) != cudaSuccess) {
        cleanup();
        return ggf_fail(ctx, GGF_ENOMEM, "selftest_flush allocation failed");
    }
    int pv = rank / R;
    cudaMemcpy(pend, &pv, 4, cudaMemcpyHostToDevice);
    cudaMemset(mx, 0, 16);
    st_fill<<<(unsigned)((nW + 255) / 256), 256>>>(W, nW, 1, 1.0f);
    st_fill<<<(unsigned)((nP + 255) / 256), 256>>>(Pan, nP, 2, 0.3f);
    st_reference<<<(unsigned)((nW + 255) / 256), 256>>>(cplx != 0, N, rank, KRM, W, Pan, ref);
    rc = launch_flush_tc(ctx, cplx != 0, N, 1, 1, W, Pan, pend, R, KRM, ctx->d_err, 0);
    if (rc == GGF_OK) {
        st_maxerr<<<(unsigned)((nW + 255) / 256), 256>>>(nW, W, ref, mx);
        unsigned long long h[2] = {0, 0};
        int herr = 0;
        if (cudaMemcpy(h, mx, 16, cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(&herr, ctx->d_err, 4, cudaMemcpyDeviceToHost) != cudaSuccess) {
            rc = ggf_cuda(ctx, cudaGetLastError(), "selftest_flush");
        } else if (herr) {
            rc = ggf_fail(ctx, GGF_ETIMEOUT, "tensor-core flush: mbarrier wait ran out");
        } else {
            double d, m;
            std::memcpy(&d, &h[0], 8);
            std::memcpy(&m, &h[1], 8);
            *max_rel_err = d / (m > 0 ? m : 1.0);
        }
    }
    cleanup();
    return rc;
}
