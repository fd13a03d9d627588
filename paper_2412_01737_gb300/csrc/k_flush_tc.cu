// Delayed-update flush on the sm_103a tensor cores (tcgen05 + TMEM).
//
// For FP32 chains, folds the pending rank-K panels into the cached inverse:
// W <- W - U V (with `upper` set, only the tiles that touch the upper
// triangle; the sampler updates the whole matrix), with U (N x K) and V^T
// (N x K) panels (rank index
// contiguous, row stride KRM), complex pairs as separate real/imaginary
// planes.  FP32 accuracy from TF32 tensor cores by the three-product split
// x = hi + lo, hi = rna_tf32(x):  a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi.
//
// The MMA computes the transposed tile D^T = V U^T (A operand: 128 rows of
// V^T, i.e. 128 columns of W; B operand: rows of U), so the TMEM lane is the
// output column and the TMEM column the output row: in the epilogue a warp's
// 32 lanes hold 32 consecutive columns of W for every row, and its loads and
// stores of W are coalesced without staging.  Every MMA is M = 128, N = 256,
// K = 8: real tiles are 128 columns x 256 rows; complex tiles are 128 complex
// columns x 128 rows, with the B operand the composite [-U_i ; U_r ; U_i]
// (384 rows), so that
//   D[:, 0:256] += V_r [U_r ; U_i]^T + V_i [-U_i ; U_r]^T
// holds re(D^T) in TMEM columns 0..127 and im(D^T) in 128..255.
//
// Two kernels share the MMA issuer and the epilogue below.  The sweep's
// flush (and the refresh's Newton product, when the scratch holds it) is
// flush_ps_kernel: the operands are split once per chain wave by
// ps_split_kernel into pre-split stage blocks, which one thread bulk-copies
// into the stages (further down).  flush_tc_kernel, laid out here, splits the
// operands per tile; it serves the Newton product when the scratch is too
// small, and the self-test.
//
// flush_tc_kernel: one persistent CTA per SM, warp-specialised:
//   warps 0-7   producers: copy an 8-wide rank chunk of the operands into
//               a private raw shared-memory slot with cp.async (16 bytes
//               per copy, zero-filled outside the matrix; PD stages of
//               copies in flight ahead), then split each thread's own
//               values into tf32 hi/lo and write them in the no-swizzle
//               K-major core-matrix layout (8 rows x 16 B core matrices,
//               LBO = 128 B along K, SBO = 256 B between 8-row groups) into a
//               ring of STAGES shared-memory stages;
//   warp 16     one thread issues the MMAs of each stage and commits them to
//               the stage's "empty" mbarrier, and after a tile's last stage
//               to the "accumulator full" mbarrier of one of two TMEM
//               accumulators (2 x 256 of the 512 columns);
//   warps 8-15  epilogue (two per TMEM lane quarter, each half of the
//               tile's rows): TMEM -> registers, W -= D, releasing the
//               accumulator, so that one tile's epilogue overlaps the next
//               tile's MMAs; meanwhile the next tile's rows of W are bulk-
//               prefetched into L2.
// Every mbarrier wait is bounded; on expiry the kernel raises the device error
// word, the other roles leave their loops, the MMA thread waits (bounded) for
// its MMAs in flight and the TMEM is freed.
#include <cstring>
#include "ggf_ctx.h"
#include "ggf_flush_layout.cuh"

namespace {

// Pipeline depths (compile-time; shared memory: STAGES x 40 KB + RAWS x 16 KB
// + 1 KB must stay within the 227 KB per CTA).
#ifndef GGF_FLUSH_STAGES
#define GGF_FLUSH_STAGES 3
#endif
#ifndef GGF_FLUSH_PD
#define GGF_FLUSH_PD 3
#endif
// Epilogue of the pre-split flush's real tiles: 1 = the W rows of the next
// 16-row chunk are loaded before the current chunk is drained (two chunks of
// loads in flight).  The per-tile flush (96 registers) never does this.
#ifndef GGF_FLUSH_EPI_PP
#define GGF_FLUSH_EPI_PP 0
#endif
// the same for complex tiles (16 float2 per chunk: two chunks in flight need
// more registers than 10 warps per SM leave)
#ifndef GGF_FLUSH_EPI_PP_C
#define GGF_FLUSH_EPI_PP_C 0
#endif
// 1: the lo part of the operand split is rounded to TF32 (else the MMA drops
// its low 13 bits)
#ifndef GGF_SPLIT_LO_RNA
#define GGF_SPLIT_LO_RNA 0
#endif
#ifndef GGF_FLUSH_PS_STAGES
#define GGF_FLUSH_PS_STAGES 5
#endif
constexpr int STAGES = GGF_FLUSH_STAGES;      // split (MMA operand) stages
constexpr int PD = GGF_FLUSH_PD;              // stages of loads in flight ahead
constexpr int RAWS = PD + 1;                  // raw cp.async slots
constexpr int NPROD = 8, NEPI = 8;            // producer and epilogue warps (+ one MMA warp)
constexpr int EPI_PARTS = NEPI / 4;           // epilogue warps per TMEM lane quarter (row groups of a tile)
constexpr int PGROUP = NPROD * 32;
constexpr int TC_THREADS = (NPROD + NEPI + 1) * 32;
constexpr int MMA_WARP = NPROD + NEPI;
constexpr int PLANE_A = 128 * KC * 4;         // 4 KB: 128 rows x 8 tf32
// stage: real    A hi, A lo, B hi, B lo (256 rows)                      24 KB
//        complex Ar hi, Ar lo, Ai hi, Ai lo, Bc hi, Bc lo (384 rows)   40 KB
__host__ __device__ constexpr int stage_bytes(bool cplx) { return cplx ? 4 * PLANE_A + 2 * 384 * KC * 4 : 2 * PLANE_A + 2 * 256 * KC * 4; }
// raw slot: one stage's operands as float4 copies (complex 1024, real 768),
// copy t of producer thread x at position t * PGROUP + x
constexpr int RAW_BYTES = 8 * 128 * 16;
// both variants reserve the complex size, so exactly one CTA fits on an SM
// (the CTA allocates all 512 TMEM columns)
__host__ __device__ constexpr int smem_bytes(bool) { return STAGES * stage_bytes(true) + RAWS * RAW_BYTES + 1024; }
static_assert(STAGES * stage_bytes(true) + RAWS * RAW_BYTES + 1024 <= 227 * 1024, "flush pipeline exceeds shared memory");

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
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
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t dt, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dt),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
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

__device__ __forceinline__ void mbar_arrive(uint32_t addr) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(addr) : "memory");
}

// Wait for the phase with the given parity; false after about two seconds or
// once another role has given up.
__device__ bool mbar_wait_bounded(uint32_t addr, uint32_t phase, volatile int* fail) {
    long long t0 = clock64();
    unsigned it = 0;
    while (!mbar_try(addr, phase)) {
        if ((++it & 31u) == 0) {
            if (*fail) return false;
            if (clock64() - t0 > (1LL << 32)) return false;
        }
    }
    return true;
}

__device__ __forceinline__ void raise_fail(volatile int* fail, int* err) {
    *fail = 1;
    atomicExch(err, 1);
}

struct TileInfo {
    int c, p, i0, j0, K;
};

__device__ __forceinline__ void prefetch_l2(const void* ptr, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(ptr), "r"(bytes) : "memory");
}

// Bulk L2 prefetch of row e of tile t's block of W (the columns j0 .. j0 + 127
// of that row, one contiguous segment).  The bulk copy needs a 16-byte
// aligned start and a length that is a multiple of 16 bytes; rows of other
// widths (possible only in the self-test) are not prefetched.
template <int ROWS, bool CPLX>
__device__ __forceinline__ void prefetch_tile_row(const TileInfo& t, const float* W, int fam_pairs, int N, int rowW,
                                                  int e) {
    const int i = t.i0 + e;
    if (e >= ROWS || i >= N) return;
    const int ncol = min(128, N - t.j0);
    if ((rowW & 3) || ((ncol * (CPLX ? 8 : 4)) & 15)) return;
    const float* ptr = W + ((size_t)t.c * fam_pairs + t.p) * (size_t)N * rowW + (size_t)i * rowW + (CPLX ? 2 : 1) * t.j0;
    prefetch_l2(ptr, (uint32_t)ncol * (CPLX ? 8u : 4u));
}

template <int ROWS>
__device__ __forceinline__ TileInfo decode_tile(long long tile, int tiles_i, int tiles_j, int fam_pairs,
                                                const int* pend, int R, int upper) {
    TileInfo t;
    long long rest = tile;
    const int tj = (int)(rest % tiles_j);
    rest /= tiles_j;
    const int ti = (int)(rest % tiles_i);
    rest /= tiles_i;
    t.p = (int)(rest % fam_pairs);
    t.c = (int)(rest / fam_pairs);
    t.i0 = ti * ROWS;
    t.j0 = tj * 128;
    // upper != 0: tiles strictly below the diagonal are skipped (no work)
    t.K = (upper && t.i0 > t.j0 + 127) ? 0 : pend[t.c] * R;
    return t;
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, uint32_t src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

// Copies of one plane's rows row0 .. row0 + NR - 1, rank columns k0 .. k0 + 7
// into raw slot positions slot0 .. (float4 units, this thread's only).  Rows
// or columns outside the matrix are zero-filled (source size 0, source
// address clamped to the plane's start).
template <int NR>
__device__ __forceinline__ void copy_plane(const float* src, int NP, int row0, int N, int k0, int K, uint32_t raw,
                                           int slot0) {
    constexpr int PER = NR * 2 / PGROUP;
#pragma unroll
    for (int t = 0; t < PER; ++t) {
        int row, kq;
        stage_elem((int)threadIdx.x + t * PGROUP, row, kq);
        const int gr = row0 + row, k = k0 + kq;
        const bool in = gr < N && k < K;
        const float* p = in ? src + pidx(gr, k, NP) : src;
        cp_async16(raw + (uint32_t)((slot0 + t) * PGROUP + threadIdx.x) * 16u, p, in ? 16u : 0u);
    }
}

template <bool CPLX>
__device__ __forceinline__ void copy_stage(const float* Pan, size_t NK, int fam_pairs, int NP, int N,
                                           const TileInfo& t, int k0, uint32_t raw) {
    const size_t blk = ((size_t)t.c * fam_pairs + t.p) * (CPLX ? 4 : 2) * NK;
    const float* U0 = Pan + blk;                         // U (re)
    const float* V0 = Pan + blk + (CPLX ? 2 : 1) * NK;   // V^T (re)
    constexpr int S1 = 256 / PGROUP;   // float4 slots per thread of a 128-row plane
    if (!CPLX) {
        copy_plane<128>(V0, NP, t.j0, N, k0, t.K, raw, 0);
        copy_plane<256>(U0, NP, t.i0, N, k0, t.K, raw, S1);
    } else {
        copy_plane<128>(V0, NP, t.j0, N, k0, t.K, raw, 0);
        copy_plane<128>(V0 + NK, NP, t.j0, N, k0, t.K, raw, S1);
        copy_plane<128>(U0, NP, t.i0, N, k0, t.K, raw, 2 * S1);
        copy_plane<128>(U0 + NK, NP, t.i0, N, k0, t.K, raw, 3 * S1);
    }
}

// Split this thread's raw values of one plane into tf32 hi/lo and write them
// at core-matrix row offset dst_row (and negated at dst_row2 when hi2 is given).
template <int NR, bool LO>
__device__ __forceinline__ void split_plane(const unsigned char* raw, int slot0, unsigned char* hi, unsigned char* lo,
                                            int dst_row, unsigned char* hi2 = nullptr, unsigned char* lo2 = nullptr,
                                            int dst_row2 = 0) {
    constexpr int PER = NR * 2 / PGROUP;
#pragma unroll
    for (int t = 0; t < PER; ++t) {
        int row, kq;
        stage_elem((int)threadIdx.x + t * PGROUP, row, kq);
        const float4 x = *(const float4*)(raw + ((slot0 + t) * PGROUP + threadIdx.x) * 16);
        const float4 h = make_float4(tf32_hi(x.x), tf32_hi(x.y), tf32_hi(x.z), tf32_hi(x.w));
        const float4 l = make_float4(x.x - h.x, x.y - h.y, x.z - h.z, x.w - h.w);
        const uint32_t o = cm_off(dst_row + row, kq);
        *(float4*)(hi + o) = h;
        if (LO) *(float4*)(lo + o) = l;
        if (hi2) {
            const uint32_t o2 = cm_off(dst_row2 + row, kq);
            *(float4*)(hi2 + o2) = make_float4(-h.x, -h.y, -h.z, -h.w);
            if (LO) *(float4*)(lo2 + o2) = make_float4(-l.x, -l.y, -l.z, -l.w);
        }
    }
}

// LO = false: the hi planes only (one TF32 product per term), for Newton
// corrections small enough that the tf32 rounding of the operands is far below
// the FP32 rounding of W.
template <bool CPLX, bool LO>
__device__ __forceinline__ void split_stage(const unsigned char* raw, unsigned char* sb) {
    constexpr int S1 = 256 / PGROUP;   // float4 slots per thread of a 128-row plane
    if (!CPLX) {
        split_plane<128, LO>(raw, 0, sb, sb + PLANE_A, 0);
        split_plane<256, LO>(raw, S1, sb + 2 * PLANE_A, sb + 2 * PLANE_A + 256 * KC * 4, 0);
    } else {
        unsigned char* bh = sb + 4 * PLANE_A;
        unsigned char* bl = bh + 384 * KC * 4;
        split_plane<128, LO>(raw, 0, sb, sb + PLANE_A, 0);                        // V_r
        split_plane<128, LO>(raw, S1, sb + 2 * PLANE_A, sb + 3 * PLANE_A, 0);     // V_i
        split_plane<128, LO>(raw, 2 * S1, bh, bl, 128);                           // U_r
        split_plane<128, LO>(raw, 3 * S1, bh, bl, 256, bh, bl, 0);                // U_i and -U_i
    }
}

// Iterator over this CTA's stages: (tile, rank chunk) pairs with work.
struct StageIter {
    long long tile;
    TileInfo t;
    int k0;
};

template <int ROWS>
__device__ __forceinline__ void stage_first(StageIter& it, long long total, int tiles_i, int tiles_j, int fam_pairs,
                                            const int* pend, int R, int upper) {
    it.k0 = 0;
    for (it.tile = blockIdx.x; it.tile < total; it.tile += gridDim.x) {
        it.t = decode_tile<ROWS>(it.tile, tiles_i, tiles_j, fam_pairs, pend, R, upper);
        if (it.t.K > 0) return;
    }
}

template <int ROWS>
__device__ __forceinline__ void stage_next(StageIter& it, long long total, int tiles_i, int tiles_j, int fam_pairs,
                                           const int* pend, int R, int upper) {
    if (it.tile >= total) return;
    it.k0 += KC;
    if (it.k0 < it.t.K) return;
    it.k0 = 0;
    for (it.tile += gridDim.x; it.tile < total; it.tile += gridDim.x) {
        it.t = decode_tile<ROWS>(it.tile, tiles_i, tiles_j, fam_pairs, pend, R, upper);
        if (it.t.K > 0) return;
    }
}

// Epilogue of one CTA, run by its NEPI epilogue warps (ew = 0 .. NEPI - 1,
// warp = the CTA warp index, whose value mod 4 is the TMEM lane quarter the
// warp may read): for each of the CTA's tiles, wait for its accumulator, W -= D
// from TMEM, and release the accumulator to the MMA thread.
template <bool CPLX, bool PP>
__device__ __forceinline__ void epilogue_tiles(int warp, int ew, int lane, long long total, int tiles_i, int tiles_j,
                                               int fam_pairs, const int* pend, int R, int upper, int N, float* W,
                                               uint32_t tbase, uint64_t* bar_accf, uint64_t* bar_acce,
                                               volatile int& s_fail, int* err) {
    constexpr int ROWS = CPLX ? 128 : 256;        // W rows per tile
    const int rowW = CPLX ? 2 * N : N;            // floats per W row
    const int q = warp & 3;                 // TMEM lane quarter this warp may access
    const int half = ew >> 2;               // which row group of the tile
    int b = 0;
    uint32_t ph = 0;
    // While a tile is drained, its successor's rows of W are prefetched into
    // L2 (one row per epilogue thread), so that the epilogue's loads, which
    // registers limit to 16 per thread in flight, hit L2 instead of DRAM.
    const int e_row = ew * 32 + lane;
    bool first = true;
    for (long long tile = blockIdx.x; tile < total && !s_fail; tile += gridDim.x) {
        const TileInfo t = decode_tile<ROWS>(tile, tiles_i, tiles_j, fam_pairs, pend, R, upper);
        if (t.K == 0) continue;
        if (first) {
            prefetch_tile_row<ROWS, CPLX>(t, W, fam_pairs, N, rowW, e_row);
            first = false;
        }
        for (long long tn = tile + gridDim.x; tn < total; tn += gridDim.x) {
            const TileInfo u = decode_tile<ROWS>(tn, tiles_i, tiles_j, fam_pairs, pend, R, upper);
            if (u.K == 0) continue;
            prefetch_tile_row<ROWS, CPLX>(u, W, fam_pairs, N, rowW, e_row);
            break;
        }
        if (!mbar_wait_bounded(smem_u32(&bar_accf[b]), ph, &s_fail)) { raise_fail(&s_fail, err); break; }
        asm volatile("tcgen05.fence::after_thread_sync;");
        const int j = t.j0 + q * 32 + lane;
        float* Wp = W + ((size_t)t.c * fam_pairs + t.p) * (size_t)N * rowW;
        const uint32_t tl = tbase + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * 256);
        if (!CPLX) {
            // rows i0 + half*RG + 16 cb + k  <->  TMEM column half*RG + 16 cb + k (RG = 256 / EPI_PARTS)
            constexpr int NCB = 256 / EPI_PARTS / 16;
            auto load_w = [&](int cb, float* w) {
                const int ib = t.i0 + half * (256 / EPI_PARTS) + cb * 16;
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    const int i = ib + k;
                    w[k] = (i < N && j < N) ? Wp[(size_t)i * N + j] : 0.f;
                }
            };
            auto drain = [&](int cb, const float* w) {
                uint32_t v[16];
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
                    "%15}, [%16];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                      "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                      "=r"(v[14]), "=r"(v[15])
                    : "r"(tl + half * (256 / EPI_PARTS) + cb * 16));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                const int ib = t.i0 + half * (256 / EPI_PARTS) + cb * 16;
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    const int i = ib + k;
                    if (i < N && j < N) Wp[(size_t)i * N + j] = w[k] - __uint_as_float(v[k]);
                }
            };
            if (PP) {
                float wa[16], wb[16];
                load_w(0, wa);
#pragma unroll 1
                for (int cb = 0; cb < NCB; cb += 2) {
                    load_w(cb + 1, wb);
                    drain(cb, wa);
                    if (cb + 2 < NCB) load_w(cb + 2, wa);
                    drain(cb + 1, wb);
                }
            } else {
#pragma unroll 1
                for (int cb = 0; cb < NCB; ++cb) {
                    float w[16];
                    load_w(cb, w);
                    drain(cb, w);
                }
            }
        } else {
            // rows i0 + half*RG + 16 cb + k  <->  re column half*RG + 16 cb + k, im column + 128
            // (RG = 128 / EPI_PARTS)
            constexpr int NCBC = 128 / EPI_PARTS / 16;
            auto load_wc = [&](int cb, float2* w) {
                const int ib = t.i0 + half * (128 / EPI_PARTS) + cb * 16;
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    const int i = ib + k;
                    w[k] = (i < N && j < N) ? *(const float2*)(Wp + (size_t)i * rowW + 2 * j) : make_float2(0.f, 0.f);
                }
            };
            auto drain_c = [&](int cb, const float2* w) {
                uint32_t v[16], vi[16];
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
                    "%15}, [%16];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                      "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                      "=r"(v[14]), "=r"(v[15])
                    : "r"(tl + half * (128 / EPI_PARTS) + cb * 16));
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
                    "%15}, [%16];"
                    : "=r"(vi[0]), "=r"(vi[1]), "=r"(vi[2]), "=r"(vi[3]), "=r"(vi[4]), "=r"(vi[5]), "=r"(vi[6]),
                      "=r"(vi[7]), "=r"(vi[8]), "=r"(vi[9]), "=r"(vi[10]), "=r"(vi[11]), "=r"(vi[12]),
                      "=r"(vi[13]), "=r"(vi[14]), "=r"(vi[15])
                    : "r"(tl + 128 + half * (128 / EPI_PARTS) + cb * 16));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                const int ib = t.i0 + half * (128 / EPI_PARTS) + cb * 16;
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    const int i = ib + k;
                    if (i < N && j < N)
                        *(float2*)(Wp + (size_t)i * rowW + 2 * j) =
                            make_float2(w[k].x - __uint_as_float(v[k]), w[k].y - __uint_as_float(vi[k]));
                }
            };
            if (PP && GGF_FLUSH_EPI_PP_C) {
                static_assert(NCBC % 2 == 0, "ping-pong epilogue drains chunk pairs");
                float2 wa[16], wb[16];
                load_wc(0, wa);
#pragma unroll 1
                for (int cb = 0; cb < NCBC; cb += 2) {
                    load_wc(cb + 1, wb);
                    drain_c(cb, wa);
                    if (cb + 2 < NCBC) load_wc(cb + 2, wa);
                    drain_c(cb + 1, wb);
                }
            } else {
#pragma unroll 1
                for (int cb = 0; cb < NCBC; ++cb) {
                    float2 w[16];
                    load_wc(cb, w);
                    drain_c(cb, w);
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        mbar_arrive(smem_u32(&bar_acce[b]));
        b ^= 1;
        if (b == 0) ph ^= 1u;
    }
}

// MMA issuer of one CTA (one thread): for each tile, wait for a free
// accumulator, then for each rank chunk wait for its stage (NST stages in a
// ring, SB bytes apart from base), issue the TF32 MMAs and commit them to the
// stage's "empty" barrier; after the tile's last chunk commit to the
// accumulator's "full" barrier.  Before returning, waits (bounded) for every
// issued MMA, so that the TMEM can be released.
template <bool CPLX, int TERMS, int NST>
__device__ __forceinline__ void mma_tiles(long long total, int tiles_i, int tiles_j, int fam_pairs, const int* pend,
                                          int R, int upper, uint32_t tbase, unsigned char* base, uint64_t* bar_full,
                                          uint64_t* bar_empty, uint64_t* bar_accf, uint64_t* bar_acce,
                                          uint64_t* bar_done_p, volatile int& s_fail, int* err) {
    constexpr int ROWS = CPLX ? 128 : 256;
    constexpr int SB = stage_bytes(CPLX);
    uint64_t& bar_done = *bar_done_p;
    int st = 0, b = 0;
    uint32_t ph = 0, bph = 0;
    constexpr uint32_t id = idesc_tf32(128, 256);
    for (long long tile = blockIdx.x; tile < total && !s_fail; tile += gridDim.x) {
        const TileInfo t = decode_tile<ROWS>(tile, tiles_i, tiles_j, fam_pairs, pend, R, upper);
        if (t.K == 0) continue;
        if (!mbar_wait_bounded(smem_u32(&bar_acce[b]), bph ^ 1u, &s_fail)) { raise_fail(&s_fail, err); break; }
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t d = tbase + (uint32_t)(b * 256);
        bool ok = true;
        for (int k0 = 0; k0 < t.K; k0 += KC) {
            if (!mbar_wait_bounded(smem_u32(&bar_full[st]), ph, &s_fail)) { ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t sb = smem_u32(base + st * SB);
            const uint32_t first = k0 == 0 ? 0u : 1u;
            if (!CPLX) {
                const uint32_t ah = sb, al = sb + PLANE_A, bh = sb + 2 * PLANE_A, bl = bh + 256 * KC * 4;
                mma_tf32(d, smem_desc(ah), smem_desc(bh), id, first);
                if (TERMS == 3) {
                    mma_tf32(d, smem_desc(ah), smem_desc(bl), id, 1u);
                    mma_tf32(d, smem_desc(al), smem_desc(bh), id, 1u);
                }
            } else {
                const uint32_t arh = sb, arl = sb + PLANE_A, aih = sb + 2 * PLANE_A, ail = sb + 3 * PLANE_A;
                const uint32_t bh = sb + 4 * PLANE_A, bl = bh + 384 * KC * 4;
                const uint32_t o1 = (128 / 8) * SBO;    // rows 128..383: [U_r ; U_i]
                // rows 0..255: [-U_i ; U_r]
                mma_tf32(d, smem_desc(arh), smem_desc(bh + o1), id, first);
                if (TERMS == 3) {
                    mma_tf32(d, smem_desc(arh), smem_desc(bl + o1), id, 1u);
                    mma_tf32(d, smem_desc(arl), smem_desc(bh + o1), id, 1u);
                }
                mma_tf32(d, smem_desc(aih), smem_desc(bh), id, 1u);
                if (TERMS == 3) {
                    mma_tf32(d, smem_desc(aih), smem_desc(bl), id, 1u);
                    mma_tf32(d, smem_desc(ail), smem_desc(bh), id, 1u);
                }
            }
            mma_commit(smem_u32(&bar_empty[st]));
            if (++st == NST) { st = 0; ph ^= 1u; }
        }
        if (!ok) { raise_fail(&s_fail, err); break; }
        mma_commit(smem_u32(&bar_accf[b]));
        b ^= 1;
        if (b == 0) bph ^= 1u;
    }
    // every issued MMA completes before the TMEM is released
    mma_commit(smem_u32(&bar_done));
    volatile int never = 0;
    if (!mbar_wait_bounded(smem_u32(&bar_done), 0u, &never)) atomicExch(err, 1);
}

// TERMS = 3: FP32-accurate TF32 split; TERMS = 1: one TF32 product.
template <bool CPLX, int TERMS>
__global__ void __launch_bounds__(TC_THREADS, 1)
flush_tc_kernel(int N, int fam_pairs, int n_chains, float* W, const float* Pan, const int* pend, int R, int KRM,
                int upper, int* err) {
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) uint64_t bar_full[STAGES], bar_empty[STAGES], bar_accf[2], bar_acce[2], bar_done;
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int s_fail;
    // an earlier bounded wait of this context ran out: do nothing (the host
    // reports GGF_ETIMEOUT after the sweep)
    if (*(volatile int*)err) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int ROWS = CPLX ? 128 : 256;        // W rows per tile
    constexpr int SB = stage_bytes(CPLX);
    const int tiles_i = (N + ROWS - 1) / ROWS, tiles_j = (N + 127) / 128;
    const size_t NK = panel_plane(N, KRM);
    const int NP = panel_rows(N);
    const long long total = (long long)n_chains * fam_pairs * tiles_i * tiles_j;
    unsigned char* base = (unsigned char*)(((uintptr_t)sm + 1023) & ~(uintptr_t)1023);

    if (warp == MMA_WARP) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bar_full[s])), "r"(NPROD * 32));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_empty[s])));
        }
        for (int b = 0; b < 2; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_accf[b])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bar_acce[b])), "r"(NEPI * 32));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_done)));
        asm volatile("fence.mbarrier_init.release.cluster;");
        s_fail = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tbase = tmem_slot;

    if (warp < NPROD) {
        // ---- producers ----
        // Stage s's copies are issued PD stages before it is split; every
        // stage (even a missing one past the end) commits one cp.async group,
        // so "wait_group PD" leaves exactly stage s's copies complete.
        unsigned char* raw = base + STAGES * SB;
        const uint32_t raw_u = smem_u32(raw);
        StageIter ahead, cur;
        stage_first<ROWS>(ahead, total, tiles_i, tiles_j, fam_pairs, pend, R, upper);
        cur = ahead;
        for (int d = 0; d < PD; ++d) {
            if (ahead.tile < total)
                copy_stage<CPLX>(Pan, NK, fam_pairs, NP, N, ahead.t, ahead.k0, raw_u + (uint32_t)(d % RAWS) * RAW_BYTES);
            cp_async_commit();
            stage_next<ROWS>(ahead, total, tiles_i, tiles_j, fam_pairs, pend, R, upper);
        }
        int st = 0;
        uint32_t ph = 0;
        for (long long sidx = 0; cur.tile < total && !s_fail; ++sidx) {
            if (ahead.tile < total)
                copy_stage<CPLX>(Pan, NK, fam_pairs, NP, N, ahead.t, ahead.k0,
                                 raw_u + (uint32_t)((sidx + PD) % RAWS) * RAW_BYTES);
            cp_async_commit();
            stage_next<ROWS>(ahead, total, tiles_i, tiles_j, fam_pairs, pend, R, upper);
            asm volatile("cp.async.wait_group %0;" ::"n"(PD) : "memory");
            if (!mbar_wait_bounded(smem_u32(&bar_empty[st]), ph ^ 1u, &s_fail)) { raise_fail(&s_fail, err); break; }
            split_stage<CPLX, TERMS == 3>(raw + (size_t)(sidx % RAWS) * RAW_BYTES, base + st * SB);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(smem_u32(&bar_full[st]));
            if (++st == STAGES) { st = 0; ph ^= 1u; }
            stage_next<ROWS>(cur, total, tiles_i, tiles_j, fam_pairs, pend, R, upper);
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
    } else if (warp < MMA_WARP) {
        epilogue_tiles<CPLX, false>(warp, warp - NPROD, lane, total, tiles_i, tiles_j, fam_pairs, pend, R, upper, N, W, tbase,
                             bar_accf, bar_acce, s_fail, err);
    } else if (lane == 0) {
        mma_tiles<CPLX, TERMS, STAGES>(total, tiles_i, tiles_j, fam_pairs, pend, R, upper, tbase, base, bar_full,
                                       bar_empty, bar_accf, bar_acce, &bar_done, s_fail, err);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == MMA_WARP) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(512));
    }
}

// ---- flush from pre-split operands (waves of chains) -------------------------
//
// The sweep's flushes run chain wave by chain wave: ps_split_kernel splits the
// wave's panels once into tf32 hi/lo blocks laid out as stage parts
// (ggf_flush_layout.cuh), then flush_ps_kernel fills each stage with two bulk
// copies (cp.async.bulk, completing on the stage's mbarrier) issued by one
// thread, instead of eight producer warps copying and splitting the same
// operands once per tile.  The MMA issuer and the epilogue are those of
// flush_tc_kernel; with the producer warps gone, the CTA is 8 epilogue warps
// (0-7), one copy warp (8) and one MMA warp (9), and holds PS_STAGES stages.
constexpr int PS_STAGES = GGF_FLUSH_PS_STAGES;
constexpr int PS_COPY_WARP = NEPI, PS_MMA_WARP = NEPI + 1;
constexpr int PS_THREADS = (NEPI + 2) * 32;
__host__ __device__ constexpr int ps_smem_bytes() { return PS_STAGES * stage_bytes(true) + 1024; }
static_assert(PS_STAGES * stage_bytes(true) + 1024 <= 227 * 1024, "pre-split flush stages exceed shared memory");
static_assert(ps_vbytes(false) + ps_ubytes(false) == stage_bytes(false) &&
                  ps_vbytes(true) + ps_ubytes(true) == stage_bytes(true),
              "pre-split blocks must fill a stage exactly");

__device__ __forceinline__ void bulk_to_smem(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// Split the panels of chains c0 .. c0 + n - 1 (all pairs of one family) into
// the wave's pre-split blocks.  One thread per (chain, pair, row, 4 rank
// columns), the 4-column group fastest, so that reads of the chunk-major panel
// and writes of the core-matrix blocks are both contiguous across a warp.
// Only the rank chunks below the chain's pending rank are written (the flush
// reads no others); inside them, rows past N and columns past the rank are 0.
template <bool CPLX>
__global__ void __launch_bounds__(256) ps_split_kernel(int N, int fam_pairs, int c0, int n, const float* Pan,
                                                       const int* pend, int R, int KRM, unsigned char* ps) {
    const size_t NK = panel_plane(N, KRM);
    const int NP = panel_rows(N);
    const int nq = panel_cols(KRM) / 4;
    const long long total = (long long)n * fam_pairs * NP * nq;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int q = (int)(e % nq);
        long long rest = e / nq;
        const int row = (int)(rest % NP);
        rest /= NP;
        const int p = (int)(rest % fam_pairs);
        const int cw = (int)(rest / fam_pairs);
        const int K = pend[c0 + cw] * R;
        const int k = 4 * q;
        if (k >= ((K + KC - 1) / KC) * KC) continue;
        const size_t blk = ((size_t)(c0 + cw) * fam_pairs + p) * (CPLX ? 4 : 2) * NK;
        auto load = [&](const float* plane) {
            float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
            if (row < N) x = *(const float4*)(plane + pidx(row, k, NP));
            if (k + 0 >= K) x.x = 0.f;
            if (k + 1 >= K) x.y = 0.f;
            if (k + 2 >= K) x.z = 0.f;
            if (k + 3 >= K) x.w = 0.f;
            return x;
        };
        auto put = [&](size_t hi, size_t lo, float4 x, float sgn) {
            const float4 h = make_float4(tf32_hi(x.x), tf32_hi(x.y), tf32_hi(x.z), tf32_hi(x.w));
            float4 l = make_float4(x.x - h.x, x.y - h.y, x.z - h.z, x.w - h.w);
            if (GGF_SPLIT_LO_RNA) l = make_float4(tf32_hi(l.x), tf32_hi(l.y), tf32_hi(l.z), tf32_hi(l.w));
            *(float4*)(ps + hi) = make_float4(sgn * h.x, sgn * h.y, sgn * h.z, sgn * h.w);
            *(float4*)(ps + lo) = make_float4(sgn * l.x, sgn * l.y, sgn * l.z, sgn * l.w);
        };
        const float* U0 = Pan + blk;
        const float* V0 = Pan + blk + (CPLX ? 2 : 1) * NK;
        size_t hi, lo, hi2, lo2;
        ps_vdst(CPLX, N, KRM, fam_pairs, cw, p, 0, row, k, hi, lo);
        put(hi, lo, load(V0), 1.f);
        ps_udst(CPLX, N, KRM, fam_pairs, n, cw, p, 0, row, k, hi, lo, hi2, lo2);
        put(hi, lo, load(U0), 1.f);
        if (CPLX) {
            ps_vdst(CPLX, N, KRM, fam_pairs, cw, p, 1, row, k, hi, lo);
            put(hi, lo, load(V0 + NK), 1.f);
            const float4 ui = load(U0 + NK);
            ps_udst(CPLX, N, KRM, fam_pairs, n, cw, p, 1, row, k, hi, lo, hi2, lo2);
            put(hi, lo, ui, 1.f);
            put(hi2, lo2, ui, -1.f);
        }
    }
}

// W -= U V for chains 0 .. n_chains - 1 of W and pend (the caller offsets
// them to the wave), operands from the wave's pre-split blocks ps.
template <bool CPLX, int TERMS>
__global__ void __launch_bounds__(PS_THREADS, 1)
flush_ps_kernel(int N, int fam_pairs, int n_chains, float* W, const unsigned char* ps, const int* pend, int R, int KRM,
                int* err) {
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) uint64_t bar_full[PS_STAGES], bar_empty[PS_STAGES], bar_accf[2], bar_acce[2], bar_done;
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int s_fail;
    if (*(volatile int*)err) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int ROWS = CPLX ? 128 : 256;
    constexpr int SB = stage_bytes(CPLX);
    constexpr uint32_t VB = ps_vbytes(CPLX), UB = ps_ubytes(CPLX);
    const int tiles_i = (N + ROWS - 1) / ROWS, tiles_j = (N + 127) / 128;
    const long long total = (long long)n_chains * fam_pairs * tiles_i * tiles_j;
    unsigned char* base = (unsigned char*)(((uintptr_t)sm + 1023) & ~(uintptr_t)1023);

    if (warp == PS_MMA_WARP) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < PS_STAGES; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_full[s])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_empty[s])));
        }
        for (int b = 0; b < 2; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_accf[b])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bar_acce[b])), "r"(NEPI * 32));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_done)));
        asm volatile("fence.mbarrier_init.release.cluster;");
        s_fail = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tbase = tmem_slot;

    if (warp < NEPI) {
        epilogue_tiles<CPLX, GGF_FLUSH_EPI_PP != 0>(warp, warp, lane, total, tiles_i, tiles_j, fam_pairs, pend, R, 0, N, W, tbase, bar_accf,
                             bar_acce, s_fail, err);
    } else if (warp == PS_COPY_WARP) {
        if (lane == 0) {
            // one stage = the V block of the tile's columns and the U block of
            // its rows for one rank chunk, two bulk copies
            StageIter it;
            stage_first<ROWS>(it, total, tiles_i, tiles_j, fam_pairs, pend, R, 0);
            int st = 0;
            uint32_t ph = 0;
            long long issued = 0;
            while (it.tile < total && !s_fail) {
                if (!mbar_wait_bounded(smem_u32(&bar_empty[st]), ph ^ 1u, &s_fail)) { raise_fail(&s_fail, err); break; }
                const int kc = it.k0 / KC;
                const unsigned char* vsrc = ps + ps_voff(CPLX, N, KRM, fam_pairs, it.t.c, it.t.p, it.t.j0 / 128, kc);
                const unsigned char* usrc =
                    ps + ps_uoff(CPLX, N, KRM, fam_pairs, n_chains, it.t.c, it.t.p, it.t.i0 / ROWS, kc);
                const uint32_t sb = smem_u32(base + st * SB), bar = smem_u32(&bar_full[st]);
                if (TERMS == 3) {
                    mbar_expect_tx(bar, VB + UB);
                    bulk_to_smem(sb, vsrc, VB, bar);
                    bulk_to_smem(sb + VB, usrc, UB, bar);
                } else {
                    // one product: the hi planes only (V hi at the start of
                    // each plane pair, U hi the first half of its block)
                    mbar_expect_tx(bar, VB / 2 + UB / 2);
                    bulk_to_smem(sb, vsrc, PS_PLANE, bar);
                    if (CPLX) bulk_to_smem(sb + 2 * PS_PLANE, vsrc + 2 * PS_PLANE, PS_PLANE, bar);
                    bulk_to_smem(sb + VB, usrc, UB / 2, bar);
                }
                ++issued;
                if (++st == PS_STAGES) { st = 0; ph ^= 1u; }
                stage_next<ROWS>(it, total, tiles_i, tiles_j, fam_pairs, pend, R, 0);
            }
            // the copies of the last stages issued have landed before the CTA
            // exits, also when another role gave up
            for (long long i = issued > PS_STAGES ? issued - PS_STAGES : 0; i < issued; ++i) {
                volatile int never = 0;
                if (!mbar_wait_bounded(smem_u32(&bar_full[i % PS_STAGES]), (uint32_t)((i / PS_STAGES) & 1), &never))
                    atomicExch(err, 1);
            }
        }
    } else if (lane == 0) {
        mma_tiles<CPLX, TERMS, PS_STAGES>(total, tiles_i, tiles_j, fam_pairs, pend, R, 0, tbase, base, bar_full, bar_empty,
                                      bar_accf, bar_acce, &bar_done, s_fail, err);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == PS_MMA_WARP) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(512));
    }
}

}  // namespace

// Shared-memory attributes of the tensor-core flush, set once per process and
// device ordinal outside any stream capture.
ggf_status ggf_prepare_flush_tc(ggf_ctx* ctx) {
    static bool done[64] = {false};
    if (ctx->device >= 0 && ctx->device < 64 && done[ctx->device]) return GGF_OK;
    GGF_CK(cudaFuncSetAttribute(flush_tc_kernel<true, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes(true)));
    GGF_CK(cudaFuncSetAttribute(flush_tc_kernel<false, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes(false)));
    GGF_CK(cudaFuncSetAttribute(flush_tc_kernel<true, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes(true)));
    GGF_CK(cudaFuncSetAttribute(flush_tc_kernel<false, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes(false)));
    GGF_CK(cudaFuncSetAttribute(flush_ps_kernel<true, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, ps_smem_bytes()));
    GGF_CK(cudaFuncSetAttribute(flush_ps_kernel<false, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, ps_smem_bytes()));
    GGF_CK(cudaFuncSetAttribute(flush_ps_kernel<true, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, ps_smem_bytes()));
    GGF_CK(cudaFuncSetAttribute(flush_ps_kernel<false, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, ps_smem_bytes()));
    if (ctx->device >= 0 && ctx->device < 64) done[ctx->device] = true;
    return GGF_OK;
}

namespace {

ggf_status launch_flush_tc(ggf_ctx* ctx, bool cplx, int N, int fam_pairs, int n_chains, float* W, const float* Pan,
                           const int* pend, int R, int KRM, bool upper, int* err, cudaStream_t st, int terms = 3) {
    if (fam_pairs == 0 || n_chains == 0) return GGF_OK;
    if (KRM < 1) return ggf_fail(ctx, GGF_EINVAL, "tensor-core flush: empty panel");
    const int rows = cplx ? 128 : 256;
    const long long total = (long long)n_chains * fam_pairs * ((N + rows - 1) / rows) * ((N + 127) / 128);
    int sms = ctx->n_sms > 0 ? ctx->n_sms : 152;
    const long long grid = std::min<long long>(total, (long long)sms);
    GGF_TRY(ggf_prepare_flush_tc(ctx));
    const int up = upper ? 1 : 0;
    if (cplx && terms == 1)
        flush_tc_kernel<true, 1><<<(unsigned)grid, TC_THREADS, smem_bytes(true), st>>>(N, fam_pairs, n_chains, W, Pan,
                                                                                       pend, R, KRM, up, err);
    else if (cplx)
        flush_tc_kernel<true, 3><<<(unsigned)grid, TC_THREADS, smem_bytes(true), st>>>(N, fam_pairs, n_chains, W, Pan,
                                                                                       pend, R, KRM, up, err);
    else if (terms == 1)
        flush_tc_kernel<false, 1><<<(unsigned)grid, TC_THREADS, smem_bytes(false), st>>>(N, fam_pairs, n_chains, W, Pan,
                                                                                         pend, R, KRM, up, err);
    else
        flush_tc_kernel<false, 3><<<(unsigned)grid, TC_THREADS, smem_bytes(false), st>>>(N, fam_pairs, n_chains, W, Pan,
                                                                                         pend, R, KRM, up, err);
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
    const size_t NK = panel_plane(N, KRM);
    const int NP = panel_rows(N);
    int i = (int)(e / rowW), f = (int)(e % rowW);
    if (!cplx) {
        double s = 0.0;
        for (int q = 0; q < K; ++q) s += (double)Pan[pidx(i, q, NP)] * (double)Pan[NK + pidx(f, q, NP)];
        ref[e] = (double)W0[e] - s;
    } else {
        int j = f >> 1, part = f & 1;
        double sr = 0.0, si = 0.0;
        for (int q = 0; q < K; ++q) {
            double ur = Pan[pidx(i, q, NP)], ui = Pan[NK + pidx(i, q, NP)];
            double vr = Pan[2 * NK + pidx(j, q, NP)], vi = Pan[3 * NK + pidx(j, q, NP)];
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

// Bytes of pre-split scratch of one rank-N product (the Newton step of the
// refresh) of the larger family.
size_t ggf_flush_ps_newton_bytes(ggf_ctx* ctx) {
    const int N = ctx->g.N;
    return ps_bytes(ctx->Kc > 0, N, N, 1, 1);
}

// Bytes of pre-split scratch per chain (the larger of the two families).
size_t ggf_flush_ps_chain_bytes(ggf_ctx* ctx, int KRM) {
    const int N = ctx->g.N;
    return std::max(ctx->K ? ps_bytes(false, N, KRM, ctx->K, 1) : 0, ctx->Kc ? ps_bytes(true, N, KRM, ctx->Kc, 1) : 0);
}

namespace {

// One wave (chains c0 .. c0 + n - 1 of W, Pan and pend): split, then flush.
template <bool CPLX, int TERMS = 3>
ggf_status flush_wave(ggf_ctx* ctx, int N, int R, int fam_pairs, int c0, int n, float* W, const float* Pan,
                      const int* pend, int KRM, unsigned char* ps, cudaStream_t st) {
    const int sms = ctx->n_sms > 0 ? ctx->n_sms : 152;
    const long long items = (long long)n * fam_pairs * panel_rows(N) * (panel_cols(KRM) / 4);
    const unsigned sgrid = (unsigned)std::min<long long>((items + 255) / 256, (long long)sms * 8);
    ps_split_kernel<CPLX><<<sgrid, 256, 0, st>>>(N, fam_pairs, c0, n, Pan, pend, R, KRM, ps);
    const int rows = CPLX ? 128 : 256;
    const long long total = (long long)n * fam_pairs * ((N + rows - 1) / rows) * ((N + 127) / 128);
    const size_t wsz = (size_t)N * N * (CPLX ? 2 : 1);
    flush_ps_kernel<CPLX, TERMS><<<(unsigned)std::min<long long>(total, sms), PS_THREADS, ps_smem_bytes(), st>>>(
        N, fam_pairs, n, W + (size_t)c0 * fam_pairs * wsz, ps, pend + c0, R, KRM, ctx->d_err);
    GGF_CK(cudaGetLastError());
    return GGF_OK;
}

}  // namespace

// The sweep's flush of every chain's pending panels: chain waves of
// ch.ps_wave chains, each split once into pre-split blocks and flushed from
// them (two launches per family and wave; the count is added to *launches);
// without a scratch, the per-tile-split kernel over all chains.
ggf_status ggf_flush_tc(ggf_ctx* ctx, cudaStream_t st, int* launches) {
    Chains& ch = ctx->ch;
    const Geometry& g = ctx->g;
    const int KRM = ch.kmax * g.r;
    if (!ch.ps || ch.ps_wave < 1) {
        // no scratch (the chains left no room for one): split per tile
        GGF_TRY(launch_flush_tc(ctx, false, g.N, ctx->K, ch.n, (float*)ch.Wr, (const float*)ch.Pr, ch.pend, g.r, KRM,
                                false, ctx->d_err, st));
        GGF_TRY(launch_flush_tc(ctx, true, g.N, ctx->Kc, ch.n, (float*)ch.Wc, (const float*)ch.Pc, ch.pend, g.r, KRM,
                                false, ctx->d_err, st));
        *launches += 1 + (ctx->Kc ? 1 : 0);
        return GGF_OK;
    }
    for (int c0 = 0; c0 < ch.n; c0 += ch.ps_wave) {
        const int n = std::min(ch.ps_wave, ch.n - c0);
        if (ctx->K) {
            GGF_TRY(flush_wave<false>(ctx, g.N, g.r, ctx->K, c0, n, (float*)ch.Wr, (const float*)ch.Pr, ch.pend, KRM,
                                      ch.ps, st));
            *launches += 2;
        }
        if (ctx->Kc) {
            GGF_TRY(flush_wave<true>(ctx, g.N, g.r, ctx->Kc, c0, n, (float*)ch.Wc, (const float*)ch.Pc, ch.pend, KRM,
                                     ch.ps, st));
            *launches += 2;
        }
    }
    return GGF_OK;
}

// W -= U V for one N x N matrix with rank-K panels (K = pend[0] * R, panel
// column count KRM), terms = 3 (FP32-accurate TF32 split) or 1 (one TF32
// product).  Used by the Newton refinement of the inverses (k_refine.cu).
ggf_status ggf_flush_tc_one(ggf_ctx* ctx, bool cplx, int N, float* W, const float* Pan, const int* pend, int R,
                            int KRM, int terms, cudaStream_t st) {
    // through the chains' pre-split scratch when it holds this product's
    // operands (outside a sweep it is free), else splitting per tile
    const Chains& ch = ctx->ch;
    if (ch.ps && ps_bytes(cplx, N, KRM, 1, 1) <= ch.ps_bytes) {
        GGF_TRY(ggf_prepare_flush_tc(ctx));
        if (cplx) return terms == 1 ? flush_wave<true, 1>(ctx, N, R, 1, 0, 1, W, Pan, pend, KRM, ch.ps, st)
                                    : flush_wave<true, 3>(ctx, N, R, 1, 0, 1, W, Pan, pend, KRM, ch.ps, st);
        return terms == 1 ? flush_wave<false, 1>(ctx, N, R, 1, 0, 1, W, Pan, pend, KRM, ch.ps, st)
                          : flush_wave<false, 3>(ctx, N, R, 1, 0, 1, W, Pan, pend, KRM, ch.ps, st);
    }
    return launch_flush_tc(ctx, cplx, N, 1, 1, W, Pan, pend, R, KRM, false, ctx->d_err, st, terms == 1 ? 1 : 3);
}

extern "C" ggf_status ggf_selftest_flush(ggf_ctx* ctx, int cplx, int N, int rank, double* max_rel_err) {
    if (!ctx || !max_rel_err || N < 1 || N > 8192 || rank < 4 || rank > 512 || rank % 4)
        return ggf_fail(ctx, GGF_EINVAL, "selftest_flush: N in [1, 8192], rank in {4, 8, ..., 512}");
    cudaSetDevice(ctx->device);
    const int R = 4, KRM = rank;
    const int rowW = cplx ? 2 * N : N;
    const size_t NK = panel_plane(N, KRM), nW = (size_t)N * rowW, nP = (cplx ? 4 : 2) * NK;
    float *W = nullptr, *Pan = nullptr;
    unsigned char* ps = nullptr;
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
        if (ps) cudaFree(ps);
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
    // both flush kernels on the same input: the one that splits operands per
    // tile, and the pre-split one (split pass + bulk-copy stages)
    double worst = 0.0;
    for (int pass = 0; pass < 2 && rc == GGF_OK; ++pass) {
        cudaMemset(mx, 0, 16);
        st_fill<<<(unsigned)((nW + 255) / 256), 256>>>(W, nW, 1, 1.0f);
        if (pass == 0) {
            rc = launch_flush_tc(ctx, cplx != 0, N, 1, 1, W, Pan, pend, R, KRM, false, ctx->d_err, 0);
        } else {
            if ((rc = ggf_prepare_flush_tc(ctx)) != GGF_OK) break;
            if (cudaMalloc(&ps, ps_bytes(cplx != 0, N, KRM, 1, 1)) != cudaSuccess) {
                rc = ggf_fail(ctx, GGF_ENOMEM, "selftest_flush allocation failed");
                break;
            }
            rc = cplx ? flush_wave<true>(ctx, N, R, 1, 0, 1, W, Pan, pend, KRM, ps, 0)
                      : flush_wave<false>(ctx, N, R, 1, 0, 1, W, Pan, pend, KRM, ps, 0);
        }
        if (rc != GGF_OK) break;
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
            worst = std::max(worst, d / (m > 0 ? m : 1.0));
        }
    }
    if (rc == GGF_OK) *max_rel_err = worst;
    cleanup();
    return rc;
}

// The self-test's seeded case with its data copied to host memory, so that a
// reference independent of the library can be computed: which = 0 runs the
// per-tile-split flush, 1 the pre-split one.
extern "C" ggf_status ggf_selftest_flush_data(ggf_ctx* ctx, int cplx, int N, int rank, int which, float* w0,
                                              float* pan, float* w1) {
    if (!ctx || !w0 || !pan || !w1 || N < 1 || N > 8192 || rank < 4 || rank > 512 || rank % 4 || which < 0 ||
        which > 1)
        return ggf_fail(ctx, GGF_EINVAL, "selftest_flush_data: N in [1, 8192], rank in {4, 8, ..., 512}, which 0 or 1");
    cudaSetDevice(ctx->device);
    const int R = 4, KRM = rank;
    const int rowW = cplx ? 2 * N : N;
    const size_t NK = panel_plane(N, KRM), nW = (size_t)N * rowW, nP = (cplx ? 4 : 2) * NK;
    float *W = nullptr, *Pan = nullptr;
    unsigned char* ps = nullptr;
    int* pend = nullptr;
    ggf_status rc = GGF_OK;
    auto cleanup = [&]() {
        if (W) cudaFree(W);
        if (Pan) cudaFree(Pan);
        if (pend) cudaFree(pend);
        if (ps) cudaFree(ps);
    };
    if (cudaMalloc(&W, nW * 4) != cudaSuccess || cudaMalloc(&Pan, nP * 4) != cudaSuccess ||
        cudaMalloc(&pend, 4) != cudaSuccess ||
        (which == 1 && cudaMalloc(&ps, ps_bytes(cplx != 0, N, KRM, 1, 1)) != cudaSuccess)) {
        cleanup();
        return ggf_fail(ctx, GGF_ENOMEM, "selftest_flush_data allocation failed");
    }
    const int pv = rank / R;
    cudaMemcpy(pend, &pv, 4, cudaMemcpyHostToDevice);
    st_fill<<<(unsigned)((nW + 255) / 256), 256>>>(W, nW, 1, 1.0f);
    st_fill<<<(unsigned)((nP + 255) / 256), 256>>>(Pan, nP, 2, 0.3f);
    if (cudaMemcpy(w0, W, nW * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(pan, Pan, nP * 4, cudaMemcpyDeviceToHost) != cudaSuccess) {
        rc = ggf_cuda(ctx, cudaGetLastError(), "selftest_flush_data");
    } else if ((rc = ggf_prepare_flush_tc(ctx)) == GGF_OK) {
        if (which == 0) rc = launch_flush_tc(ctx, cplx != 0, N, 1, 1, W, Pan, pend, R, KRM, false, ctx->d_err, 0);
        else rc = cplx ? flush_wave<true>(ctx, N, R, 1, 0, 1, W, Pan, pend, KRM, ps, 0)
                       : flush_wave<false>(ctx, N, R, 1, 0, 1, W, Pan, pend, KRM, ps, 0);
        int herr = 0;
        if (rc == GGF_OK) {
            if (cudaMemcpy(w1, W, nW * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
                cudaMemcpy(&herr, ctx->d_err, 4, cudaMemcpyDeviceToHost) != cudaSuccess)
                rc = ggf_cuda(ctx, cudaGetLastError(), "selftest_flush_data");
            else if (herr)
                rc = ggf_fail(ctx, GGF_ETIMEOUT, "tensor-core flush: mbarrier wait ran out");
        }
    }
    cleanup();
    return rc;
}
