// Newton refinement of an FP32 inverse W ~ M_nm(G)^{-1} (the periodic refresh
// of the cached inverses of FP32 chains):
//     R = I - M W,     W <- W + W R.
// M is sparse (each row couples a virtual Majorana to its own site and to
// the partner end of its link, <= B + 2 n_v entries), so R costs O(N^2 B)
// FP32 work assembled from the links; the dense product W R runs on the
// tcgen05 tensor cores through the flush kernel (W -= U V with U = W and
// V = -R, rank N).  The error of W after a step is about ||R||^2 plus the
// FP32 floor of computing R; for a residual below 1e-4 one TF32 product per
// term suffices (its 2^-11 rounding of a correction that small is below the
// FP32 rounding of W), larger residuals take the three-product split.
#include <algorithm>
#include <cstring>
#include "ggf_ctx.h"
#include "ggf_geom.cuh"

ggf_status ggf_flush_tc_one(ggf_ctx* ctx, bool cplx, int N, float* W, const float* Pan, const int* pend, int R,
                            int KRM, int nprod, cudaStream_t st);

namespace {

constexpr int RB = 8;          // output rows per CTA (one panel chunk)
constexpr int RT = 256;        // columns per CTA
constexpr int MAXC = 64;       // distinct columns of M touched by RB rows

template <class T> struct RefTy;
template <> struct RefTy<double> { typedef float S; };
template <> struct RefTy<cxd> { typedef cxf S; };

__device__ __forceinline__ float to_s(double v) { return (float)v; }
__device__ __forceinline__ cxf to_s(cxd v) { return {(float)v.x, (float)v.y}; }

// V^T panel (chunk-major, row = output column j, rank = output row q) of
// -R = M W - I for rows q0 .. q0 + 7 and columns j0 .. j0 + 255; the largest
// |R| entry goes to rmax (float bits, non-negative values compare as ints).
template <class T>
__global__ void __launch_bounds__(RT) resid_kernel(DevConst dc, const void* links, int cfg, int pair, const float* W,
                                                   float* Vt, size_t NK, int NP, unsigned* rmax) {
    typedef typename RefTy<T>::S S;
    constexpr bool CPLX = Sc<T>::CPLX;
    __shared__ int cols[MAXC];
    __shared__ S coef[RB][MAXC];
    __shared__ int ncol;
    __shared__ float red[RT / 32];
    const Geometry& g = dc.g;
    const int N = g.N, B = g.B;
    const int q0 = blockIdx.y * RB;
    const int j = blockIdx.x * RT + threadIdx.x;
    if (threadIdx.x == 0) {
        // columns: the site of q0 .. q0 + 7, then the partner ends of their links
        int n = 0;
        const int s = q0 / B;
        for (int k = 0; k < B; ++k) cols[n++] = s * B + k;
        for (int r = 0; r < RB; ++r) {
            const int q = q0 + r;
            if (q >= N) break;
            // the other end of q's link: the end e ^ 1 of the neighbouring site
            const int e = (q % B) / g.h2, d = e >> 1;
            const int x = s % g.L, y = s / g.L;
            int ps;
            if (e & 1) ps = d == 0 ? y * g.L + (x + 1) % g.L : ((y + 1) % g.L) * g.L + x;
            else ps = d == 0 ? y * g.L + (x + g.L - 1) % g.L : ((y + g.L - 1) % g.L) * g.L + x;
            const int pe = e ^ 1;
            for (int k = 0; k < g.h2; ++k) {
                const int c = ps * B + pe * g.h2 + k;
                bool dup = false;
                for (int z = 0; z < n; ++z) dup |= cols[z] == c;
                if (!dup && n < MAXC) cols[n++] = c;
            }
        }
        ncol = n;
    }
    __syncthreads();
    const int nc = ncol;
    for (int e = threadIdx.x; e < RB * nc; e += RT) {
        const int r = e / nc, c = e - r * nc;
        const int q = q0 + r;
        coef[r][c] = q < N ? to_s(assemble_elem<T>(dc, links, cfg, pair, q, cols[c])) : to_s(Sc<T>::zero());
    }
    __syncthreads();
    float mx = 0.f;
    if (j < N) {
        S acc[RB];
#pragma unroll
        for (int r = 0; r < RB; ++r) acc[r] = S{};
        for (int c = 0; c < nc; ++c) {
            if (!CPLX) {
                const float w = W[(size_t)cols[c] * N + j];
#pragma unroll
                for (int r = 0; r < RB; ++r) {
                    float& a = *(float*)&acc[r];
                    a = fmaf(*(const float*)&coef[r][c], w, a);
                }
            } else {
                const float2 w = *(const float2*)(W + ((size_t)cols[c] * N + j) * 2);
#pragma unroll
                for (int r = 0; r < RB; ++r) {
                    cxf& a = *(cxf*)&acc[r];
                    const cxf m = *(const cxf*)&coef[r][c];
                    a.x = fmaf(m.x, w.x, a.x);
                    a.x = fmaf(-m.y, w.y, a.x);
                    a.y = fmaf(m.x, w.y, a.y);
                    a.y = fmaf(m.y, w.x, a.y);
                }
            }
        }
        float out_r[RB], out_i[RB];
#pragma unroll
        for (int r = 0; r < RB; ++r) {
            const int q = q0 + r;
            if (!CPLX) {
                float v = *(float*)&acc[r];
                if (q == j) v -= 1.f;
                out_r[r] = v;
                out_i[r] = 0.f;
                mx = (v == v) ? fmaxf(mx, fabsf(v)) : __int_as_float(0x7f800000);
            } else {
                cxf v = *(cxf*)&acc[r];
                if (q == j) v.x -= 1.f;
                out_r[r] = v.x;
                out_i[r] = v.y;
                mx = (v.x == v.x && v.y == v.y) ? fmaxf(mx, fmaxf(fabsf(v.x), fabsf(v.y))) : __int_as_float(0x7f800000);
            }
            if (q >= N) { out_r[r] = 0.f; out_i[r] = 0.f; }
        }
        float* dst = Vt + pidx(j, q0, NP);
        *(float4*)dst = make_float4(out_r[0], out_r[1], out_r[2], out_r[3]);
        *(float4*)(dst + 4) = make_float4(out_r[4], out_r[5], out_r[6], out_r[7]);
        if (CPLX) {
            float* di = dst + NK;
            *(float4*)di = make_float4(out_i[0], out_i[1], out_i[2], out_i[3]);
            *(float4*)(di + 4) = make_float4(out_i[4], out_i[5], out_i[6], out_i[7]);
        }
    }
    if (!(mx == mx)) mx = __int_as_float(0x7f800000);   // NaN -> +inf
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_down_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = 0.f;
        for (int w = 0; w < RT / 32; ++w) m = fmaxf(m, red[w]);
        atomicMax(rmax, __float_as_uint(m));
    }
}

// U panel = W: element (row i, rank q) <- W[i][q], eight rank columns per thread
template <bool CPLX>
__global__ void upanel_kernel(int N, const float* W, float* U, size_t NK, int NP) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int q0 = blockIdx.y * 8;
    if (i >= N) return;
    float* dst = U + pidx(i, q0, NP);
    if (!CPLX) {
        const float* src = W + (size_t)i * N + q0;
        *(float4*)dst = *(const float4*)src;
        *(float4*)(dst + 4) = *(const float4*)(src + 4);
    } else {
        const float4* src = (const float4*)(W + ((size_t)i * N + q0) * 2);
        float re[8], im[8];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const float4 v = src[t];
            re[2 * t] = v.x; im[2 * t] = v.y; re[2 * t + 1] = v.z; im[2 * t + 1] = v.w;
        }
        *(float4*)dst = make_float4(re[0], re[1], re[2], re[3]);
        *(float4*)(dst + 4) = make_float4(re[4], re[5], re[6], re[7]);
        *(float4*)(dst + NK) = make_float4(im[0], im[1], im[2], im[3]);
        *(float4*)(dst + NK + 4) = make_float4(im[4], im[5], im[6], im[7]);
    }
}

__global__ void set_int(int* p, int v) { *p = v; }

}  // namespace

// Bytes of the refinement workspace for one matrix (U and V^T panels, rank N).
size_t ggf_refine_bytes(int N, bool cplx) {
    return panel_plane(N, N) * (cplx ? 4 : 2) * sizeof(float) + 256;
}

// Newton refinement of W (FP32, N x N, real or interleaved complex) for the
// matrix M of (cfg, pair-within-family), in two calls:
//   terms = 0: measure, *rmax = max |I - M W| over the entries, and keep
//              -R = M W - I in the workspace (synchronises the stream);
//   terms = 1 or 3: apply W <- W + W R with the R the last measure left (one
//              TF32 product, or the FP32-accurate three-product split).
// ws holds ggf_refine_bytes(N, cplx) bytes and must not change in between.
ggf_status ggf_refine_inverse(ggf_ctx* ctx, bool cplx, const void* d_links, int cfg, int pair, float* W, void* ws,
                              int terms, double* rmax, cudaStream_t st) {
    const Geometry& g = ctx->g;
    const int N = g.N, NP = panel_rows(N);
    if (N % 8) return ggf_fail(ctx, GGF_EINVAL, "refinement needs N divisible by 8");
    const size_t NK = panel_plane(N, N);
    float* Pan = (float*)ws;
    float* U = Pan;
    float* Vt = Pan + (cplx ? 2 : 1) * NK;
    unsigned* d_rmax = (unsigned*)(Pan + (cplx ? 4 : 2) * NK);
    int* d_pend = (int*)(d_rmax + 1);
    if (terms != 0) {
        dim3 ug((N + 255) / 256, N / 8);
        if (cplx) upanel_kernel<true><<<ug, 256, 0, st>>>(N, W, U, NK, NP);
        else upanel_kernel<false><<<ug, 256, 0, st>>>(N, W, U, NK, NP);
        set_int<<<1, 1, 0, st>>>(d_pend, N / 8);
        GGF_CK(cudaGetLastError());
        ctx->launches += 3;
        return ggf_flush_tc_one(ctx, cplx, N, W, Pan, d_pend, 8, N, terms, st);
    }
    GGF_CK(cudaMemsetAsync(d_rmax, 0, sizeof(unsigned), st));
    dim3 grid((N + RT - 1) / RT, (N + RB - 1) / RB);
    if (cplx)
        resid_kernel<cxd><<<grid, RT, 0, st>>>(ctx->dc(), d_links, cfg, pair, W, Vt, NK, NP, d_rmax);
    else
        resid_kernel<double><<<grid, RT, 0, st>>>(ctx->dc(), d_links, cfg, pair, W, Vt, NK, NP, d_rmax);
    GGF_CK(cudaGetLastError());
    ctx->launches += 1;
    unsigned hb = 0;
    GGF_CK(cudaMemcpyAsync(&hb, d_rmax, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    GGF_CK(cudaStreamSynchronize(st));
    float hr;
    std::memcpy(&hr, &hb, sizeof(float));
    *rmax = hr;
    return GGF_OK;
}
