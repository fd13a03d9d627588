// Score of the site blocks: d log N(G) / d D_s for every chain and site, from
// the chains' inverses (the per-thread item is score_item in ggf_obs.cuh).
// With it the gradient of a Wilson-loop energy with respect to the site
// parameters is the covariance E_p[(W(G) - E) sum_s tr(S_s^T dD_s)].
#include "ggf_obs.cuh"

namespace {

constexpr int STHREADS = 128;

// One thread per (chain, site).
template <class RW, class CW>
__global__ void __launch_bounds__(STHREADS) score_kernel(DevConst dc, int n_chains, const RW* Wr, const CW* Wc,
                                                         const cxd* ell, double* out) {
    const long long t = (long long)blockIdx.x * STHREADS + threadIdx.x;
    if (t >= (long long)n_chains * dc.g.V) return;
    const int c = (int)(t / dc.g.V), s = (int)(t - (long long)c * dc.g.V);
    score_item<RW, CW>(dc, c, s, Wr, Wc, ell, out);
}

// One thread per (chain, pair, link).
template <class RW, class CW, int R>
__global__ void __launch_bounds__(STHREADS) link_score_kernel(DevConst dc, int n_chains, const void* links,
                                                              const RW* Wr, const CW* Wc, const cxd* ell,
                                                              cxd* out) {
    const long long t = (long long)blockIdx.x * STHREADS + threadIdx.x;
    const long long per_chain = (long long)dc.P * dc.g.n_links;
    if (t >= (long long)n_chains * per_chain) return;
    const int c = (int)(t / per_chain);
    const long long rem = t - (long long)c * per_chain;
    const int p = (int)(rem / dc.g.n_links), l = (int)(rem - (long long)p * dc.g.n_links);
    link_score_item<RW, CW, R>(dc, c, p, l, links, Wr, Wc, ell, out);
}

}  // namespace

ggf_status ggf_flush(ggf_ctx* ctx, cudaStream_t st);

// Link-block scores of every chain, pair and link into d_out
// [n_chains][P][n_links][r][r] (device, complex).
ggf_status ggf_link_score(ggf_ctx* ctx, cxd* d_out, cudaStream_t st) {
    Chains& ch = ctx->ch;
    const Geometry& g = ctx->g;
    GGF_TRY(ggf_flush(ctx, st));
    const long long items = (long long)ch.n * ctx->P * g.n_links;
    const long long blocks = (items + STHREADS - 1) / STHREADS;
    if (blocks > 0x7fffffffLL) return ggf_fail(ctx, GGF_EINVAL, "too many chains for one launch");
    const bool fp64 = ch.opts.precision == GGF_FP64;
#define GGF_LS(RW, CW, R_)                                                                                   \
    link_score_kernel<RW, CW, R_><<<(unsigned)blocks, STHREADS, 0, st>>>(ctx->dc(), ch.n, ch.links,           \
                                                                        (const RW*)ch.Wr, (const CW*)ch.Wc, \
                                                                        ch.ell, d_out)
    if (g.r == 4) {
        if (fp64) GGF_LS(double, cxd, 4); else GGF_LS(float, cxf, 4);
    } else if (g.r == 8) {
        if (fp64) GGF_LS(double, cxd, 8); else GGF_LS(float, cxf, 8);
    } else {
        return ggf_fail(ctx, GGF_EINVAL, "n_v must be 1 or 2");
    }
#undef GGF_LS
    GGF_CK(cudaGetLastError());
    return GGF_OK;
}

// Site scores of every chain into d_out [n_chains][V][B][B] (device, FP64).
ggf_status ggf_score(ggf_ctx* ctx, double* d_out, cudaStream_t st) {
    Chains& ch = ctx->ch;
    const Geometry& g = ctx->g;
    GGF_TRY(ggf_flush(ctx, st));
    const long long items = (long long)ch.n * g.V;
    const long long blocks = (items + STHREADS - 1) / STHREADS;
    if (blocks > 0x7fffffffLL) return ggf_fail(ctx, GGF_EINVAL, "too many chains for one launch");
    if (ch.opts.precision == GGF_FP64)
        score_kernel<double, cxd><<<(unsigned)blocks, STHREADS, 0, st>>>(ctx->dc(), ch.n, (const double*)ch.Wr,
                                                                          (const cxd*)ch.Wc, ch.ell, d_out);
    else
        score_kernel<float, cxf><<<(unsigned)blocks, STHREADS, 0, st>>>(ctx->dc(), ch.n, (const float*)ch.Wr,
                                                                         (const cxf*)ch.Wc, ch.ell, d_out);
    GGF_CK(cudaGetLastError());
    return GGF_OK;
}
