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

}  // namespace

ggf_status ggf_flush(ggf_ctx* ctx, cudaStream_t st);

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
