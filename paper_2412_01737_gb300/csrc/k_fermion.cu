// Fermionic observables (Sec. 5.2): Majorana bilinears on the physical modes
// for every chain, from the inverses W_nm = M_nm(G)^{-1} the sampler keeps.
//
// Contracting the virtual modes of the site states with the bond operator
// X_nm leaves a Gaussian operator on the physical Majoranas whose covariance
// is the Schur complement
//   Gamma_eff^nm = A + B W_nm B^T,
// A the sites' physical blocks and B their physical-virtual couplings (both
// block diagonal by site; the twist sits on the bond side of M = D + O Gamma_X
// O^T, so A and B are untwisted).  By Wick's theorem
//   <psi_n(G)| c_a c_b |psi_m(G)> = N_nm(G) (-i Gamma_eff^nm[a, b])   (a != b).
// Entry (a on site s, b on site t) needs only the B x B block W[site s, site t].
// A and B are real and M_mn = conj(M_nm), so Gamma_eff^mn = A + conj(B W_nm B^T):
// one product serves both orders of a pair n < m.  Outputs per chain:
//   site[s]           = sum_nm lambda_n^* lambda_m <psi_n|c_2s c_2s+1|psi_m> / N(G)
//   link[l][alpha][beta] = same for c_{2s+alpha} c_{2t+beta}, link l = (s -> t)
// (densities n_s = (1 + i site[s]) / 2; hoppings and pairings are linear in
// the link block, and link_term_kernel forms the gauge-invariant one with the
// link operator, u_l F_s F_t, from it).
#include "ggf_obs.cuh"

namespace {

constexpr int FTHREADS = 128;

// One thread per (chain, item).
template <class RW, class CW, int BW>
__global__ void __launch_bounds__(FTHREADS) fermion_kernel(DevConst dc, int n_chains, int blocks_per_chain,
                                                           const RW* Wr, const CW* Wc, const cxd* ell,
                                                           cxd* site_out, cxd* link_out, cxd* pair_site,
                                                           cxd* pair_link) {
    const int c = blockIdx.x / blocks_per_chain;
    const int it = (blockIdx.x - c * blocks_per_chain) * FTHREADS + threadIdx.x;
    if (c >= n_chains || it >= dc.g.V + dc.g.n_links) return;
    fermion_item<RW, CW, BW>(dc, c, it, Wr, Wc, ell, site_out, link_out, pair_site, pair_link);
}

// One thread per (chain, link).
template <class RW, class CW, int BW>
__global__ void __launch_bounds__(FTHREADS) fermion4_kernel(DevConst dc, int n_chains, int blocks_per_chain,
                                                            const RW* Wr, const CW* Wc, const cxd* ell, cxd* out,
                                                            cxd* pair_out) {
    const int c = blockIdx.x / blocks_per_chain;
    const int l = (blockIdx.x - c * blocks_per_chain) * FTHREADS + threadIdx.x;
    if (c >= n_chains || l >= dc.g.n_links) return;
    fermion4_item<RW, CW, BW>(dc, c, l, Wr, Wc, ell, out, pair_out);
}

// One thread per (chain, link).
__global__ void __launch_bounds__(FTHREADS) link_term_kernel(DevConst dc, int n_chains, const void* links,
                                                             const int* q, const cxd* blk, const cxd* pair_blk,
                                                             cxd* out, cxd* pair_out) {
    const long long t = (long long)blockIdx.x * FTHREADS + threadIdx.x;
    if (t >= (long long)n_chains * dc.g.n_links) return;
    const int c = (int)(t / dc.g.n_links), l = (int)(t - (long long)c * dc.g.n_links);
    link_term_item(dc, c, l, links, q, blk, pair_blk, out, pair_out);
}

}  // namespace

ggf_status ggf_flush(ggf_ctx* ctx, cudaStream_t st);
ggf_status ggf_fermion(ggf_ctx* ctx, cxd* d_site, cxd* d_link, cxd* d_pair_site, cxd* d_pair_link,
                       cudaStream_t st);

// Gauge-invariant link terms of every chain into d_out [n][n_links] and/or
// their per-pair parts into d_pair_out [n][n_links][K][K] (device; either may
// be null), through the link blocks written to the scratch buffers d_blk
// [n][n_links][2][2] and d_pair_blk [n][n_links][2][2][K][K]; d_q [V] device.
ggf_status ggf_link_terms(ggf_ctx* ctx, const int* d_q, cxd* d_blk, cxd* d_pair_blk, cxd* d_out, cxd* d_pair_out,
                          cudaStream_t st) {
    Chains& ch = ctx->ch;
    const Geometry& g = ctx->g;
    if (!d_out) d_blk = nullptr;
    if (!d_pair_out) d_pair_blk = nullptr;
    if (!d_blk && !d_pair_blk) return GGF_OK;
    GGF_TRY(ggf_fermion(ctx, nullptr, d_blk, nullptr, d_pair_blk, st));
    const long long items = (long long)ch.n * g.n_links;
    const long long blocks = (items + FTHREADS - 1) / FTHREADS;
    if (blocks > 0x7fffffffLL) return ggf_fail(ctx, GGF_EINVAL, "too many chains for one launch");
    link_term_kernel<<<(unsigned)blocks, FTHREADS, 0, st>>>(ctx->dc(), ch.n, ch.links, d_q, d_blk, d_pair_blk,
                                                             d_out, d_pair_out);
    GGF_CK(cudaGetLastError());
    return GGF_OK;
}

// <c_2s c_2s+1 c_2t c_2t+1> of every chain and link into d_out [n][n_links]
// and/or its per-pair parts into d_pairs [n][n_links][K][K] (device; either
// may be null).
ggf_status ggf_fermion4(ggf_ctx* ctx, cxd* d_out, cudaStream_t st, cxd* d_pairs) {
    Chains& ch = ctx->ch;
    const Geometry& g = ctx->g;
    GGF_TRY(ggf_flush(ctx, st));
    const int bpc = (g.n_links + FTHREADS - 1) / FTHREADS;
    const long long blocks = (long long)bpc * ch.n;
    if (blocks > 0x7fffffffLL) return ggf_fail(ctx, GGF_EINVAL, "too many chains for one launch");
    const bool fp64 = ch.opts.precision == GGF_FP64;
#define GGF_F4(RW, CW, BW)                                                                                 \
    fermion4_kernel<RW, CW, BW><<<(unsigned)blocks, FTHREADS, 0, st>>>(ctx->dc(), ch.n, bpc, (const RW*)ch.Wr, \
                                                                       (const CW*)ch.Wc, ch.ell, d_out, d_pairs)
    if (g.B == 8) {
        if (fp64) GGF_F4(double, cxd, 8); else GGF_F4(float, cxf, 8);
    } else if (g.B == 16) {
        if (fp64) GGF_F4(double, cxd, 16); else GGF_F4(float, cxf, 16);
    } else {
        return ggf_fail(ctx, GGF_EINVAL, "n_v must be 1 or 2");
    }
#undef GGF_F4
    GGF_CK(cudaGetLastError());
    return GGF_OK;
}

// Site and link bilinears of every chain into d_site [n][V] and d_link
// [n][n_links][2][2], and their per-pair parts into d_pair_site [n][V][K][K]
// and d_pair_link [n][n_links][2][2][K][K] (device; any may be null).
ggf_status ggf_fermion(ggf_ctx* ctx, cxd* d_site, cxd* d_link, cxd* d_pair_site, cxd* d_pair_link,
                       cudaStream_t st) {
    Chains& ch = ctx->ch;
    const Geometry& g = ctx->g;
    GGF_TRY(ggf_flush(ctx, st));
    const int items = g.V + g.n_links;
    const int bpc = (items + FTHREADS - 1) / FTHREADS;
    const long long blocks = (long long)bpc * ch.n;
    if (blocks > 0x7fffffffLL) return ggf_fail(ctx, GGF_EINVAL, "too many chains for one launch");
    const bool fp64 = ch.opts.precision == GGF_FP64;
#define GGF_FE(RW, CW, BW)                                                                                 \
    fermion_kernel<RW, CW, BW><<<(unsigned)blocks, FTHREADS, 0, st>>>(ctx->dc(), ch.n, bpc, (const RW*)ch.Wr, \
                                                                      (const CW*)ch.Wc, ch.ell, d_site, d_link, \
                                                                      d_pair_site, d_pair_link)
    if (g.B == 8) {
        if (fp64) GGF_FE(double, cxd, 8); else GGF_FE(float, cxf, 8);
    } else if (g.B == 16) {
        if (fp64) GGF_FE(double, cxd, 16); else GGF_FE(float, cxf, 16);
    } else {
        return ggf_fail(ctx, GGF_EINVAL, "n_v must be 1 or 2");
    }
#undef GGF_FE
    GGF_CK(cudaGetLastError());
    return GGF_OK;
}
