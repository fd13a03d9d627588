// Electric-field observables (Sec. 5.3), evaluated for every chain and link
// from the inverses W_nm = M_nm(G)^{-1} the sampler keeps:
//   f_E(G)_l = sum_nm lambda_n^* lambda_m <psi_n(G)| I_l |psi_m(G)>_ket / N(G),
// with the insertion I_l acting on the ket's source-end modes of link l (the
// end that carries the twist) before the contraction:
//   Z2:   I_l = the parity of those modes, so that the ket becomes psi_m(G^(l))
//         (the flip X_l of the link, of which the Z2 electric term is a
//         linear function);
//   U(1): I_l = Q_l^2, Q_l = sum_j q_j n_j the twist charge of those modes: the
//         ket depends on its link angle through exp(i theta Q_l), so the
//         single-link integral with <G|J^2|g; G> (J = -i d/dtheta) is
//         -d^2/dtheta^2 of the overlap, i.e. the insertion of Q_l^2;
//   SU(2): I_l = sum_a (Q^a)^2 on the source doublet, Q^a = psi^dag (sigma_a / 2)
//         psi (right translations of the link act on the twist as
//         exp(i eps Q^a)), which is (3/4)(n_0 + n_1 - 2 n_0 n_1).
// The U(1) field <J_l> itself inserts I_l = Q_l (one derivative of the
// overlap), R_nm = sum_j q_j <n_j>; with charge-conserving site tensors and
// neutral bond pairs it obeys Gauss's law configuration by configuration.
// Wick's theorem on the Gaussian operator composed of the sites' virtual
// state and the bond operator X_nm gives the insertion's normalised
// expectation from the covariance of that operator on the end's 2 n_v
// Majoranas S,
//   Gamma_O = i 1 - (1 + i D) W_nm (1 + i Gamma_tw),   G = Gamma_O[S, S],
//   Z2:   R_nm = (-1)^{n_v} Pf(G),
//   SU(2): R_nm = (3/4)(<n_0> + <n_1> - 2 <n_0 n_1>),
//   U(1): R_nm = sum_j q_j^2 <n_j> + 2 sum_{j<k} q_j q_k <n_j n_k>,
//         <n_j> = (1 + G_{2j,2j+1}) / 2,
//         <n_j n_k> = (1 + G_{2j,2j+1} + G_{2k,2k+1} + Pf G[2j, 2j+1, 2k, 2k+1]) / 4,
// with M_nm = D + Gamma_tw, D the sites' virtual blocks and Gamma_tw =
// O(G) Gamma_X O(G)^T the twisted link blocks.  D is block diagonal by site
// and Gamma_tw by link, so [(1 + i D) W (1 + i Gamma_tw)]_SS involves only the
// B x r block of W between the source site's virtual Majoranas and the link's
// r Majoranas.  D and the twist are real and Gamma_X of (m, n) is the complex
// conjugate of that of (n, m), so M_mn = conj(M_nm): both orders of a pair
// n < m come from its one stored inverse.  With N_nm = e^{logc + ell}
// (N_mn = conj N_nm) and the pair weights of the sampler's combination,
//   f_E(G)_l = sum_nm lambda_n^* lambda_m N_nm R_nm / sum_nm lambda_n^* lambda_m N_nm.
#include "ggf_obs.cuh"

namespace {

constexpr int ETHREADS = 128;

// One thread per (chain, link); FIELD: the U(1) electric field instead of J^2.
template <class RW, class CW, int H, bool FIELD>
__global__ void __launch_bounds__(ETHREADS) electric_kernel(DevConst dc, int n_chains, int blocks_per_chain,
                                                            const void* links, const RW* Wr, const CW* Wc,
                                                            const cxd* ell, cxd* out, cxd* pair_out) {
    const int c = blockIdx.x / blocks_per_chain;
    const int l = (blockIdx.x - c * blocks_per_chain) * ETHREADS + threadIdx.x;
    if (c >= n_chains || l >= dc.g.n_links) return;
    electric_item<RW, CW, H, FIELD>(dc, c, l, links, Wr, Wc, ell, out, pair_out);
}

// One thread per chain.
__global__ void pair_norm_kernel(DevConst dc, int n_chains, const cxd* ell, cxd* out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_chains) return;
    pair_norm_item(dc, c, ell, out);
}

}  // namespace

ggf_status ggf_flush(ggf_ctx* ctx, cudaStream_t st);

// N_nm(G) / N(G) of every chain into d_out [n_chains][K][K] (device).
ggf_status ggf_pair_norm(ggf_ctx* ctx, cxd* d_out, cudaStream_t st) {
    Chains& ch = ctx->ch;
    pair_norm_kernel<<<(ch.n + 127) / 128, 128, 0, st>>>(ctx->dc(), ch.n, ch.ell, d_out);
    GGF_CK(cudaGetLastError());
    return GGF_OK;
}

// f_E for every chain and link into d_out [n_chains][n_links] and/or its
// per-pair parts into d_pairs [n_chains][n_links][K][K] (device; either may
// be null): Z2 the flip, U(1) and SU(2) the Casimir J^2.
ggf_status ggf_electric(ggf_ctx* ctx, cxd* d_out, cxd* d_pairs, cudaStream_t st, bool field) {
    Chains& ch = ctx->ch;
    const Geometry& g = ctx->g;
    // pending delayed updates first, so that W is the inverse at the current links
    GGF_TRY(ggf_flush(ctx, st));
    const int bpc = (g.n_links + ETHREADS - 1) / ETHREADS;
    const long long blocks = (long long)bpc * ch.n;
    if (blocks > 0x7fffffffLL) return ggf_fail(ctx, GGF_EINVAL, "too many chains for one launch");
    const bool fp64 = ch.opts.precision == GGF_FP64;
    const void* lk = ch.links;
#define GGF_EL2(RW, CW, H, F)                                                                            \
    electric_kernel<RW, CW, H, F><<<(unsigned)blocks, ETHREADS, 0, st>>>(ctx->dc(), ch.n, bpc, lk,       \
                                                                         (const RW*)ch.Wr,                \
                                                                         (const CW*)ch.Wc, ch.ell, d_out, \
                                                                         d_pairs)
#define GGF_EL(RW, CW, H)                  \
    do {                                   \
        if (field) GGF_EL2(RW, CW, H, true); \
        else GGF_EL2(RW, CW, H, false);      \
    } while (0)
    if (g.h2 == 2) {
        if (fp64) GGF_EL(double, cxd, 2); else GGF_EL(float, cxf, 2);
    } else if (g.h2 == 4) {
        if (fp64) GGF_EL(double, cxd, 4); else GGF_EL(float, cxf, 4);
    } else {
        return ggf_fail(ctx, GGF_EINVAL, "n_v must be 1 or 2");
    }
#undef GGF_EL
#undef GGF_EL2
    GGF_CK(cudaGetLastError());
    return GGF_OK;
}
