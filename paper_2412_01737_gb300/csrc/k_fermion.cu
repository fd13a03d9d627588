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
// the link block; the gauge string of the operator multiplies them).
#include "ggf_ctx.h"
#include "ggf_sweep.cuh"

namespace {

constexpr int FTHREADS = 128;

__device__ __forceinline__ cxd times_minus_i(cxd v) { return {v.y, -v.x}; }

// X[alpha][beta] = sum_ij B_s[alpha][i] W[sB + i][tB + j] B_t[beta][j] for
// alpha in {0, 1} (rows) and beta in {0, 1}, BW = B (virtual Majoranas per site).
template <class T, int BW>
__device__ void coupled_block(const DevConst& dc, const T* W, int s, int t, cxd (&X)[2][2]) {
    const int N = dc.g.N;
    const double* Bs = dc.Bp + (size_t)s * 2 * BW;
    const double* Bt = dc.Bp + (size_t)t * 2 * BW;
    X[0][0] = X[0][1] = X[1][0] = X[1][1] = cxd{0.0, 0.0};
    for (int i = 0; i < BW; ++i) {
        const T* row = W + (size_t)(s * BW + i) * N + (size_t)t * BW;
        cxd u0 = {0.0, 0.0}, u1 = {0.0, 0.0};
#pragma unroll
        for (int j = 0; j < BW; ++j) {
            const cxd w = Sc<T>::to(row[j]);
            u0 += w * Bt[j];
            u1 += w * Bt[BW + j];
        }
        X[0][0] += Bs[i] * u0;
        X[0][1] += Bs[i] * u1;
        X[1][0] += Bs[BW + i] * u0;
        X[1][1] += Bs[BW + i] * u1;
    }
}

// Per-pair expectation -i (A + X)[alpha][beta] of entry (alpha, beta) of item
// (s, t), with c_a c_a = 1 where both Majoranas coincide (self-links).
__device__ __forceinline__ cxd pair_bilinear(const DevConst& dc, int s, int t, int a, int b, cxd x) {
    if (s == t) {
        if (a == b) return cxd{1.0, 0.0};
        x.x += dc.Ap[(size_t)s * 4 + a * 2 + b];
    }
    return times_minus_i(x);
}

// One thread per (chain, item): items 0 .. V-1 are sites, V .. V + n_links - 1 links.
// Combined outputs site_out / link_out and per-pair outputs
// pair_site[c][s][n][m], pair_link[c][l][alpha][beta][n][m] =
// N_nm(G) <c c>_nm / N(G) (each may be null).
template <class RW, class CW, int BW>
__global__ void __launch_bounds__(FTHREADS) fermion_kernel(DevConst dc, int n_chains, int blocks_per_chain,
                                                           const RW* Wr, const CW* Wc, const cxd* ell,
                                                           cxd* site_out, cxd* link_out, cxd* pair_site,
                                                           cxd* pair_link) {
    const Geometry& g = dc.g;
    const int c = blockIdx.x / blocks_per_chain;
    const int it = (blockIdx.x - c * blocks_per_chain) * FTHREADS + threadIdx.x;
    const int items = g.V + g.n_links;
    if (c >= n_chains || it >= items) return;
    const bool is_site = it < g.V;
    int s, t;
    if (is_site) {
        s = t = it;
    } else {
        int a0, b0;
        link_ends(g, it - g.V, a0, b0);
        s = a0 / g.B;
        t = b0 / g.B;
    }
    cxd* out = is_site ? site_out : link_out;
    cxd* pout = is_site ? pair_site : pair_link;
    if (!out && !pout) return;
    const int K = dc.K;
    if (pout) pout += is_site ? ((size_t)c * g.V + s) * K * K : ((size_t)c * g.n_links + (it - g.V)) * 4 * K * K;
    const size_t NN = (size_t)g.N * g.N;
    const cxd* el = ell + (size_t)c * dc.P;
    double amax, iden;
    pair_scale(dc, el, amax, iden);
    cxd acc[2][2] = {{{0.0, 0.0}, {0.0, 0.0}}, {{0.0, 0.0}, {0.0, 0.0}}};
    for (int p = 0; p < dc.P; ++p) {
        const bool cplx = p >= K;
        const cxd Np = pair_norm(dc, el, p, amax, iden);   // N_nm(G) / N(G)
        const cxd E = dc.w[p] * Np;              // w_p N_p / N(G)
        int n, m;
        pair_nm(K, p, n, m);
        cxd X[2][2];
        if (cplx) {
            coupled_block<CW, BW>(dc, Wc + ((size_t)c * dc.Kc + (p - K)) * NN, s, t, X);
            // (n, m) with weight E / 2 (w_p = 2 lambda_n^* lambda_m), (m, n) with
            // conj(E) / 2 and the conjugate product; A is added after the loop
            const cxd h = 0.5 * E, hc = conjg(h);
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
                for (int b = 0; b < 2; ++b) {
                    acc[a][b] += h * X[a][b] + hc * conjg(X[a][b]);
                    if (pout && (!is_site || (a == 0 && b == 1))) {
                        cxd* q = pout + (is_site ? 0 : (size_t)(a * 2 + b) * K * K);
                        q[n * K + m] = Np * pair_bilinear(dc, s, t, a, b, X[a][b]);
                        q[m * K + n] = conjg(Np) * pair_bilinear(dc, s, t, a, b, conjg(X[a][b]));
                    }
                }
        } else {
            coupled_block<RW, BW>(dc, Wr + ((size_t)c * dc.K + p) * NN, s, t, X);
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
                for (int b = 0; b < 2; ++b) {
                    acc[a][b] += E * X[a][b];
                    if (pout && (!is_site || (a == 0 && b == 1))) {
                        cxd* q = pout + (is_site ? 0 : (size_t)(a * 2 + b) * K * K);
                        q[n * K + n] = Np * pair_bilinear(dc, s, t, a, b, X[a][b]);
                    }
                }
        }
    }
    if (!out) return;
    // F = -i (A + sum_p weight_p X_p); A enters with the total weight
    // sum_nm lambda_n^* lambda_m N_nm / N(G) = 1 (only where s == t)
    cxd F[2][2];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) F[a][b] = pair_bilinear(dc, s, t, a, b, acc[a][b]);
    if (is_site) {
        out[(size_t)c * g.V + s] = F[0][1];
    } else {
        cxd* o = out + ((size_t)c * g.n_links + (it - g.V)) * 4;
        o[0] = F[0][0]; o[1] = F[0][1]; o[2] = F[1][0]; o[3] = F[1][1];
    }
}

}  // namespace

ggf_status ggf_flush(ggf_ctx* ctx, cudaStream_t st);

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
