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
#include "ggf_ctx.h"
#include "ggf_sweep.cuh"

namespace {

constexpr int ETHREADS = 128;

// Pfaffian of an H x H antisymmetric matrix (H = 2 n_v = 2 or 4), closed form.
template <int H>
__device__ __forceinline__ cxd small_pf(const cxd (&A)[H][H]);
template <>
__device__ __forceinline__ cxd small_pf<2>(const cxd (&A)[2][2]) { return A[0][1]; }
template <>
__device__ __forceinline__ cxd small_pf<4>(const cxd (&A)[4][4]) {
    return A[0][1] * A[2][3] - A[0][2] * A[1][3] + A[0][3] * A[1][2];
}

__device__ __forceinline__ cxd times_i(cxd v) { return {-v.y, v.x}; }

// Normalised expectation of the insertion from G = Gamma_O[S, S].
template <int H>
__device__ __forceinline__ cxd insertion(const Geometry& g, const cxd (&G)[H][H]) {
    if (g.group == GGF_Z2) {
        const double sg = (H / 2) % 2 ? -1.0 : 1.0;    // (-1)^{n_v}
        return sg * small_pf<H>(G);
    }
    if constexpr (H == 4) {
        if (g.group == GGF_SU2) {
            // sum_a (Q^a)^2 on the doublet = (3/4)(n_0 + n_1 - 2 n_0 n_1)
            cxd o = G[0][1] + G[2][3];
            o.x += 2.0;                                  // 2 (<n_0> + <n_1>)
            cxd pr = G[0][1] + G[2][3] + small_pf<H>(G);
            pr.x += 1.0;                                 // 4 <n_0 n_1>
            return 0.375 * (o - pr);                     // (3/4)(o / 2 - 2 pr / 4)
        }
    }
    cxd val = {0.0, 0.0};
#pragma unroll
    for (int j = 0; j < H / 2; ++j) {
        const double qj = g.q[j];
        cxd occ = G[2 * j][2 * j + 1];
        occ.x += 1.0;
        val += (0.5 * qj * qj) * occ;
    }
    if constexpr (H == 4) {
        cxd pr = G[0][1] + G[2][3] + small_pf<H>(G);
        pr.x += 1.0;
        val += (0.5 * g.q[0] * g.q[1]) * pr;            // 2 q_0 q_1 <n_0 n_1>
    }
    return val;
}

// R for both orders of pair p at link l: Rf from (W, Gamma_tw), Rr from their
// conjugates.  W points at the pair's N x N inverse (row-major).
template <class T, int H>
__device__ void flip_ratios(const DevConst& dc, int p, bool cplx_pair, const T* W, int l, double gval,
                            double theta, const double* Rsu2, cxd& Rf, cxd& Rr) {
    constexpr int R = 2 * H, B = 4 * H;
    const Geometry& g = dc.g;
    int a0, b0;
    link_ends(g, l, a0, b0);
    const int s0 = (l >> 1) * g.B;        // first virtual Majorana of the source site
    const int loc0 = a0 - s0;             // position of S inside the site block
    const double* Ds = dc.D + (size_t)(l >> 1) * B * B;
    cxd Xf[H][H], Xr[H][H];
#pragma unroll
    for (int a = 0; a < H; ++a)
#pragma unroll
        for (int b = 0; b < H; ++b) Xf[a][b] = Xr[a][b] = cxd{0.0, 0.0};
#pragma unroll
    for (int b = 0; b < H; ++b) {
        // column b of (1 + i Gamma_tw)[link, S] and of its conjugate
        cxd cf[R], cr[R];
#pragma unroll
        for (int j = 0; j < R; ++j) {
            cxd gt;
            if (Rsu2) {
                if (cplx_pair) gt = twisted_su2<cxd>(dc, p - dc.K, l, j, b, Rsu2);
                else gt = cxd{twisted_su2<double>(dc, p, l, j, b, Rsu2), 0.0};
            } else {
                if (cplx_pair) gt = twisted<cxd>(dc, p - dc.K, l, j, b, gval, theta);
                else gt = cxd{twisted<double>(dc, p, l, j, b, gval, theta), 0.0};
            }
            cf[j] = times_i(gt);
            cr[j] = times_i(conjg(gt));
            if (j == b) { cf[j].x += 1.0; cr[j].x += 1.0; }
        }
        for (int i = 0; i < B; ++i) {
            const T* row = W + (size_t)(s0 + i) * g.N;
            cxd yf = {0.0, 0.0}, yr = {0.0, 0.0};
#pragma unroll
            for (int j = 0; j < R; ++j) {
                const cxd w = Sc<T>::to(row[link_majorana(g, a0, b0, j)]);
                yf += w * cf[j];
                yr += conjg(w) * cr[j];
            }
            // row a of (1 + i D)[S, site] at column i
#pragma unroll
            for (int a = 0; a < H; ++a) {
                cxd dp = {0.0, Ds[(size_t)(loc0 + a) * B + i]};
                if (loc0 + a == i) dp.x = 1.0;
                Xf[a][b] += dp * yf;
                Xr[a][b] += dp * yr;
            }
        }
    }
#pragma unroll
    for (int a = 0; a < H; ++a)
#pragma unroll
        for (int b = 0; b < H; ++b) {
            Xf[a][b] = -Xf[a][b];
            Xr[a][b] = -Xr[a][b];
            if (a == b) { Xf[a][b].y += 1.0; Xr[a][b].y += 1.0; }
        }
    Rf = insertion<H>(g, Xf);
    Rr = insertion<H>(g, Xr);
}

// One thread per (chain, link); out[c][l] = f_E(G_c)_l (if out is set) and
// pair_out[c][l][n][m] = N_nm(G) R_nm / N(G) for every ordered pair (if set).
template <class RW, class CW, int H>
__global__ void __launch_bounds__(ETHREADS) electric_kernel(DevConst dc, int n_chains, int blocks_per_chain,
                                                            const void* links, const RW* Wr, const CW* Wc,
                                                            const cxd* ell, cxd* out, cxd* pair_out) {
    const Geometry& g = dc.g;
    const int c = blockIdx.x / blocks_per_chain;
    const int l = (blockIdx.x - c * blocks_per_chain) * ETHREADS + threadIdx.x;
    if (c >= n_chains || l >= g.n_links) return;
    const size_t NN = (size_t)g.N * g.N;
    double gval = 1.0, theta = 0.0, Rq[16];
    const double* Rsu2 = nullptr;
    if (g.group == GGF_SU2) {
        doublet_rotation(link_quat(g, links, c, l), Rq);
        Rsu2 = Rq;
    } else {
        link_value<double>(dc, links, c, l, gval, theta);
    }
    const cxd* el = ell + (size_t)c * dc.P;
    double amax, iden;
    pair_scale(dc, el, amax, iden);
    cxd num = {0.0, 0.0};
    for (int p = 0; p < dc.P; ++p) {
        const bool cplx = p >= dc.K;
        const cxd Np = pair_norm(dc, el, p, amax, iden);   // N_nm(G) / N(G)
        const cxd E = dc.w[p] * Np;              // w_p N_p / N(G)
        cxd Rf, Rr;
        int n, m;
        pair_nm(dc.K, p, n, m);
        cxd* po = pair_out ? pair_out + ((size_t)c * g.n_links + l) * dc.K * dc.K : nullptr;
        if (cplx) {
            flip_ratios<CW, H>(dc, p, true, Wc + ((size_t)c * dc.Kc + (p - dc.K)) * NN, l, gval, theta, Rsu2, Rf, Rr);
            // w_p = 2 lambda_n^* lambda_m: the (n, m) term takes E / 2, the (m, n) term its conjugate
            num += 0.5 * (E * Rf) + 0.5 * (conjg(E) * Rr);
            if (po) {
                po[n * dc.K + m] = Np * Rf;
                po[m * dc.K + n] = conjg(Np) * Rr;
            }
        } else {
            flip_ratios<RW, H>(dc, p, false, Wr + ((size_t)c * dc.K + p) * NN, l, gval, theta, Rsu2, Rf, Rr);
            num += E * Rf;
            if (po) po[n * dc.K + n] = Np * Rf;
        }
    }
    if (out) out[(size_t)c * g.n_links + l] = num;
}

// One thread per chain: out[c][n][m] = N_nm(G) / N(G) for every ordered pair.
__global__ void pair_norm_kernel(DevConst dc, int n_chains, const cxd* ell, cxd* out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_chains) return;
    const int K = dc.K;
    const cxd* el = ell + (size_t)c * dc.P;
    double amax, iden;
    pair_scale(dc, el, amax, iden);
    cxd* o = out + (size_t)c * K * K;
    for (int p = 0; p < dc.P; ++p) {
        const cxd Np = pair_norm(dc, el, p, amax, iden);
        int n, m;
        pair_nm(K, p, n, m);
        o[n * K + m] = Np;
        if (n != m) o[m * K + n] = conjg(Np);
    }
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
ggf_status ggf_electric(ggf_ctx* ctx, cxd* d_out, cxd* d_pairs, cudaStream_t st) {
    Chains& ch = ctx->ch;
    const Geometry& g = ctx->g;
    // pending delayed updates first, so that W is the inverse at the current links
    GGF_TRY(ggf_flush(ctx, st));
    const int bpc = (g.n_links + ETHREADS - 1) / ETHREADS;
    const long long blocks = (long long)bpc * ch.n;
    if (blocks > 0x7fffffffLL) return ggf_fail(ctx, GGF_EINVAL, "too many chains for one launch");
    const bool fp64 = ch.opts.precision == GGF_FP64;
    const void* lk = ch.links;
#define GGF_EL(RW, CW, H)                                                                                \
    electric_kernel<RW, CW, H><<<(unsigned)blocks, ETHREADS, 0, st>>>(ctx->dc(), ch.n, bpc, lk,          \
                                                                      (const RW*)ch.Wr, (const CW*)ch.Wc, \
                                                                      ch.ell, d_out, d_pairs)
    if (g.h2 == 2) {
        if (fp64) GGF_EL(double, cxd, 2); else GGF_EL(float, cxf, 2);
    } else if (g.h2 == 4) {
        if (fp64) GGF_EL(double, cxd, 4); else GGF_EL(float, cxf, 4);
    } else {
        return ggf_fail(ctx, GGF_EINVAL, "n_v must be 1 or 2");
    }
#undef GGF_EL
    GGF_CK(cudaGetLastError());
    return GGF_OK;
}
