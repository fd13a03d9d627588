// Per-thread bodies of the observable kernels (electric, Sec. 5.3; fermionic,
// Sec. 5.2; per-pair norms), host and device callable; the kernels in
// k_electric.cu and k_fermion.cu run one item per thread.
#pragma once
#include "ggf_ctx.h"
#include "ggf_sweep.cuh"

namespace {

// ---- electric (the derivation is in k_electric.cu) ---------------------------

// Pfaffian of an H x H antisymmetric matrix (H = 2 n_v = 2 or 4), closed form.
template <int H>
GGF_HD cxd small_pf(const cxd (&A)[H][H]);
template <>
GGF_HD cxd small_pf<2>(const cxd (&A)[2][2]) { return A[0][1]; }
template <>
GGF_HD cxd small_pf<4>(const cxd (&A)[4][4]) {
    return A[0][1] * A[2][3] - A[0][2] * A[1][3] + A[0][3] * A[1][2];
}

GGF_HD cxd times_i(cxd v) { return {-v.y, v.x}; }

// Normalised expectation of the insertion from G = Gamma_O[S, S]; FIELD: the
// U(1) twist charge Q_l itself (the electric field) instead of Q_l^2.
template <int H, bool FIELD = false>
GGF_HD cxd insertion(const Geometry& g, const cxd (&G)[H][H]) {
    if constexpr (FIELD) {
        cxd val = {0.0, 0.0};
#pragma unroll
        for (int j = 0; j < H / 2; ++j) {
            cxd occ = G[2 * j][2 * j + 1];
            occ.x += 1.0;
            val += (0.5 * (double)g.q[j]) * occ;       // q_j <n_j>
        }
        return val;
    }
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
template <class T, int H, bool FIELD = false>
__host__ __device__ void flip_ratios(const DevConst& dc, int p, bool cplx_pair, const T* W, int l, double gval,
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
    Rf = insertion<H, FIELD>(g, Xf);
    Rr = insertion<H, FIELD>(g, Xr);
}

// f_E(G_c)_l into out[c][l] (if out is set) and N_nm(G) R_nm / N(G) into
// pair_out[c][l][n][m] for every ordered pair (if set).
template <class RW, class CW, int H, bool FIELD = false>
__host__ __device__ void electric_item(const DevConst& dc, int c, int l, const void* links, const RW* Wr,
                                       const CW* Wc, const cxd* ell, cxd* out, cxd* pair_out) {
    const Geometry& g = dc.g;
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
            flip_ratios<CW, H, FIELD>(dc, p, true, Wc + ((size_t)c * dc.Kc + (p - dc.K)) * NN, l, gval, theta, Rsu2,
                                      Rf, Rr);
            // w_p = 2 lambda_n^* lambda_m: the (n, m) term takes E / 2, the (m, n) term its conjugate
            num += 0.5 * (E * Rf) + 0.5 * (conjg(E) * Rr);
            if (po) {
                po[n * dc.K + m] = Np * Rf;
                po[m * dc.K + n] = conjg(Np) * Rr;
            }
        } else {
            flip_ratios<RW, H, FIELD>(dc, p, false, Wr + ((size_t)c * dc.K + p) * NN, l, gval, theta, Rsu2, Rf, Rr);
            num += E * Rf;
            if (po) po[n * dc.K + n] = Np * Rf;
        }
    }
    if (out) out[(size_t)c * g.n_links + l] = num;
}

// N_nm(G) / N(G) of chain c into out[c][n][m] for every ordered pair.
__host__ __device__ inline void pair_norm_item(const DevConst& dc, int c, const cxd* ell, cxd* out) {
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

// ---- fermionic (the derivation is in k_fermion.cu) ---------------------------


GGF_HD cxd times_minus_i(cxd v) { return {v.y, -v.x}; }

// X[alpha][beta] = sum_ij B_s[alpha][i] W[sB + i][tB + j] B_t[beta][j] for
// alpha in {0, 1} (rows) and beta in {0, 1}, BW = B (virtual Majoranas per site).
template <class T, int BW>
__host__ __device__ void coupled_block(const DevConst& dc, const T* W, int s, int t, cxd (&X)[2][2]) {
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
GGF_HD cxd pair_bilinear(const DevConst& dc, int s, int t, int a, int b, cxd x) {
    if (s == t) {
        if (a == b) return cxd{1.0, 0.0};
        x.x += dc.Ap[(size_t)s * 4 + a * 2 + b];
    }
    return times_minus_i(x);
}

// Item it of chain c (items 0 .. V-1 are sites, V .. V + n_links - 1 links):
// combined outputs site_out / link_out and per-pair outputs
// pair_site[c][s][n][m], pair_link[c][l][alpha][beta][n][m] =
// N_nm(G) <c c>_nm / N(G) (each may be null).
template <class RW, class CW, int BW>
__host__ __device__ void fermion_item(const DevConst& dc, int c, int it, const RW* Wr, const CW* Wc,
                                      const cxd* ell, cxd* site_out, cxd* link_out, cxd* pair_site,
                                      cxd* pair_link) {
    const Geometry& g = dc.g;
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

// ---- gauge-invariant link terms ------------------------------------------------
// A physical bilinear across link l = (s -> t) is gauge invariant together with
// the link operator u_l (Z2: g_l; U(1): e^{i theta_l}, diagonal in G) when it
// carries the charge u_l removes: T_l = u_l F_s F_t with F_s = psi_s (q_s > 0)
// or psi_s^dag (q_s < 0) and F_t = psi_t^dag (q_t > 0) or psi_t (q_t < 0); for
// staggered charges that is the pair term, and T_l + T_l^dag the link's hopping
// term.  With psi = (c_0 + i c_1) / 2 and the link block X[alpha][beta] =
// <c_{2s+alpha} c_{2t+beta}> (entries `stride` apart),
//   T_l = u_l (1/4) (X00 + i e_t X01 + i e_s X10 - e_s e_t X11),
// e = +1 for psi, -1 for psi^dag.
GGF_HD cxd link_term(const cxd* X, size_t stride, int e_s, int e_t, cxd u) {
    const cxd v = X[0] + cxd{0.0, (double)e_t} * X[stride] + cxd{0.0, (double)e_s} * X[2 * stride] +
                  (-(double)(e_s * e_t)) * X[3 * stride];
    return u * (0.25 * v);
}

// Chain c, link l: T_l from the combined link block blk [n][n_links][2][2]
// into out[c][l], and from the per-pair blocks pair_blk
// [n][n_links][2][2][K][K] into pair_out[c][l][n][m] (either pair of pointers
// may be null); q [V] the sites' physical charges.
GGF_HD void link_term_item(const DevConst& dc, int c, int l, const void* links, const int* q, const cxd* blk,
                           const cxd* pair_blk, cxd* out, cxd* pair_out) {
    const Geometry& g = dc.g;
    int a0, b0;
    link_ends(g, l, a0, b0);
    const int s = a0 / g.B, t = b0 / g.B;
    const int e_s = q[s] > 0 ? 1 : -1, e_t = q[t] > 0 ? -1 : 1;
    const size_t cl = (size_t)c * g.n_links + l;
    cxd u;
    if (g.group == GGF_Z2) {
        u = cxd{(double)((const int8_t*)links)[cl], 0.0};
    } else {
        const double th = ((const double*)links)[cl];
        u = cxd{cos(th), sin(th)};
    }
    if (blk && out) out[cl] = link_term(blk + cl * 4, 1, e_s, e_t, u);
    if (pair_blk && pair_out) {
        const int KK = dc.K * dc.K;
        for (int nm = 0; nm < KK; ++nm)
            pair_out[cl * KK + nm] = link_term(pair_blk + cl * 4 * KK + nm, (size_t)KK, e_s, e_t, u);
    }
}

// ---- nearest-neighbour four-point function ----------------------------------
// <c_2s c_2s+1 c_2t c_2t+1> of link l = (s -> t) for chain c into out[c][l]:
// per pair, Wick's theorem gives Pf(-i G4) = -Pf(G4) with G4 the physical
// covariance A + B W B^T on those four Majoranas (blocks (s, s), (t, t) and
// (s, t); (t, s) = -(s, t)^T), and the pairs combine with lambda_n^* lambda_m
// N_nm / N(G) as for the bilinears.  A self-link (s = t) gives -1.
template <class RW, class CW, int BW>
__host__ __device__ void fermion4_item(const DevConst& dc, int c, int l, const RW* Wr, const CW* Wc,
                                       const cxd* ell, cxd* out, cxd* pair_out = nullptr) {
    const Geometry& g = dc.g;
    int a0, b0;
    link_ends(g, l, a0, b0);
    const int s = a0 / g.B, t = b0 / g.B;
    const int K = dc.K;
    const cxd* el = ell + (size_t)c * dc.P;
    double amax, iden;
    pair_scale(dc, el, amax, iden);
    // per-pair parts pair_out[c][l][n][m] = N_nm(G) <c c c c>_nm / N(G)
    cxd* q = pair_out ? pair_out + ((size_t)c * g.n_links + l) * K * K : nullptr;
    if (s == t) {   // c_2s c_2s+1 c_2s c_2s+1 = -1
        if (out) out[(size_t)c * g.n_links + l] = cxd{-1.0, 0.0};
        if (q)
            for (int p = 0; p < dc.P; ++p) {
                int n, m;
                pair_nm(K, p, n, m);
                const cxd Np = pair_norm(dc, el, p, amax, iden);
                q[n * K + m] = -1.0 * Np;
                if (p >= K) q[m * K + n] = -1.0 * conjg(Np);
            }
        return;
    }
    const size_t NN = (size_t)g.N * g.N;
    const double* As = dc.Ap + (size_t)s * 4;
    const double* At = dc.Ap + (size_t)t * 4;
    cxd acc = {0.0, 0.0};
    for (int p = 0; p < dc.P; ++p) {
        const bool cplx = p >= K;
        const cxd Np = pair_norm(dc, el, p, amax, iden);
        const cxd E = dc.w[p] * Np;
        int n, m;
        pair_nm(K, p, n, m);
        cxd Xss[2][2], Xtt[2][2], Xst[2][2];
        if (cplx) {
            const CW* W = Wc + ((size_t)c * dc.Kc + (p - K)) * NN;
            coupled_block<CW, BW>(dc, W, s, s, Xss);
            coupled_block<CW, BW>(dc, W, t, t, Xtt);
            coupled_block<CW, BW>(dc, W, s, t, Xst);
        } else {
            const RW* W = Wr + ((size_t)c * K + p) * NN;
            coupled_block<RW, BW>(dc, W, s, s, Xss);
            coupled_block<RW, BW>(dc, W, t, t, Xtt);
            coupled_block<RW, BW>(dc, W, s, t, Xst);
        }
        // both orders of a complex pair: (n, m) with E / 2 and X, (m, n) with
        // conj(E) / 2 and conj(X); a diagonal pair once with E
        for (int ord = 0; ord < (cplx ? 2 : 1); ++ord) {
            auto cj = [&](cxd v) { return ord ? conjg(v) : v; };
            const cxd g01 = cj(Xss[0][1]) + cxd{As[1], 0.0};
            const cxd g23 = cj(Xtt[0][1]) + cxd{At[1], 0.0};
            const cxd g02 = cj(Xst[0][0]), g03 = cj(Xst[0][1]), g12 = cj(Xst[1][0]), g13 = cj(Xst[1][1]);
            const cxd pf = g01 * g23 - g02 * g13 + g03 * g12;
            const cxd wgt = cplx ? (ord ? 0.5 * conjg(E) : 0.5 * E) : E;
            acc -= wgt * pf;
            if (q) {
                if (ord) q[m * K + n] = -1.0 * (conjg(Np) * pf);
                else q[n * K + m] = -1.0 * (Np * pf);
            }
        }
    }
    if (out) out[(size_t)c * g.n_links + l] = acc;
}

// ---- score of the site blocks ------------------------------------------------
// d log N(G) / d D_s[i][j] of chain c and site s into out[c][s][i][j] (B x B,
// FP64, entries treated as independent).  For pure site states
// N_nm(G) = const Pf(D + O Gamma_X O^T) and d log Pf(M) = (1/2) tr(M^{-1} dM),
// so the score is Re sum_p w_p (N_p / N(G)) (1/2) W_p[s, s]^T (the (m, n)
// order of a pair n < m is the conjugate term, hence the real part).
template <class RW, class CW>
__host__ __device__ void score_item(const DevConst& dc, int c, int s, const RW* Wr, const CW* Wc, const cxd* ell,
                                    double* out) {
    const Geometry& g = dc.g;
    const int B = g.B, N = g.N;
    const size_t NN = (size_t)N * N;
    const cxd* el = ell + (size_t)c * dc.P;
    double amax, iden;
    pair_scale(dc, el, amax, iden);
    double* o = out + ((size_t)c * g.V + s) * B * B;
    for (int e = 0; e < B * B; ++e) o[e] = 0.0;
    for (int p = 0; p < dc.P; ++p) {
        const cxd E = dc.w[p] * pair_norm(dc, el, p, amax, iden);
        for (int i = 0; i < B; ++i)
            for (int j = 0; j < B; ++j) {
                const size_t off = (size_t)(s * B + j) * N + (size_t)s * B + i;     // W_p[sB + j][sB + i]
                const cxd wv = p < dc.K ? Sc<RW>::to(Wr[((size_t)c * dc.K + p) * NN + off])
                                        : Sc<CW>::to(Wc[((size_t)c * dc.Kc + (p - dc.K)) * NN + off]);
                o[i * B + j] += 0.5 * (E * wv).x;
            }
    }
}

// ---- score of the link blocks ------------------------------------------------
// Pair p, link l of chain c: out[c][p][l] (R x R complex, R = r) =
// (w_p N_p / N(G)) (1/2) (O_l^T W_p[l, l] O_l)^T with W_p[l, l] the block of the
// pair's inverse on the link's Majoranas and O_l the link's twist, so that
// d log N(G) = Re sum_p sum_l tr(U_p[l]^T dGamma_X^p[l]) + the pair constants'
// terms (none for K = 1, where this is the gradient for the bond blocks).
template <class RW, class CW, int R>
__host__ __device__ void link_score_item(const DevConst& dc, int c, int p, int l, const void* links, const RW* Wr,
                                         const CW* Wc, const cxd* ell, cxd* out) {
    const Geometry& g = dc.g;
    const size_t NN = (size_t)g.N * g.N;
    const cxd* el = ell + (size_t)c * dc.P;
    double amax, iden;
    pair_scale(dc, el, amax, iden);
    const cxd f = 0.5 * (dc.w[p] * pair_norm(dc, el, p, amax, iden));
    // the link's twist O (rows), source end positions 0 .. h2 - 1
    double O[R][R];
    for (int x = 0; x < R; ++x)
        for (int y = 0; y < R; ++y) O[x][y] = 0.0;
    if (g.group == GGF_SU2) {
        double Rq[16];
        doublet_rotation(link_quat(g, links, c, l), Rq);
        for (int x = 0; x < R; ++x) {
            if (x < 4)
                for (int a = 0; a < 4; ++a) O[x][a] = Rq[x * 4 + a];
            else
                O[x][x] = 1.0;
        }
    } else {
        double gval, theta;
        link_value<double>(dc, links, c, l, gval, theta);
        for (int x = 0; x < R; ++x) {
            double cs = 1.0, sn = 0.0;
            if (g.group == GGF_U1 && x < g.h2) {
                cs = cos(g.q[x >> 1] * theta);
                sn = sin(g.q[x >> 1] * theta);
            }
            int i0, i1;
            double c0, c1;
            twist_row(g, x, gval, cs, sn, i0, c0, i1, c1);
            O[x][i0] += c0;
            if (i1 != i0) O[x][i1] += c1;
        }
    }
    int a0, b0;
    link_ends(g, l, a0, b0);
    cxd Wl[R][R];
    for (int a = 0; a < R; ++a)
        for (int b = 0; b < R; ++b) {
            const size_t off = (size_t)link_majorana(g, a0, b0, a) * g.N + link_majorana(g, a0, b0, b);
            Wl[a][b] = p < dc.K ? Sc<RW>::to(Wr[((size_t)c * dc.K + p) * NN + off])
                                : Sc<CW>::to(Wc[((size_t)c * dc.Kc + (p - dc.K)) * NN + off]);
        }
    cxd* o = out + (((size_t)c * dc.P + p) * g.n_links + l) * R * R;
    for (int x = 0; x < R; ++x)
        for (int y = 0; y < R; ++y) {
            // (O^T W O)[y][x] = sum_ab O[a][y] W[a][b] O[b][x]
            cxd v = {0.0, 0.0};
            for (int a = 0; a < R; ++a) {
                if (O[a][y] == 0.0) continue;
                cxd t = {0.0, 0.0};
                for (int b = 0; b < R; ++b) t += O[b][x] * Wl[a][b];
                v += O[a][y] * t;
            }
            o[x * R + y] = f * v;
        }
}

}  // namespace
