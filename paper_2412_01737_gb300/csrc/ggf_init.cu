// Host-side set-up of the per-pair constants (Sec. 5), done once per
// ggf_init_gaussians call in FP64.  Small dense complex algebra on r x r
// link blocks only (r = 4 n_v <= 8).
//
// For a pair (n, m) and one link with bond covariances Gn, Gm:
//  * X = |b_n><b_m| / <b_m|b_n> is a Gaussian operator; with F = -i Gamma its
//    covariance is  G_nm = i [1 - (1 - Fn)(1 + Fm Fn)^{-1}(1 - Fm)]
//    (composition of Gaussian operators, Bravyi-Gosset);  G_nn = Gn.
//  * tr(rho_a rho_b) = 2^{-h} Pf(Ga) Pf(Ga + Gb), h = r/2 modes (Sec. 3.2).
//  * <b_m|b_n> from the reference b_0 with <b_k|b_0> > 0 (Sec. 5):
//    <b_0|b_m><b_m|b_n><b_n|b_0> = tr(rho_0 rho_m rho_n)
//       = tr(rho_m rho_n) 2^{-h} Pf(G0) Pf(G0 + G(ket m, bra n)).
// Globally N_nm(G) = <B_m|B_n> tr(sigma_D(G) X_nm) with sigma_D the virtual
// reduced state of the twisted sites; for the rank-one X,
//   tr(sigma X) = 2^{-n_virt} Pf(Gamma_X) Pf(D + O Gamma_X O^T)  (site-major),
// and Pf(Gamma_X) = sign(link-major -> site-major) prod_l Pf(G_l).
#include <complex>
#include <cstring>
#include <string>
#include <vector>
#include "ggf_ctx.h"

typedef std::complex<double> zc;

namespace {

struct Mat {
    int n;
    std::vector<zc> a;
    explicit Mat(int n_ = 0) : n(n_), a((size_t)n_ * n_, 0.0) {}
    zc& operator()(int i, int j) { return a[(size_t)i * n + j]; }
    zc operator()(int i, int j) const { return a[(size_t)i * n + j]; }
};

Mat eye(int n) {
    Mat m(n);
    for (int i = 0; i < n; ++i) m(i, i) = 1.0;
    return m;
}
Mat mul(const Mat& A, const Mat& B) {
    Mat C(A.n);
    for (int i = 0; i < A.n; ++i)
        for (int k = 0; k < A.n; ++k) {
            zc v = A(i, k);
            if (v == 0.0) continue;
            for (int j = 0; j < A.n; ++j) C(i, j) += v * B(k, j);
        }
    return C;
}
Mat add(const Mat& A, const Mat& B, zc s = 1.0) {
    Mat C(A.n);
    for (size_t i = 0; i < A.a.size(); ++i) C.a[i] = A.a[i] + s * B.a[i];
    return C;
}
Mat scale(const Mat& A, zc s) {
    Mat C(A.n);
    for (size_t i = 0; i < A.a.size(); ++i) C.a[i] = s * A.a[i];
    return C;
}
// Gauss-Jordan inverse with partial pivoting; returns false if singular.
bool inverse(Mat A, Mat& out) {
    int n = A.n;
    out = eye(n);
    for (int k = 0; k < n; ++k) {
        int p = k;
        for (int i = k + 1; i < n; ++i)
            if (std::abs(A(i, k)) > std::abs(A(p, k))) p = i;
        if (std::abs(A(p, k)) == 0.0) return false;
        if (p != k)
            for (int j = 0; j < n; ++j) { std::swap(A(k, j), A(p, j)); std::swap(out(k, j), out(p, j)); }
        zc d = A(k, k);
        for (int j = 0; j < n; ++j) { A(k, j) /= d; out(k, j) /= d; }
        for (int i = 0; i < n; ++i) {
            if (i == k) continue;
            zc f = A(i, k);
            if (f == 0.0) continue;
            for (int j = 0; j < n; ++j) { A(i, j) -= f * A(k, j); out(i, j) -= f * out(k, j); }
        }
    }
    return true;
}
// Pfaffian by skew Gaussian elimination with pivoting (Parlett-Reid), full storage.
zc pfaffian(Mat A) {
    int n = A.n;
    if (n % 2) return 0.0;
    zc res = 1.0;
    for (int k = 0; k < n - 1; k += 2) {
        int p = k + 1;
        for (int i = k + 2; i < n; ++i)
            if (std::abs(A(i, k)) > std::abs(A(p, k))) p = i;
        if (p != k + 1) {
            int q = k + 1;
            for (int j = 0; j < n; ++j) std::swap(A(q, j), A(p, j));
            for (int i = 0; i < n; ++i) std::swap(A(i, q), A(i, p));
            res = -res;
        }
        zc piv = A(k + 1, k);
        if (std::abs(piv) == 0.0) return 0.0;
        res *= A(k, k + 1);
        for (int i = k + 2; i < n; ++i) {
            zc ti = A(i, k) / piv, ci = A(i, k + 1);
            for (int j = k + 2; j < n; ++j) {
                zc tj = A(j, k) / piv, cj = A(j, k + 1);
                A(i, j) += ti * cj - ci * tj;
            }
        }
    }
    return res;
}

Mat from_real(const double* p, int n) {
    Mat m(n);
    for (int i = 0; i < n * n; ++i) m.a[i] = p[i];
    return m;
}

// covariance of |ket><bra| / <bra|ket>
bool transition(const Mat& Gket, const Mat& Gbra, Mat& out) {
    int n = Gket.n;
    Mat I = eye(n);
    zc mi(0.0, -1.0);
    Mat Fk = scale(Gket, mi), Fb = scale(Gbra, mi);
    Mat inv;
    if (!inverse(add(I, mul(Fb, Fk)), inv)) return false;
    Mat t = mul(mul(add(I, Fk, -1.0), inv), add(I, Fb, -1.0));
    out = scale(add(I, t, -1.0), zc(0.0, 1.0));
    return true;
}

zc trace_pair(const Mat& Ga, const Mat& Gb) {
    int h = Ga.n / 2;
    return std::pow(2.0, -h) * pfaffian(Ga) * pfaffian(add(Ga, Gb));
}

bool check_pure(const double* G, int n, double tol) {
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            if (std::abs(G[i * n + j] + G[j * n + i]) > tol) return false;
            double s = 0.0;
            for (int k = 0; k < n; ++k) s += G[i * n + k] * G[j * n + k];
            if (std::abs(s - (i == j ? 1.0 : 0.0)) > tol) return false;
        }
    return true;
}

}  // namespace

// sign of the permutation taking link-major virtual Majoranas to site-major
static int link_to_site_sign(const Geometry& g) {
    std::vector<int> pos;  // pos[k] = site-major index of the k-th link-major Majorana
    pos.reserve(g.N);
    for (int l = 0; l < g.n_links; ++l) {
        int s = l / 2, d = l % 2, x = s % g.L, y = s / g.L;
        int t = d == 0 ? y * g.L + (x + 1) % g.L : ((y + 1) % g.L) * g.L + x;
        int a0 = s * g.B + (2 * d + 1) * g.h2, b0 = t * g.B + (2 * d) * g.h2;
        for (int k = 0; k < g.h2; ++k) pos.push_back(a0 + k);
        for (int k = 0; k < g.h2; ++k) pos.push_back(b0 + k);
    }
    std::vector<char> seen(g.N, 0);
    int cycles = 0;
    for (int i = 0; i < g.N; ++i) {
        if (seen[i]) continue;
        ++cycles;
        for (int j = i; !seen[j]; j = pos[j]) seen[j] = 1;
    }
    return ((g.N - cycles) % 2) ? -1 : 1;
}

ggf_status ggf_build_constants(ggf_ctx* ctx, const double* gamma_site, int K,
                               const double* gamma_bond, const double* lambda) {
    const Geometry& g = ctx->g;
    const int m_s = 2 + g.B, r = g.r, nl = g.n_links, h = r / 2;
    for (int s = 0; s < g.V; ++s)
        if (!check_pure(gamma_site + (size_t)s * m_s * m_s, m_s, 1e-8))
            return ggf_fail(ctx, GGF_EINVAL, "gamma_site[" + std::to_string(s) + "] is not a pure covariance");
    for (int n = 0; n < K; ++n)
        for (int l = 0; l < nl; ++l)
            if (!check_pure(gamma_bond + ((size_t)n * nl + l) * r * r, r, 1e-8))
                return ggf_fail(ctx, GGF_EINVAL, "gamma_bond is not a pure covariance");
    const int Kc = K * (K - 1) / 2, P = K + Kc;
    ctx->K = K; ctx->Kc = Kc; ctx->P = P;
    ctx->pair_n.clear(); ctx->pair_m.clear();
    for (int n = 0; n < K; ++n) { ctx->pair_n.push_back(n); ctx->pair_m.push_back(n); }
    for (int n = 0; n < K; ++n)
        for (int m = n + 1; m < K; ++m) { ctx->pair_n.push_back(n); ctx->pair_m.push_back(m); }
    const double n_virt = 0.5 * g.N;
    const int sigma = link_to_site_sign(g);
    std::vector<cxd> logc(P), w(P);
    std::vector<cxd> Gc((size_t)std::max(Kc, 1) * nl * r * r);
    auto bond = [&](int n, int l) { return from_real(gamma_bond + ((size_t)n * nl + l) * r * r, r); };
    for (int p = 0; p < P; ++p) {
        int n = ctx->pair_n[p], m = ctx->pair_m[p];
        zc ln = std::conj(std::complex<double>(lambda[2 * n], lambda[2 * n + 1]));
        zc lm(lambda[2 * m], lambda[2 * m + 1]);
        if (n == m) {
            w[p] = {std::norm(lm), 0.0};
            logc[p] = {-n_virt * std::log(2.0), 0.0};
            continue;
        }
        zc wv = 2.0 * ln * lm;
        w[p] = {wv.real(), wv.imag()};
        zc lg = 0.0;         // log <B_m|B_n> + log prod Pf(G_l)
        double sgn_re = sigma;
        zc pf_prod = sigma;
        for (int l = 0; l < nl; ++l) {
            Mat G0 = bond(0, l), Gn = bond(n, l), Gm = bond(m, l);
            Mat Gx, Gmn;
            if (!transition(Gn, Gm, Gx) || !transition(Gm, Gn, Gmn))
                return ggf_fail(ctx, GGF_ESINGULAR, "orthogonal bond states: <b_m|b_n> = 0");
            zc tmn = trace_pair(Gm, Gn), t0m = trace_pair(G0, Gm), t0n = trace_pair(G0, Gn);
            if (t0m.real() <= 0.0 || t0n.real() <= 0.0)
                return ggf_fail(ctx, GGF_ESINGULAR, "bond state orthogonal to the reference b_0");
            zc num = tmn * std::pow(2.0, -h) * pfaffian(G0) * pfaffian(add(G0, Gmn));
            zc ov = num / std::sqrt(t0m.real() * t0n.real());     // <b_m|b_n>
            lg += std::log(ov);
            pf_prod *= pfaffian(Gx);
            for (int i = 0; i < r * r; ++i) {
                cxd v = {Gx.a[i].real(), Gx.a[i].imag()};
                Gc[((size_t)(p - K) * nl + l) * r * r + i] = v;
            }
        }
        (void)sgn_re;
        // pf_prod is +-1 up to rounding; keep its phase exactly as +-1
        double ps = pf_prod.real() >= 0 ? 1.0 : -1.0;
        zc lc = lg + std::log(zc(ps, 0.0)) - n_virt * std::log(2.0);
        logc[p] = {lc.real(), lc.imag()};
    }
    // device constants
    ggf_free_consts(ctx);
    std::vector<double> D((size_t)g.V * g.B * g.B), Gr((size_t)K * nl * r * r);
    for (int s = 0; s < g.V; ++s)
        for (int i = 0; i < g.B; ++i)
            for (int j = 0; j < g.B; ++j)
                D[((size_t)s * g.B + i) * g.B + j] = gamma_site[((size_t)s * m_s + 2 + i) * m_s + 2 + j];
    std::memcpy(Gr.data(), gamma_bond, Gr.size() * sizeof(double));
    // physical block A_s (2 x 2) and physical-virtual coupling B_s (2 x B) of
    // every site, for the fermionic observables
    std::vector<double> Ap((size_t)g.V * 4), Bp((size_t)g.V * 2 * g.B);
    for (int s = 0; s < g.V; ++s)
        for (int a = 0; a < 2; ++a) {
            for (int b = 0; b < 2; ++b) Ap[(size_t)s * 4 + a * 2 + b] = gamma_site[((size_t)s * m_s + a) * m_s + b];
            for (int j = 0; j < g.B; ++j)
                Bp[((size_t)s * 2 + a) * g.B + j] = gamma_site[((size_t)s * m_s + a) * m_s + 2 + j];
        }
    GGF_CK(cudaMalloc(&ctx->d_D, D.size() * sizeof(double)));
    GGF_CK(cudaMalloc(&ctx->d_Gr, Gr.size() * sizeof(double)));
    GGF_CK(cudaMalloc(&ctx->d_Gc, Gc.size() * sizeof(cxd)));
    GGF_CK(cudaMalloc(&ctx->d_Ap, Ap.size() * sizeof(double)));
    GGF_CK(cudaMalloc(&ctx->d_Bp, Bp.size() * sizeof(double)));
    GGF_CK(cudaMalloc(&ctx->d_logc, P * sizeof(cxd)));
    GGF_CK(cudaMalloc(&ctx->d_w, P * sizeof(cxd)));
    GGF_CK(cudaMemcpy(ctx->d_D, D.data(), D.size() * sizeof(double), cudaMemcpyHostToDevice));
    GGF_CK(cudaMemcpy(ctx->d_Gr, Gr.data(), Gr.size() * sizeof(double), cudaMemcpyHostToDevice));
    GGF_CK(cudaMemcpy(ctx->d_Gc, Gc.data(), Gc.size() * sizeof(cxd), cudaMemcpyHostToDevice));
    GGF_CK(cudaMemcpy(ctx->d_Ap, Ap.data(), Ap.size() * sizeof(double), cudaMemcpyHostToDevice));
    GGF_CK(cudaMemcpy(ctx->d_Bp, Bp.data(), Bp.size() * sizeof(double), cudaMemcpyHostToDevice));
    GGF_CK(cudaMemcpy(ctx->d_logc, logc.data(), P * sizeof(cxd), cudaMemcpyHostToDevice));
    GGF_CK(cudaMemcpy(ctx->d_w, w.data(), P * sizeof(cxd), cudaMemcpyHostToDevice));
    ctx->logc = logc;
    ctx->w = w;
    ctx->have_gauss = true;
    return GGF_OK;
}
