// Warp-level helpers and per-link pieces of a Metropolis link step, shared by
// the one-link-per-launch kernels (k_sample.cu) and the batched link steps
// on the small matrix W[T, T] (k_batch.cu).
#pragma once
#include "ggf_ctx.h"
#include "ggf_geom.cuh"

namespace {
constexpr int NWARP = 8;

__device__ __forceinline__ double magc(cxd v) { return fabs(v.x) + fabs(v.y); }

// warp argmax over lanes (ties: lowest index).  The result is taken from
// lane 0 so that every lane follows the same pivot even when a NaN makes the
// comparisons inconsistent (the callers branch on it around __syncwarp).
__device__ __forceinline__ int warp_argmax(double v, int idx) {
    for (int o = 16; o > 0; o >>= 1) {
        double ov = __shfl_xor_sync(0xffffffffu, v, o);
        int oi = __shfl_xor_sync(0xffffffffu, idx, o);
        if (ov > v || (ov == v && oi < idx)) { v = ov; idx = oi; }
    }
    return __shfl_sync(0xffffffffu, idx, 0);
}

// Pfaffian of an n x n (n <= 32) antisymmetric matrix in shared memory, by one
// warp (skew Gaussian elimination with pivoting).  A is destroyed.
__device__ cxd warp_pfaffian(cxd* A, int n) {
    const int lane = threadIdx.x & 31;
    cxd res = {1.0, 0.0};
    for (int k = 0; k < n - 1; k += 2) {
        double m = (lane >= k + 1 && lane < n) ? magc(A[lane * n + k]) : -1.0;
        int p = warp_argmax(m, lane);
        const int q = k + 1;
        if (p != q) {
            if (lane >= k && lane < n) {
                cxd t = A[q * n + lane]; A[q * n + lane] = A[p * n + lane]; A[p * n + lane] = t;
            }
            __syncwarp();
            if (lane >= k && lane < n) {
                cxd t = A[lane * n + q]; A[lane * n + q] = A[lane * n + p]; A[lane * n + p] = t;
            }
            __syncwarp();
            res = -res;
        }
        cxd piv = A[q * n + k];
        if (piv.x == 0.0 && piv.y == 0.0) { __syncwarp(); return {0.0, 0.0}; }
        res = res * A[k * n + q];
        const cxd ipiv = cxd{1.0, 0.0} / piv;
        int mm = n - k - 2;
        // multipliers l_i = A[i][k] / A[q][k], one per row, in column k
        // (column k is not read again)
        if (lane < mm) A[(k + 2 + lane) * n + k] = A[(k + 2 + lane) * n + k] * ipiv;
        __syncwarp();
        for (int e = lane; e < mm * mm; e += 32) {
            int i = k + 2 + e / mm, j = k + 2 + e % mm;
            A[i * n + j] += A[i * n + k] * A[j * n + q] - A[i * n + q] * A[j * n + k];
        }
        __syncwarp();
    }
    return res;
}

// Solve [A | B] (r x 2r, row-major, stride 2r) in place by Gauss-Jordan with
// partial pivoting; the right half becomes A^{-1} B.  fcol: r scratch.
__device__ bool warp_solve(cxd* A, int r, cxd* fcol) {
    const int lane = threadIdx.x & 31;
    const int w = 2 * r;
    for (int k = 0; k < r; ++k) {
        double m = (lane >= k && lane < r) ? magc(A[lane * w + k]) : -1.0;
        int p = warp_argmax(m, lane);
        if (p != k) {
            if (lane < w) { cxd t = A[k * w + lane]; A[k * w + lane] = A[p * w + lane]; A[p * w + lane] = t; }
            __syncwarp();
        }
        cxd d = A[k * w + k];
        if (d.x == 0.0 && d.y == 0.0) return false;
        __syncwarp();
        if (lane < w) A[k * w + lane] = A[k * w + lane] / d;
        if (lane < r) fcol[lane] = A[lane * w + k];
        __syncwarp();
        for (int e = lane; e < r * w; e += 32) {
            int i = e / w, j = e % w;
            if (i != k) A[i * w + j] -= fcol[i] * A[k * w + j];
        }
        __syncwarp();
    }
    return true;
}

template <class T>
__device__ __forceinline__ cxd loadc(const T* p) { return Sc<T>::to(*p); }

// Pending-update panels of one (chain, pair): U (N x KRM) followed by V^T
// (N x KRM), K-major (row index first, rank index contiguous); complex
// values are stored as a real plane followed by an imaginary plane, so a
// (chain, pair) block holds 2 (real) or 4 (complex) planes of N * KRM.
template <class T> struct PanelIO {
    typedef typename Sc<T>::R R;
    static constexpr int PLANES = Sc<T>::CPLX ? 2 : 1;
    __device__ static T ld(const R* p, size_t plane, size_t idx);
    __device__ static void st(R* p, size_t plane, size_t idx, T v);
};
template <> __device__ __forceinline__ double PanelIO<double>::ld(const double* p, size_t, size_t i) { return p[i]; }
template <> __device__ __forceinline__ float PanelIO<float>::ld(const float* p, size_t, size_t i) { return p[i]; }
template <> __device__ __forceinline__ cxd PanelIO<cxd>::ld(const double* p, size_t pl, size_t i) { return {p[i], p[pl + i]}; }
template <> __device__ __forceinline__ cxf PanelIO<cxf>::ld(const float* p, size_t pl, size_t i) { return {p[i], p[pl + i]}; }
template <> __device__ __forceinline__ void PanelIO<double>::st(double* p, size_t, size_t i, double v) { p[i] = v; }
template <> __device__ __forceinline__ void PanelIO<float>::st(float* p, size_t, size_t i, float v) { p[i] = v; }
template <> __device__ __forceinline__ void PanelIO<cxd>::st(double* p, size_t pl, size_t i, cxd v) { p[i] = v.x; p[pl + i] = v.y; }
template <> __device__ __forceinline__ void PanelIO<cxf>::st(float* p, size_t pl, size_t i, cxf v) { p[i] = v.x; p[pl + i] = v.y; }

// Majorana offsets of the two ends of link l = 2 s + d: the source end (+d
// end of site s, which carries the twist) and the target end (-d end of the
// neighbour t).  Majorana xi < h2 of the link is a0 + xi, the others b0 + xi - h2.
GGF_HD void link_ends(const Geometry& g, int l, int& a0, int& b0) {
    const int s = l >> 1, d = l & 1, x = s % g.L, y = s / g.L;
    const int t = d == 0 ? y * g.L + (x + 1) % g.L : ((y + 1) % g.L) * g.L + x;
    a0 = s * g.B + (2 * d + 1) * g.h2;
    b0 = t * g.B + (2 * d) * g.h2;
}
GGF_HD int link_majorana(const Geometry& g, int a0, int b0, int xi) {
    return xi < g.h2 ? a0 + xi : b0 + xi - g.h2;
}

// One proposal (Sec. 5.1): accept draw, old and new link value.
struct Proposal {
    double u_acc, g_old, g_new, th_old, th_new;
};

// Philox4x64-10 with counter (sweep, link, 0, 0) and key (seed, chain):
// word 0 -> u_accept, word 1 -> u_propose.  Z2 flips the link; U(1) moves
// theta by width (u - 1/2) and wraps into [0, 2 pi).
__device__ __forceinline__ Proposal draw_proposal(const Geometry& g, const void* links, int c, int l,
                                                  unsigned long long sweep, uint64_t seed, double width,
                                                  uint64_t coff = 0) {
    uint64_t ctr[4] = {(uint64_t)sweep, (uint64_t)l, 0, 0}, out[4];
    philox4x64_10(ctr, seed, coff + (uint64_t)c, out);
    Proposal q;
    q.u_acc = u53(out[0]);
    const double u_prop = u53(out[1]);
    if (g.group == GGF_Z2) {
        double gv = (double)((const int8_t*)links)[(size_t)c * g.n_links + l];
        q.g_old = gv; q.g_new = -gv; q.th_old = 0.0; q.th_new = 0.0;
    } else {
        double th = ((const double*)links)[(size_t)c * g.n_links + l];
        double tn = th + width * (u_prop - 0.5);
        if (tn >= GGF_TWO_PI) tn -= GGF_TWO_PI;
        else if (tn < 0.0) tn += GGF_TWO_PI;
        q.g_old = 1.0; q.g_new = 1.0; q.th_old = th; q.th_new = tn;
    }
    return q;
}

// Change of pair p's twisted link block, Delta = O' G O'^T - O G O^T on the
// r Majoranas of link l (r x r, one warp).
// cs: cos, sin of q_j theta for the old angle (cs[0 .. 2 n_v)) and the new
// one (cs[4 ..]), from twist_table.
__device__ __forceinline__ void pair_delta(const DevConst& dc, int p, int l, const Proposal& q, const double* cs,
                                           cxd* D) {
    const int r = dc.g.r, lane = threadIdx.x & 31;
    for (int e = lane; e < r * r; e += 32) {
        int xi = e / r, yi = e % r;
        cxd nv, ov;
        if (p < dc.K) {
            nv = {twisted_tab<double>(dc, p, l, xi, yi, q.g_new, cs + 4), 0.0};
            ov = {twisted_tab<double>(dc, p, l, xi, yi, q.g_old, cs), 0.0};
        } else {
            nv = twisted_tab<cxd>(dc, p - dc.K, l, xi, yi, q.g_new, cs + 4);
            ov = twisted_tab<cxd>(dc, p - dc.K, l, xi, yi, q.g_old, cs);
        }
        D[e] = nv - ov;
    }
}

// SU(2) proposal (n_v = 2, one doublet per link end), thread-local: with
// Philox words (u_acc, u_prop, u_z, u_phi) of counter (sweep, l, 0, 0) and
// key (seed, chain), g -> r g with r = cos d + i sin d (n . sigma),
// d = width (u_prop - 1/2), n = (sqrt(1 - z^2) cos phi, sqrt(1 - z^2) sin phi, z),
// z = 2 u_z - 1, phi = 2 pi u_phi, renormalised to a unit quaternion.  r and
// r^dag are equally likely (a Haar-symmetric move).  Writes the new
// quaternion and the old and new doublet rotations; returns u_acc.
GGF_HD double draw_su2(const Geometry& g, const void* links, int c, int l,
                                           unsigned long long sweep, uint64_t seed, double width, double* qn,
                                           double* Rold, double* Rnew, uint64_t coff = 0) {
    uint64_t ctr[4] = {(uint64_t)sweep, (uint64_t)l, 0, 0}, out[4];
    philox4x64_10(ctr, seed, coff + (uint64_t)c, out);
    const double d = width * (u53(out[1]) - 0.5);
    const double z = 2.0 * u53(out[2]) - 1.0;
    const double rho = sqrt(fmax(0.0, 1.0 - z * z));
    const double ph = GGF_TWO_PI * u53(out[3]);
    double sd, cd, sp, cp;
    sincos(d, &sd, &cd);
    sincos(ph, &sp, &cp);
    const double r[4] = {cd, sd * rho * cp, sd * rho * sp, sd * z};
    const double* q = link_quat(g, links, c, l);
    double t[4];
    quat_mul(r, q, t);
    const double nrm = sqrt(t[0] * t[0] + t[1] * t[1] + t[2] * t[2] + t[3] * t[3]);
    for (int k = 0; k < 4; ++k) qn[k] = t[k] / nrm;
    doublet_rotation(q, Rold);
    doublet_rotation(qn, Rnew);
    return u53(out[0]);
}

// Delta of pair p for an SU(2) proposal (rotations Rold, Rnew of the source
// doublet), r x r, one warp.
__device__ __forceinline__ void pair_delta_su2(const DevConst& dc, int p, int l, const double* Rold,
                                               const double* Rnew, cxd* D) {
    const int r = dc.g.r, lane = threadIdx.x & 31;
    for (int e = lane; e < r * r; e += 32) {
        int xi = e / r, yi = e % r;
        cxd nv, ov;
        if (p < dc.K) {
            nv = {twisted_su2<double>(dc, p, l, xi, yi, Rnew), 0.0};
            ov = {twisted_su2<double>(dc, p, l, xi, yi, Rold), 0.0};
        } else {
            nv = twisted_su2<cxd>(dc, p - dc.K, l, xi, yi, Rnew);
            ov = twisted_su2<cxd>(dc, p - dc.K, l, xi, yi, Rold);
        }
        D[e] = nv - ov;
    }
}

// cos, sin of q_j theta for the old and the new angle of a U(1) proposal
// (threads 0 .. 2 n_v - 1 of the block; cs holds 8 doubles).
__device__ __forceinline__ void twist_table(const Geometry& g, const Proposal& q, double* cs) {
    const int t = threadIdx.x;
    if (g.group == GGF_U1 && t < 2 * g.n_v) {
        const int j = t % g.n_v, nw = t / g.n_v;
        double sv, cv;
        sincos(g.q[j] * (nw ? q.th_new : q.th_old), &sv, &cv);
        cs[4 * nw + 2 * j] = cv;
        cs[4 * nw + 2 * j + 1] = sv;
    }
}

// Pf(M') / Pf(M) = Pf([[Delta, -1], [1, W_SS]]) (r/2 = 2 n_v even: no extra
// sign), one warp; Bw is 2r x 2r scratch.
__device__ __forceinline__ cxd bordered_ratio(const cxd* D, const cxd* Ws, cxd* Bw, int r) {
    const int lane = threadIdx.x & 31, n2 = 2 * r;
    // a non-finite block (an inverse that overflowed) gives ratio 0: the
    // proposal is rejected
    bool fin = true;
    for (int e = lane; e < r * r; e += 32)
        fin = fin && isfinite(Ws[e].x) && isfinite(Ws[e].y) && isfinite(D[e].x) && isfinite(D[e].y);
    if (!__all_sync(0xffffffffu, fin)) return {0.0, 0.0};
    for (int e = lane; e < n2 * n2; e += 32) {
        int i = e / n2, j = e % n2;
        cxd v = {0.0, 0.0};
        if (i < r && j < r) v = D[i * r + j];
        else if (i >= r && j >= r) v = Ws[(i - r) * r + (j - r)];
        else if (i < r && j == i + r) v = {-1.0, 0.0};
        else if (i >= r && j == i - r) v = {1.0, 0.0};
        Bw[e] = v;
    }
    __syncwarp();
    return warp_pfaffian(Bw, n2);
}

// Ordered Gaussian indices (n, m) of pair p: p < K is (p, p); the pairs n < m
// follow in lexicographic order.
GGF_HD void pair_nm(int K, int p, int& n, int& m) {
    if (p < K) { n = m = p; return; }
    int k = p - K;
    n = 0;
    while (k >= K - 1 - n) { k -= K - 1 - n; ++n; }
    m = n + 1 + k;
}

// Scale of the pair terms of one configuration: amax = max_p Re(logc_p + ell_p)
// and 1 / (N(G) e^{-amax}), N(G) = Re sum_p w_p e^{logc_p + ell_p}; then
// pair_norm gives N_nm(G) / N(G) for pair p (diagonal pairs real).
GGF_HD void pair_scale(const DevConst& dc, const cxd* ell_c, double& amax, double& iden) {
    amax = -INFINITY;
    for (int p = 0; p < dc.P; ++p) amax = fmax(amax, dc.logc[p].x + ell_c[p].x);
    double den = 0.0;
    for (int p = 0; p < dc.P; ++p) {
        cxd e = dc.logc[p] + ell_c[p];
        if (p < dc.K) e.y = 0.0;
        e.x -= amax;
        den += (dc.w[p] * cexp_(e)).x;
    }
    iden = 1.0 / den;
}
GGF_HD cxd pair_norm(const DevConst& dc, const cxd* ell_c, int p, double amax, double iden) {
    cxd e = dc.logc[p] + ell_c[p];
    if (p < dc.K) e.y = 0.0;
    e.x -= amax;
    return iden * cexp_(e);
}

// Numerator and denominator of N(G')/N(G) = Re sum_p w_p e^{logc_p + ell_p} rho_p
// / Re sum_p w_p e^{logc_p + ell_p}, scaled by the largest modulus (FP64).
__device__ __forceinline__ void combine_pairs(const DevConst& dc, const cxd* ell_c, const cxd* rho, double& sn,
                                              double& so) {
    double amax = -INFINITY;
    for (int p = 0; p < dc.P; ++p) amax = fmax(amax, dc.logc[p].x + ell_c[p].x);
    so = 0.0;
    sn = 0.0;
    for (int p = 0; p < dc.P; ++p) {
        cxd e = dc.logc[p] + ell_c[p];
        if (p < dc.K) e.y = 0.0;
        e.x -= amax;
        cxd tt = dc.w[p] * cexp_(e);
        so += tt.x;
        sn += (tt * rho[p]).x;
    }
}

// Z = (1 + Delta W_SS)^{-1} Delta (r x r) into Zout, one warp; Aug is r x 2r
// scratch, fcol r.  Returns false for a singular system.
__device__ __forceinline__ bool pair_z(const cxd* D, const cxd* Ws, cxd* Aug, cxd* fcol, int r, cxd* Zout) {
    const int lane = threadIdx.x & 31, w2 = 2 * r;
    for (int e = lane; e < r * w2; e += 32) {
        int i = e / w2, j = e % w2;
        cxd v;
        if (j < r) {
            v = {i == j ? 1.0 : 0.0, 0.0};
            for (int z = 0; z < r; ++z) v += D[i * r + z] * Ws[z * r + j];
        } else {
            v = D[i * r + (j - r)];
        }
        Aug[e] = v;
    }
    __syncwarp();
    const bool ok = warp_solve(Aug, r, fcol);
    for (int e = lane; e < r * r; e += 32) Zout[e] = Aug[(e / r) * w2 + r + e % r];
    __syncwarp();
    return ok;
}

// ell_p += log rho_p: modulus only for diagonal pairs, phase wrapped into
// (-pi, pi] for pairs n < m.
__device__ __forceinline__ void ell_add(cxd& el, cxd rho, bool real_pair) {
    cxd lr = clog_(rho);
    if (real_pair) {
        el.x += lr.x;
    } else {
        el = el + lr;
        if (el.y > M_PI) el.y -= 2 * M_PI;
        else if (el.y <= -M_PI) el.y += 2 * M_PI;
    }
}

}  // namespace
