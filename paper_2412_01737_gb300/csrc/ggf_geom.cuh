// Lattice geometry and the twisted link blocks O Gamma_X O^T (Sec. 3.1,
// Sec. 5), shared by the assembly, sampler and observable kernels (host and
// device callable).
#pragma once
#include "ggf_ctx.h"

namespace {
// ---- geometry helpers -------------------------------------------------------
GGF_HD void link_of(const Geometry& g, int i, int& link, int& pos) {
    int s = i / g.B, li = i - s * g.B, e = li / g.h2, k = li - e * g.h2;
    int d = e >> 1;
    if (e & 1) {           // +d end: source of link (s, d)
        link = 2 * s + d;
        pos = k;
    } else {               // -d end: target of link (s - e_d, d)
        int x = s % g.L, y = s / g.L;
        int src = d == 0 ? y * g.L + (x + g.L - 1) % g.L : ((y + g.L - 1) % g.L) * g.L + x;
        link = 2 * src + d;
        pos = g.h2 + k;
    }
}

// Row of the twist O restricted to link position x: up to two (index, coef).
GGF_HD void twist_row(const Geometry& g, int x, double gval, double c, double s,
                                          int& i0, double& c0, int& i1, double& c1) {
    if (x >= g.h2) { i0 = x; c0 = 1.0; i1 = x; c1 = 0.0; return; }
    if (g.group == GGF_Z2) { i0 = x; c0 = gval; i1 = x; c1 = 0.0; return; }
    int j = x >> 1;
    i0 = 2 * j; i1 = 2 * j + 1;
    if ((x & 1) == 0) { c0 = c; c1 = s; } else { c0 = -s; c1 = c; }
}

template <class T>
GGF_HD T bond_elem(const DevConst& dc, int pair, int link, int x, int y);
template <>
GGF_HD double bond_elem<double>(const DevConst& dc, int pair, int link, int x, int y) {
    return dc.Gr[((size_t)pair * dc.g.n_links + link) * dc.g.r * dc.g.r + x * dc.g.r + y];
}
template <>
GGF_HD cxd bond_elem<cxd>(const DevConst& dc, int pair, int link, int x, int y) {
    return dc.Gc[((size_t)pair * dc.g.n_links + link) * dc.g.r * dc.g.r + x * dc.g.r + y];
}

GGF_HD double mulc(double c, double v) { return c * v; }
GGF_HD cxd mulc(double c, cxd v) { return c * v; }

// twisted link block element (O G O^T)[x][y] for link value (Z2 g / U(1) theta)
template <class T>
__host__ __device__ T twisted(const DevConst& dc, int pair, int link, int x, int y, double gval, double theta) {
    const Geometry& g = dc.g;
    double cx_ = 1, sx_ = 0, cy_ = 1, sy_ = 0;
    if (g.group == GGF_U1) {
        if (x < g.h2) sincos(g.q[x >> 1] * theta, &sx_, &cx_);
        if (y < g.h2) sincos(g.q[y >> 1] * theta, &sy_, &cy_);
    }
    int a0, a1, b0, b1;
    double ca0, ca1, cb0, cb1;
    twist_row(g, x, gval, cx_, sx_, a0, ca0, a1, ca1);
    twist_row(g, y, gval, cy_, sy_, b0, cb0, b1, cb1);
    T v = mulc(ca0 * cb0, bond_elem<T>(dc, pair, link, a0, b0));
    if (cb1 != 0.0) v += mulc(ca0 * cb1, bond_elem<T>(dc, pair, link, a0, b1));
    if (ca1 != 0.0) {
        v += mulc(ca1 * cb0, bond_elem<T>(dc, pair, link, a1, b0));
        if (cb1 != 0.0) v += mulc(ca1 * cb1, bond_elem<T>(dc, pair, link, a1, b1));
    }
    return v;
}

// Same element with the twist's cos/sin precomputed: cs[2 j], cs[2 j + 1] =
// cos, sin of q_j theta for source-end mode j (U(1); unused for Z2).
template <class T>
__host__ __device__ T twisted_tab(const DevConst& dc, int pair, int link, int x, int y, double gval, const double* cs) {
    const Geometry& g = dc.g;
    double cx_ = 1, sx_ = 0, cy_ = 1, sy_ = 0;
    if (g.group == GGF_U1) {
        if (x < g.h2) { cx_ = cs[2 * (x >> 1)]; sx_ = cs[2 * (x >> 1) + 1]; }
        if (y < g.h2) { cy_ = cs[2 * (y >> 1)]; sy_ = cs[2 * (y >> 1) + 1]; }
    }
    int a0, a1, b0, b1;
    double ca0, ca1, cb0, cb1;
    twist_row(g, x, gval, cx_, sx_, a0, ca0, a1, ca1);
    twist_row(g, y, gval, cy_, sy_, b0, cb0, b1, cb1);
    T v = mulc(ca0 * cb0, bond_elem<T>(dc, pair, link, a0, b0));
    if (cb1 != 0.0) v += mulc(ca0 * cb1, bond_elem<T>(dc, pair, link, a0, b1));
    if (ca1 != 0.0) {
        v += mulc(ca1 * cb0, bond_elem<T>(dc, pair, link, a1, b0));
        if (cb1 != 0.0) v += mulc(ca1 * cb1, bond_elem<T>(dc, pair, link, a1, b1));
    }
    return v;
}

template <class T>
GGF_HD void link_value(const DevConst& dc, const void* links, int cfg, int link,
                                           double& gval, double& theta) {
    if (dc.g.group == GGF_Z2) {
        gval = (double)((const int8_t*)links)[(size_t)cfg * dc.g.n_links + link];
        theta = 0.0;
    } else {
        gval = 1.0;
        theta = ((const double*)links)[(size_t)cfg * dc.g.n_links + link];
    }
}

// ---- SU(2) links ------------------------------------------------------------
// A link value is a unit quaternion q = (a0, a1, a2, a3), the group element
// u = a0 1 + i (a1 sigma_x + a2 sigma_y + a3 sigma_z).  The twist acts on the
// source-end doublet by psi^dag_j -> sum_k psi^dag_k u_kj (the right-regular
// action of App. A), whose Majorana rotation R (4 x 4, row-major) has rows
//   c_2j   -> sum_k  Re u_kj c_2k + Im u_kj c_2k+1,
//   c_2j+1 -> sum_k -Im u_kj c_2k + Re u_kj c_2k+1.

GGF_HD const double* link_quat(const Geometry& g, const void* links, int cfg, int link) {
    return (const double*)links + ((size_t)cfg * g.n_links + link) * 4;
}

// (a0 + i a.s)(b0 + i b.s) = a0 b0 - a.b + i (a0 b + b0 a - a x b).s
GGF_HD void quat_mul(const double* a, const double* b, double* o) {
    o[0] = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
    o[1] = a[0] * b[1] + b[0] * a[1] - (a[2] * b[3] - a[3] * b[2]);
    o[2] = a[0] * b[2] + b[0] * a[2] - (a[3] * b[1] - a[1] * b[3]);
    o[3] = a[0] * b[3] + b[0] * a[3] - (a[1] * b[2] - a[2] * b[1]);
}

// (1/2) tr(u1^dag u2^dag u3 u4): the scalar part of conj(q1) conj(q2) q3 q4.
// The weight is invariant under u_l -> h_t^dag u_l h_s, so the covariant link
// matrix is u^dag and this is the oriented plaquette trace.
GGF_HD double plaquette_su2(const double* q1, const double* q2, const double* q3,
                                                const double* q4) {
    const double c1[4] = {q1[0], -q1[1], -q1[2], -q1[3]}, c2[4] = {q2[0], -q2[1], -q2[2], -q2[3]};
    double a[4], b[4];
    quat_mul(c1, c2, a);
    quat_mul(q3, q4, b);
    return a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
}

GGF_HD void doublet_rotation(const double* q, double* R) {
    // u00 = a0 + i a3, u01 = a2 + i a1, u10 = -a2 + i a1, u11 = a0 - i a3
    const double ure[2][2] = {{q[0], q[2]}, {-q[2], q[0]}};
    const double uim[2][2] = {{q[3], q[1]}, {q[1], -q[3]}};
    for (int j = 0; j < 2; ++j)
        for (int k = 0; k < 2; ++k) {
            R[(2 * j) * 4 + 2 * k] = ure[k][j];
            R[(2 * j) * 4 + 2 * k + 1] = uim[k][j];
            R[(2 * j + 1) * 4 + 2 * k] = -uim[k][j];
            R[(2 * j + 1) * 4 + 2 * k + 1] = ure[k][j];
        }
}

// (O G O^T)[x][y] on one link (n_v = 2: the source end is one doublet at link
// positions 0..3, rotated by R; the target end 4..7 is untouched).
template <class T>
__host__ __device__ T twisted_su2(const DevConst& dc, int pair, int link, int x, int y, const double* R) {
    T v = T{};
    if (x < 4 && y < 4) {
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b) v += mulc(R[x * 4 + a] * R[y * 4 + b], bond_elem<T>(dc, pair, link, a, b));
    } else if (x < 4) {
        for (int a = 0; a < 4; ++a) v += mulc(R[x * 4 + a], bond_elem<T>(dc, pair, link, a, y));
    } else if (y < 4) {
        for (int b = 0; b < 4; ++b) v += mulc(R[y * 4 + b], bond_elem<T>(dc, pair, link, x, b));
    } else {
        v = bond_elem<T>(dc, pair, link, x, y);
    }
    return v;
}

// Trace of the oriented product of link matrices along a closed path
// (Sec. 5.1): mode 0 the R x T rectangle with lower-left corner s (R steps +x,
// T steps +y, R steps -x, T steps -y); mode 1 the loop winding once around
// the torus along y at column x = s.  A forward step contributes the covariant
// link matrix (Z2 g; U(1) e^{i theta}, real part at the end; SU(2) u^dag), a
// backward step its inverse, multiplied in path order.
GGF_HD double loop_value(const Geometry& g, const void* links, int cfg, int s, int R, int T, int mode) {
    const int L = g.L, x = s % L, y = s / L;
    const int n = mode ? L : 2 * (R + T);
    int prod = 1;
    double ang = 0.0;
    double M[4] = {1.0, 0.0, 0.0, 0.0};
    for (int k = 0; k < n; ++k) {
        int l;
        bool fw;
        if (mode) {
            l = 2 * (((y + k) % L) * L + x) + 1;
            fw = true;
        } else if (k < R) {
            l = 2 * (y * L + (x + k) % L);
            fw = true;
        } else if (k < R + T) {
            l = 2 * (((y + k - R) % L) * L + (x + R) % L) + 1;
            fw = true;
        } else if (k < 2 * R + T) {
            l = 2 * (((y + T) % L) * L + (x + 2 * R + T - 1 - k) % L);
            fw = false;
        } else {
            l = 2 * (((y + 2 * R + 2 * T - 1 - k) % L) * L + x) + 1;
            fw = false;
        }
        if (g.group == GGF_Z2) {
            prod *= ((const int8_t*)links)[(size_t)cfg * g.n_links + l];
        } else if (g.group == GGF_U1) {
            const double th = ((const double*)links)[(size_t)cfg * g.n_links + l];
            ang += fw ? th : -th;
        } else {
            const double* q = link_quat(g, links, cfg, l);
            const double st[4] = {q[0], fw ? -q[1] : q[1], fw ? -q[2] : q[2], fw ? -q[3] : q[3]};
            double t[4];
            quat_mul(M, st, t);
            for (int i = 0; i < 4; ++i) M[i] = t[i];
        }
    }
    if (g.group == GGF_Z2) return (double)prod;
    if (g.group == GGF_U1) return cos(ang);
    return M[0];                                     // (1/2) tr of the SU(2) product
}

// Element (i, j) of M_p(G) = D + O(G) Gamma_X^p O(G)^T for configuration cfg
// (T = double for the diagonal pairs, cxd for the pairs n < m, indexed within
// their family).
template <class T>
__host__ __device__ T assemble_elem(const DevConst& dc, const void* links, int cfg, int pair, int i, int j) {
    const Geometry& g = dc.g;
    T v = Sc<T>::zero();
    int si = i / g.B, sj = j / g.B;
    if (si == sj) v = Sc<T>::from(Sc<double>::to(dc.D[((size_t)si * g.B + (i - si * g.B)) * g.B + (j - sj * g.B)]));
    int li, pi, lj, pj;
    link_of(g, i, li, pi);
    link_of(g, j, lj, pj);
    if (li == lj) {
        if (g.group == GGF_SU2) {
            double R[16];
            doublet_rotation(link_quat(g, links, cfg, li), R);
            v += twisted_su2<T>(dc, pair, li, pi, pj, R);
        } else {
            double gv, th;
            link_value<T>(dc, links, cfg, li, gv, th);
            v += twisted<T>(dc, pair, li, pi, pj, gv, th);
        }
    }
    return v;
}

}  // namespace
