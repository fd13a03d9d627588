// Device-side lattice geometry and the twisted link blocks O Gamma_X O^T
// (Sec. 3.1, Sec. 5), shared by the assembly and the sampler kernels.
#pragma once
#include "ggf_ctx.h"

namespace {
// ---- geometry helpers -------------------------------------------------------
__device__ __forceinline__ void link_of(const Geometry& g, int i, int& link, int& pos) {
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
__device__ __forceinline__ void twist_row(const Geometry& g, int x, double gval, double c, double s,
                                          int& i0, double& c0, int& i1, double& c1) {
    if (x >= g.h2) { i0 = x; c0 = 1.0; i1 = x; c1 = 0.0; return; }
    if (g.group == GGF_Z2) { i0 = x; c0 = gval; i1 = x; c1 = 0.0; return; }
    int j = x >> 1;
    i0 = 2 * j; i1 = 2 * j + 1;
    if ((x & 1) == 0) { c0 = c; c1 = s; } else { c0 = -s; c1 = c; }
}

template <class T>
__device__ __forceinline__ T bond_elem(const DevConst& dc, int pair, int link, int x, int y);
template <>
__device__ __forceinline__ double bond_elem<double>(const DevConst& dc, int pair, int link, int x, int y) {
    return dc.Gr[((size_t)pair * dc.g.n_links + link) * dc.g.r * dc.g.r + x * dc.g.r + y];
}
template <>
__device__ __forceinline__ cxd bond_elem<cxd>(const DevConst& dc, int pair, int link, int x, int y) {
    return dc.Gc[((size_t)pair * dc.g.n_links + link) * dc.g.r * dc.g.r + x * dc.g.r + y];
}

__device__ __forceinline__ double mulc(double c, double v) { return c * v; }
__device__ __forceinline__ cxd mulc(double c, cxd v) { return c * v; }

// twisted link block element (O G O^T)[x][y] for link value (Z2 g / U(1) theta)
template <class T>
__device__ T twisted(const DevConst& dc, int pair, int link, int x, int y, double gval, double theta) {
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
__device__ T twisted_tab(const DevConst& dc, int pair, int link, int x, int y, double gval, const double* cs) {
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
__device__ __forceinline__ void link_value(const DevConst& dc, const void* links, int cfg, int link,
                                           double& gval, double& theta) {
    if (dc.g.group == GGF_Z2) {
        gval = (double)((const int8_t*)links)[(size_t)cfg * dc.g.n_links + link];
        theta = 0.0;
    } else {
        gval = 1.0;
        theta = ((const double*)links)[(size_t)cfg * dc.g.n_links + link];
    }
}


}  // namespace
