// Test-only host build of the observable kernels' per-thread code
// (paper_2412_01737_gb300/csrc/ggf_obs.cuh).  It runs the items the GPU
// kernels run, one after another on the CPU, on host arrays laid out as the
// library lays them out on the device, so that tests can check the index
// arithmetic and data layout against the oracle without a GPU.  It is not
// part of the library and nothing in the library calls it.
#include <vector>
#include "../../paper_2412_01737_gb300/csrc/ggf_obs.cuh"

namespace {
DevConst make_dc(int L, int group, int n_v, const int* q, int K, const double* D, const double* Ap,
                 const double* Bp, const double* Gr, const double* Gc, const double* logc, const double* w) {
    DevConst dc;
    Geometry& g = dc.g;
    g.L = L; g.V = L * L; g.n_links = 2 * g.V; g.group = group; g.n_v = n_v;
    g.B = 8 * n_v; g.h2 = 2 * n_v; g.r = 4 * n_v; g.N = g.B * g.V;
    g.q[0] = q[0]; g.q[1] = q[1];
    dc.K = K; dc.Kc = K * (K - 1) / 2; dc.P = dc.K + dc.Kc;
    dc.D = D; dc.Ap = Ap; dc.Bp = Bp; dc.Gr = Gr; dc.Gc = (const cxd*)Gc;
    dc.logc = (const cxd*)logc; dc.w = (const cxd*)w;
    return dc;
}
}  // namespace

extern "C" {

// Constant arrays: D [V][B][B], Ap [V][2][2], Bp [V][2][B], Gr [K][2V][r][r],
// Gc [Kc][2V][r][r] complex, logc [P] and w [P] complex; chains: links as the
// library stores them, Wr [n][K][N][N], Wc [n][Kc][N][N] complex, ell [n][P]
// complex (complex = interleaved re, im).  Outputs as the entry points'.
void emu_electric(int L, int group, int n_v, const int* q, int K, const double* D, const double* Ap,
                  const double* Bp, const double* Gr, const double* Gc, const double* logc, const double* w,
                  int n_chains, const void* links, const double* Wr, const double* Wc, const double* ell,
                  double* out, double* pair_out) {
    DevConst dc = make_dc(L, group, n_v, q, K, D, Ap, Bp, Gr, Gc, logc, w);
    for (int c = 0; c < n_chains; ++c)
        for (int l = 0; l < dc.g.n_links; ++l) {
            if (dc.g.h2 == 2)
                electric_item<double, cxd, 2>(dc, c, l, links, Wr, (const cxd*)Wc, (const cxd*)ell, (cxd*)out,
                                              (cxd*)pair_out);
            else
                electric_item<double, cxd, 4>(dc, c, l, links, Wr, (const cxd*)Wc, (const cxd*)ell, (cxd*)out,
                                              (cxd*)pair_out);
        }
}

void emu_field(int L, int group, int n_v, const int* q, int K, const double* D, const double* Ap,
               const double* Bp, const double* Gr, const double* Gc, const double* logc, const double* w,
               int n_chains, const void* links, const double* Wr, const double* Wc, const double* ell, double* out,
               double* pairs) {
    DevConst dc = make_dc(L, group, n_v, q, K, D, Ap, Bp, Gr, Gc, logc, w);
    for (int c = 0; c < n_chains; ++c)
        for (int l = 0; l < dc.g.n_links; ++l) {
            if (dc.g.h2 == 2)
                electric_item<double, cxd, 2, true>(dc, c, l, links, Wr, (const cxd*)Wc, (const cxd*)ell, (cxd*)out,
                                                    (cxd*)pairs);
            else
                electric_item<double, cxd, 4, true>(dc, c, l, links, Wr, (const cxd*)Wc, (const cxd*)ell, (cxd*)out,
                                                    (cxd*)pairs);
        }
}

void emu_link_terms(int L, int group, int n_v, int K, int n_chains, const void* links, const int* q_phys,
                    const double* blk, const double* pair_blk, double* out, double* pair_out) {
    const int q[2] = {1, 1};
    DevConst dc = make_dc(L, group, n_v, q, K, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr);
    for (int c = 0; c < n_chains; ++c)
        for (int l = 0; l < dc.g.n_links; ++l)
            link_term_item(dc, c, l, links, q_phys, (const cxd*)blk, (const cxd*)pair_blk, (cxd*)out,
                           (cxd*)pair_out);
}

void emu_fermion(int L, int group, int n_v, const int* q, int K, const double* D, const double* Ap,
                 const double* Bp, const double* Gr, const double* Gc, const double* logc, const double* w,
                 int n_chains, const double* Wr, const double* Wc, const double* ell, double* site,
                 double* link, double* pair_site, double* pair_link) {
    DevConst dc = make_dc(L, group, n_v, q, K, D, Ap, Bp, Gr, Gc, logc, w);
    for (int c = 0; c < n_chains; ++c)
        for (int it = 0; it < dc.g.V + dc.g.n_links; ++it) {
            if (dc.g.B == 8)
                fermion_item<double, cxd, 8>(dc, c, it, Wr, (const cxd*)Wc, (const cxd*)ell, (cxd*)site,
                                             (cxd*)link, (cxd*)pair_site, (cxd*)pair_link);
            else
                fermion_item<double, cxd, 16>(dc, c, it, Wr, (const cxd*)Wc, (const cxd*)ell, (cxd*)site,
                                              (cxd*)link, (cxd*)pair_site, (cxd*)pair_link);
        }
}

// SU(2) proposal of chain c at (sweep, link l) from the quaternion q_in
// (links holds one link): new quaternion and old/new doublet rotations.
double emu_draw_su2(unsigned long long sweep, uint64_t seed, int c, double width, const double* q_in,
                    double* qn, double* Rold, double* Rnew) {
    Geometry g{};
    g.n_links = 1;
    // link_quat(g, links, cfg, 0) reads links + cfg * 4: chain c's slot holds q_in
    std::vector<double> buf((size_t)(c + 1) * 4, 0.0);
    for (int k = 0; k < 4; ++k) buf[(size_t)c * 4 + k] = q_in[k];
    return draw_su2(g, buf.data(), c, 0, sweep, seed, width, qn, Rold, Rnew);
}

// (O Gamma O^T)[x][y] of an SU(2) link block: Gr one real r x r block.
double emu_twisted_su2(const double* Gr, int x, int y, const double* R) {
    DevConst dc{};
    dc.g.n_links = 1;
    dc.g.r = 8;
    dc.Gr = Gr;
    return twisted_su2<double>(dc, 0, 0, x, y, R);
}

// M_p of configuration 0 (links holds one configuration) into M [N][N]
// (cplx: complex pair p of its family, complex out).
void emu_assemble(int L, int group, int n_v, const int* q, int K, const double* D, const double* Gr,
                  const double* Gc, const void* links, int pair, int cplx, double* M) {
    DevConst dc = make_dc(L, group, n_v, q, K, D, nullptr, nullptr, Gr, Gc, nullptr, nullptr);
    const int N = dc.g.N;
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) {
            if (cplx) ((cxd*)M)[(size_t)i * N + j] = assemble_elem<cxd>(dc, links, 0, pair, i, j);
            else M[(size_t)i * N + j] = assemble_elem<double>(dc, links, 0, pair, i, j);
        }
}

void emu_score(int L, int group, int n_v, const int* q, int K, const double* logc, const double* w, int n_chains,
               const double* Wr, const double* Wc, const double* ell, double* out) {
    DevConst dc = make_dc(L, group, n_v, q, K, nullptr, nullptr, nullptr, nullptr, nullptr, logc, w);
    for (int c = 0; c < n_chains; ++c)
        for (int s = 0; s < dc.g.V; ++s) score_item<double, cxd>(dc, c, s, Wr, (const cxd*)Wc, (const cxd*)ell, out);
}

void emu_fermion4(int L, int group, int n_v, const int* q, int K, const double* D, const double* Ap,
                  const double* Bp, const double* Gr, const double* Gc, const double* logc, const double* w,
                  int n_chains, const double* Wr, const double* Wc, const double* ell, double* out,
                  double* pairs) {
    DevConst dc = make_dc(L, group, n_v, q, K, D, Ap, Bp, Gr, Gc, logc, w);
    for (int c = 0; c < n_chains; ++c)
        for (int l = 0; l < dc.g.n_links; ++l) {
            if (dc.g.B == 8)
                fermion4_item<double, cxd, 8>(dc, c, l, Wr, (const cxd*)Wc, (const cxd*)ell, (cxd*)out, (cxd*)pairs);
            else
                fermion4_item<double, cxd, 16>(dc, c, l, Wr, (const cxd*)Wc, (const cxd*)ell, (cxd*)out, (cxd*)pairs);
        }
}

// Mean SU(2) plaquette of one configuration (links [2V][4]) on an L x L lattice,
// with the link order of the plaquette kernels.
double emu_plaquette_su2(int L, const double* links) {
    Geometry g{};
    g.L = L; g.V = L * L; g.n_links = 2 * g.V;
    double acc = 0.0;
    for (int s = 0; s < g.V; ++s) {
        int x = s % L, y = s / L;
        int sx = y * L + (x + 1) % L, sy = ((y + 1) % L) * L + x;
        int l1 = 2 * s, l2 = 2 * sx + 1, l3 = 2 * sy, l4 = 2 * s + 1;
        acc += plaquette_su2(link_quat(g, links, 0, l1), link_quat(g, links, 0, l2), link_quat(g, links, 0, l3),
                             link_quat(g, links, 0, l4));
    }
    return acc / g.V;
}

void emu_link_score(int L, int group, int n_v, const int* q, int K, const double* D, const double* Gr,
                    const double* Gc, const double* logc, const double* w, int n_chains, const void* links,
                    const double* Wr, const double* Wc, const double* ell, double* out) {
    DevConst dc = make_dc(L, group, n_v, q, K, D, nullptr, nullptr, Gr, Gc, logc, w);
    for (int c = 0; c < n_chains; ++c)
        for (int p = 0; p < dc.P; ++p)
            for (int l = 0; l < dc.g.n_links; ++l) {
                if (dc.g.r == 4)
                    link_score_item<double, cxd, 4>(dc, c, p, l, links, Wr, (const cxd*)Wc, (const cxd*)ell, (cxd*)out);
                else
                    link_score_item<double, cxd, 8>(dc, c, p, l, links, Wr, (const cxd*)Wc, (const cxd*)ell, (cxd*)out);
            }
}

// loop_value of every loop position of configuration 0 into out (mode 0: V
// rectangles; mode 1: L winding loops).
void emu_loops(int L, int group, const void* links, int R, int T, int mode, double* out) {
    Geometry g{};
    g.L = L; g.V = L * L; g.n_links = 2 * g.V; g.group = group;
    const int items = mode ? L : g.V;
    for (int s = 0; s < items; ++s) out[s] = loop_value(g, links, 0, s, R, T, mode);
}

void emu_pair_norm(int L, int group, int n_v, const int* q, int K, const double* logc, const double* w,
                   int n_chains, const double* ell, double* out) {
    DevConst dc = make_dc(L, group, n_v, q, K, nullptr, nullptr, nullptr, nullptr, nullptr, logc, w);
    for (int c = 0; c < n_chains; ++c) pair_norm_item(dc, c, (const cxd*)ell, (cxd*)out);
}

}  // extern "C"
