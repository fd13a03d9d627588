// Metropolis sweep kernels of libggf (Sec. 5.1 sampling of p(G) = N(G)/N).
//
// Per link step, for every chain in lockstep:
//  ratio_kernel   one CTA per chain.  Draws the Philox numbers, forms the
//                 change Delta of the twisted link block for every pair
//                 (n, m), gathers W_SS from the cached inverse W = M^{-1},
//                 evaluates the Pfaffian ratio
//                    Pf(M') / Pf(M) = Pf([[Delta, -1], [1, W_SS]])
//                 (r/2 = 2 n_v even, so no extra sign) warp-parallel in FP64,
//                 combines the pairs into N(G')/N(G), decides, and on accept
//                 writes Z = (1 + Delta W_SS)^{-1} Delta, the rows Y = W[S, :]
//                 and the columns C = W[:, S].
//  update_kernel  rank-r Sherman-Morrison-Woodbury update of every pair's W
//                 of the accepted chains:  W <- W - C Z Y.
//                 The columns are gathered explicitly: replacing C by -Y^T
//                 (exact for an antisymmetric W) lets the rounding error's
//                 symmetric part grow geometrically from update to update.
//  observe_kernel per sweep: plaquette mean, log N(G), acceptance rate.
#include "ggf_ctx.h"
#include "ggf_geom.cuh"

#include "ggf_sweep.cuh"

namespace {

struct SweepArgs {
    DevConst dc;
    int n_chains;
    const unsigned long long* d_sweep;   // sweep index (device, so captured sweeps replay)
    int link;
    uint64_t seed;
    uint64_t coff;         // Philox key word 1 = coff + chain
    double width;
    void* links;
    const void* Wr;
    const void* Wc;
    cxd* ell;
    cxd* zbuf;
    void* ybuf_r;
    void* ybuf_c;
    int* accept;
    int* since_refresh;
    int* sweep_acc;
    unsigned long long* counters;
    // delayed updates
    const void* Pr;   // real-family panels  [n][K][2][N][KRM]
    const void* Pc;   // complex-family panels [n][Kc][2][2][N][KRM]
    int* pend;
    int kmax;   // > 1: delayed
    // block moves: per-chain link, forced new angle prop[c][32] entry k, dead flags
    const int* link_of_chain;
    const double* forced;
    int forced_k;
    int* dead;
};

// SU2: SU(2) links (quaternion proposal and doublet twist); the Z2 and U(1)
// instantiations (SU2 = false) do not contain that code.
template <class RW, class CW, bool SU2>
__global__ void __launch_bounds__(NWARP * 32) ratio_kernel(SweepArgs a) {
    extern __shared__ cxd sm[];
    const Geometry& g = a.dc.g;
    const int P = a.dc.P, K = a.dc.K, r = g.r, N = g.N;
    const int c = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    cxd* Delta = sm;                       // [P][r][r]
    cxd* Wss = Delta + P * r * r;          // [P][r][r]
    cxd* Bord = Wss + P * r * r;           // [NWARP][2r][2r]
    cxd* rho = Bord + NWARP * 4 * r * r;   // [P]
    cxd* fcol = rho + P;                   // [NWARP][r]
    __shared__ Proposal s_q;
    __shared__ double s_cs[8];
    __shared__ int s_accept;
    __shared__ double s_su2[36];          // SU2: new quaternion, old and new doublet rotations

    const int l = a.link_of_chain ? a.link_of_chain[c] : a.link;
    int a0, b0;
    link_ends(g, l, a0, b0);

    if constexpr (SU2) {
        if (threadIdx.x == 0) {
            Proposal q{};
            q.u_acc = draw_su2(g, a.links, c, l, *a.d_sweep, a.seed, a.width, s_su2, s_su2 + 4, s_su2 + 20,
                                   a.coff);
            s_q = q;
        }
        __syncthreads();
    } else {
        if (threadIdx.x == 0) {
            Proposal q = draw_proposal(g, a.links, c, l, *a.d_sweep, a.seed, a.width, a.coff);
            if (a.forced && g.group == GGF_U1) q.th_new = a.forced[(size_t)c * 32 + a.forced_k];   // block move
            s_q = q;
        }
        __syncthreads();
    }
    const Proposal q = s_q;
    if constexpr (!SU2) twist_table(g, q, s_cs);
    __syncthreads();

    for (int p = warp; p < P; p += NWARP) {
        cxd* D = Delta + p * r * r;
        cxd* Ws = Wss + p * r * r;
        if constexpr (SU2) pair_delta_su2(a.dc, p, l, s_su2 + 4, s_su2 + 20, D);
        else pair_delta(a.dc, p, l, q, s_cs, D);
        for (int e = lane; e < r * r; e += 32) {
            const int gi = link_majorana(g, a0, b0, e / r), gj = link_majorana(g, a0, b0, e % r);
            cxd wv;
            if (p < K) wv = loadc((const RW*)a.Wr + (((size_t)c * K + p) * N + gi) * N + gj);
            else wv = loadc((const CW*)a.Wc + (((size_t)c * (P - K) + (p - K)) * N + gi) * N + gj);
            if (a.kmax > 1) {
                // pending updates: W_eff[S, S] = W[S, S] - U[S, :] V[:, S]
                const int kr = a.pend[c] * r;
                const int KRM = a.kmax * r, NP = panel_rows(N);
                const size_t NK = panel_plane(N, KRM);
                typedef typename Sc<RW>::R R;
                if (p < K) {
                    const R* U = (const R*)a.Pr + ((size_t)c * K + p) * 2 * NK;
                    const R* Vt = U + NK;
                    for (int qq = 0; qq < kr; ++qq)
                        wv -= Sc<RW>::to(PanelIO<RW>::ld(U, NK, pidx(gi, qq, NP))) *
                              Sc<RW>::to(PanelIO<RW>::ld(Vt, NK, pidx(gj, qq, NP)));
                } else {
                    const R* U = (const R*)a.Pc + ((size_t)c * (P - K) + (p - K)) * 4 * NK;
                    const R* Vt = U + 2 * NK;
                    for (int qq = 0; qq < kr; ++qq)
                        wv -= Sc<CW>::to(PanelIO<CW>::ld(U, NK, pidx(gi, qq, NP))) *
                              Sc<CW>::to(PanelIO<CW>::ld(Vt, NK, pidx(gj, qq, NP)));
                }
            }
            Ws[e] = wv;
        }
        __syncwarp();
        cxd pf = bordered_ratio(D, Ws, Bord + warp * 4 * r * r, r);
        if (lane == 0) rho[p] = pf;
        __syncwarp();
    }
    __syncthreads();

    if (threadIdx.x == 0) {
        double sn, so;
        combine_pairs(a.dc, a.ell + (size_t)c * P, rho, sn, so);
        int acc;
        if (a.forced) {
            // block move: every link of the block is taken tentatively; the move is
            // decided once the whole block's ratio is known
            bool ok = a.dead[c] == 0;
            for (int p = 0; p < P; ++p) ok = ok && isfinite(rho[p].x) && isfinite(rho[p].y) && (rho[p].x != 0.0 || rho[p].y != 0.0);
            if (!ok) a.dead[c] = 1;
            acc = ok ? 1 : 0;
        } else {
            acc = (sn > 0.0 && so > 0.0 && q.u_acc < sn / so) ? 1 : 0;
            atomicAdd(&a.counters[0], 1ULL);
        }
        s_accept = acc;
        a.accept[c] = acc;
        if (acc) {
            if (a.kmax > 1) a.pend[c] += 1;
            if (!a.forced) {
                atomicAdd(&a.counters[1], 1ULL);
                a.since_refresh[c] += 1;
                a.sweep_acc[c] += 1;
            }
            if constexpr (SU2) {
                double* dst = (double*)a.links + ((size_t)c * g.n_links + l) * 4;
                for (int k = 0; k < 4; ++k) dst[k] = s_su2[k];
            } else {
                if (g.group == GGF_Z2) ((int8_t*)a.links)[(size_t)c * g.n_links + l] = (int8_t)q.g_new;
                else ((double*)a.links)[(size_t)c * g.n_links + l] = q.th_new;
            }
        }
    }
    __syncthreads();
    if (!s_accept) return;

    for (int p = warp; p < P; p += NWARP) {
        const bool ok = pair_z(Delta + p * r * r, Wss + p * r * r, Bord + warp * 4 * r * r, fcol + warp * r, r,
                               a.zbuf + ((size_t)c * P + p) * r * r);
        if (!ok && a.forced && lane == 0) a.dead[c] = 1;
        if (lane == 0) ell_add(a.ell[(size_t)c * P + p], rho[p], p < K);
        __syncwarp();
    }
    // rows Y = W[S, :] and columns C^T = W[:, S]^T for the update kernel,
    // stored per (chain, pair) as [2][r][N] (delayed mode: gather_kernel)
    if (a.kmax > 1) return;
    for (int p = 0; p < P; ++p) {
        for (int e = threadIdx.x; e < r * N; e += blockDim.x) {
            int xi = e / N, j = e - xi * N;
            int gi = xi < g.h2 ? a0 + xi : b0 + xi - g.h2;
            if (p < K) {
                const RW* W = (const RW*)a.Wr + ((size_t)c * K + p) * N * N;
                RW* yb = (RW*)a.ybuf_r + ((size_t)c * K + p) * 2 * r * N;
                yb[(size_t)xi * N + j] = W[(size_t)gi * N + j];
                yb[(size_t)(r + xi) * N + j] = W[(size_t)j * N + gi];
            } else {
                const CW* W = (const CW*)a.Wc + ((size_t)c * (P - K) + (p - K)) * N * N;
                CW* yb = (CW*)a.ybuf_c + ((size_t)c * (P - K) + (p - K)) * 2 * r * N;
                yb[(size_t)xi * N + j] = W[(size_t)gi * N + j];
                yb[(size_t)(r + xi) * N + j] = W[(size_t)j * N + gi];
            }
        }
    }
}

template <class T, int R>
__global__ void __launch_bounds__(256) update_kernel(int N, int P, int fam_pairs, int pair_off, T* W,
                                                     const T* ybuf, const cxd* zbuf, const int* accept, int TI) {
    const int c = blockIdx.z;
    if (!accept[c]) return;
    const int p = blockIdx.y;
    extern __shared__ unsigned char smraw[];
    T* Zs = (T*)smraw;        // [R][R]
    T* Pr = Zs + R * R;       // [TI][R]
    T* Wp = W + ((size_t)c * fam_pairs + p) * N * N;
    const T* Y = ybuf + ((size_t)c * fam_pairs + p) * 2 * R * N;   // rows W[S, :]
    const T* Ct = Y + (size_t)R * N;                                 // columns W[:, S]^T
    const cxd* Z = zbuf + ((size_t)c * P + pair_off + p) * R * R;
    for (int e = threadIdx.x; e < R * R; e += blockDim.x) Zs[e] = Sc<T>::from(Z[e]);
    __syncthreads();
    const int i0 = blockIdx.x * TI;
    const int ti = min(TI, N - i0);
    for (int e = threadIdx.x; e < ti * R; e += blockDim.x) {
        int i = e / R, b = e % R;
        T acc = Sc<T>::zero();
#pragma unroll
        for (int q = 0; q < R; ++q) acc += Ct[(size_t)q * N + i0 + i] * Zs[q * R + b];
        Pr[i * R + b] = acc;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        T yv[R];
#pragma unroll
        for (int b = 0; b < R; ++b) yv[b] = Y[(size_t)b * N + j];
        for (int i = 0; i < ti; ++i) {
            T acc = Wp[(size_t)(i0 + i) * N + j];
#pragma unroll
            for (int b = 0; b < R; ++b) acc -= Pr[i * R + b] * yv[b];
            Wp[(size_t)(i0 + i) * N + j] = acc;
        }
    }
}

// Delayed mode, accepted chains: rows Y = W_eff[S, :] and columns
// C = W_eff[:, S] of the effective inverse W_eff = W - U V, then the new
// panel entries U[:, slot] = C Z and V[slot, :] = Y (stored as V^T rows).
// Grid (ceil(N / 128), family pairs, chains), 128 threads, one index each.
template <class T, int R>
__global__ void __launch_bounds__(128) gather_kernel(Geometry g, int P, int fam_pairs, int pair_off, int link_all,
                                                     const int* link_of_chain, const T* W,
                                                     typename Sc<T>::R* Pan, const cxd* zbuf,
                                                     const int* accept, const int* pend, int kmax) {
    typedef typename Sc<T>::R RR;
    const int c = blockIdx.z;
    if (!accept[c]) return;
    const int p = blockIdx.y, N = g.N;
    const int slot = pend[c] - 1, kr = slot * R;
    const int KRM = kmax * R, NP = panel_rows(N);
    const size_t NK = panel_plane(N, KRM);
    extern __shared__ unsigned char smraw[];
    constexpr int QC = 128 / sizeof(T);  // rank chunk staged per step
    T* UtS = (T*)smraw;            // [kr][R]  U[S_a, q]
    T* VS = UtS + kmax * R * R;    // [kr][R]  V[q, S_a]
    T* Zs = VS + kmax * R * R;     // [R][R]
    T* Uc = Zs + R * R;            // [128][QC + 1] panel rows j0.., rank chunk
    T* Vc = Uc + 128 * (QC + 1);
    __shared__ int S[R];
    const int link = link_of_chain ? link_of_chain[c] : link_all;
    const int s = link >> 1, d = link & 1, x = s % g.L, y = s / g.L;
    const int t = d == 0 ? y * g.L + (x + 1) % g.L : ((y + 1) % g.L) * g.L + x;
    const int a0 = s * g.B + (2 * d + 1) * g.h2, b0 = t * g.B + (2 * d) * g.h2;
    if (threadIdx.x < R) S[threadIdx.x] = threadIdx.x < g.h2 ? a0 + threadIdx.x : b0 + threadIdx.x - g.h2;
    __syncthreads();
    const size_t base = ((size_t)c * fam_pairs + p);
    const T* Wp = W + base * N * N;
    RR* U = Pan + base * 2 * PanelIO<T>::PLANES * NK;
    RR* Vt = U + PanelIO<T>::PLANES * NK;
    const cxd* Z = zbuf + ((size_t)c * P + pair_off + p) * R * R;
    for (int e = threadIdx.x; e < kr * R; e += blockDim.x) {
        int q = e / R, a = e % R;
        UtS[e] = PanelIO<T>::ld(U, NK, pidx(S[a], q, NP));
        VS[e] = PanelIO<T>::ld(Vt, NK, pidx(S[a], q, NP));
    }
    for (int e = threadIdx.x; e < R * R; e += blockDim.x) Zs[e] = Sc<T>::from(Z[e]);
    __syncthreads();
    const int j0 = blockIdx.x * blockDim.x;
    const int j = j0 + threadIdx.x;
    const bool live = j < N;
    T yv[R], cv[R];
#pragma unroll
    for (int a = 0; a < R; ++a) {
        yv[a] = live ? Wp[(size_t)S[a] * N + j] : Sc<T>::zero();
        cv[a] = live ? Wp[(size_t)j * N + S[a]] : Sc<T>::zero();
    }
    // panel rows j0 .. j0+127 staged chunk by chunk with coalesced loads
    for (int q0 = 0; q0 < kr; q0 += QC) {
        const int qn = min(QC, kr - q0);
        __syncthreads();
        for (int e = threadIdx.x; e < 128 * QC; e += blockDim.x) {
            int row = e / QC, qq = e % QC;
            bool ok = qq < qn && j0 + row < N;
            size_t idx = pidx(j0 + row, q0 + qq, NP);
            Uc[row * (QC + 1) + qq] = ok ? PanelIO<T>::ld(U, NK, idx) : Sc<T>::zero();
            Vc[row * (QC + 1) + qq] = ok ? PanelIO<T>::ld(Vt, NK, idx) : Sc<T>::zero();
        }
        __syncthreads();
        for (int qq = 0; qq < qn; ++qq) {
            const T vq = Vc[threadIdx.x * (QC + 1) + qq];
            const T uq = Uc[threadIdx.x * (QC + 1) + qq];
            const int q = q0 + qq;
#pragma unroll
            for (int a = 0; a < R; ++a) {
                yv[a] -= UtS[q * R + a] * vq;
                cv[a] -= uq * VS[q * R + a];
            }
        }
    }
    if (!live) return;
#pragma unroll
    for (int b = 0; b < R; ++b) {
        T u = Sc<T>::zero();
#pragma unroll
        for (int a = 0; a < R; ++a) u += cv[a] * Zs[a * R + b];
        PanelIO<T>::st(U, NK, pidx(j, kr + b, NP), u);
        PanelIO<T>::st(Vt, NK, pidx(j, kr + b, NP), yv[b]);
    }
}

// W <- W - U V over the pending panels (rank pend[c] * R), SIMT tiled product
// (FP64 chains, and FP32 when the tensor-core flush is not used).
// Grid (tiles_i * tiles_j, family pairs, chains), 256 threads as 16 x 16, each
// a 4 x 4 block of a 64 x 64 tile of W.
template <class T, int R>
__global__ void __launch_bounds__(256) flush_kernel(int N, int fam_pairs, T* W, const typename Sc<T>::R* Pan,
                                                    const int* pend, int kmax, int tiles) {
    typedef typename Sc<T>::R RR;
    const int c = blockIdx.z;
    const int kc = pend[c];
    if (kc == 0) return;
    const int kr = kc * R, KRM = kmax * R, NP = panel_rows(N);
    const size_t NK = panel_plane(N, KRM);
    const int p = blockIdx.y;
    const int ti = blockIdx.x / tiles, tj = blockIdx.x - ti * tiles;
    const int i0 = ti * 64, j0 = tj * 64;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    __shared__ T As[16][65];
    __shared__ T Bs[16][65];
    const size_t base = ((size_t)c * fam_pairs + p);
    T* Wp = W + base * N * N;
    const RR* U = Pan + base * 2 * PanelIO<T>::PLANES * NK;
    const RR* Vt = U + PanelIO<T>::PLANES * NK;
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = Sc<T>::zero();
    for (int q0 = 0; q0 < kr; q0 += 16) {
        for (int e = threadIdx.x; e < 16 * 64; e += 256) {
            int k = e >> 4, qq = e & 15;      // consecutive threads walk the rank index
            int q = q0 + qq;
            As[qq][k] = (q < kr && i0 + k < N) ? PanelIO<T>::ld(U, NK, pidx(i0 + k, q, NP)) : Sc<T>::zero();
            Bs[qq][k] = (q < kr && j0 + k < N) ? PanelIO<T>::ld(Vt, NK, pidx(j0 + k, q, NP)) : Sc<T>::zero();
        }
        __syncthreads();
#pragma unroll
        for (int qq = 0; qq < 16; ++qq) {
            T av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = As[qq][ty * 4 + a];
#pragma unroll
            for (int b = 0; b < 4; ++b) bv[b] = Bs[qq][tx * 4 + b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] += av[a] * bv[b];
        }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        int i = i0 + ty * 4 + a;
        if (i >= N) continue;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            int j = j0 + tx * 4 + b;
            if (j < N) Wp[(size_t)i * N + j] -= acc[a][b];
        }
    }
}

__global__ void reset_pend(int n, int* pend) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < n) pend[c] = 0;
}

__global__ void observe_kernel(DevConst dc, int n_chains, const void* links, const cxd* ell, const int* sweep_acc,
                               double* obs) {
    __shared__ double red[256];
    const Geometry& g = dc.g;
    int c = blockIdx.x;
    double acc = 0.0;
    for (int s = threadIdx.x; s < g.V; s += blockDim.x) {
        int x = s % g.L, y = s / g.L;
        int sx = y * g.L + (x + 1) % g.L, sy = ((y + 1) % g.L) * g.L + x;
        int l1 = 2 * s, l2 = 2 * sx + 1, l3 = 2 * sy, l4 = 2 * s + 1;
        if (g.group == GGF_Z2) {
            const int8_t* L8 = (const int8_t*)links + (size_t)c * g.n_links;
            acc += (double)(L8[l1] * L8[l2] * L8[l3] * L8[l4]);
        } else if (g.group == GGF_SU2) {
            acc += plaquette_su2(link_quat(g, links, c, l1), link_quat(g, links, c, l2), link_quat(g, links, c, l3),
                                 link_quat(g, links, c, l4));
        } else {
            const double* T = (const double*)links + (size_t)c * g.n_links;
            acc += cos(T[l1] + T[l2] - T[l3] - T[l4]);
        }
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double amax = -INFINITY;
        for (int p = 0; p < dc.P; ++p) amax = fmax(amax, dc.logc[p].x + ell[(size_t)c * dc.P + p].x);
        double sv = 0.0;
        for (int p = 0; p < dc.P; ++p) {
            cxd e = dc.logc[p] + ell[(size_t)c * dc.P + p];
            if (p < dc.K) e.y = 0.0;
            e.x -= amax;
            sv += (dc.w[p] * cexp_(e)).x;
        }
        obs[(size_t)c * GGF_N_OBS + 0] = red[0] / g.V;
        obs[(size_t)c * GGF_N_OBS + 1] = sv > 0 ? amax + log(sv) : -INFINITY;
        obs[(size_t)c * GGF_N_OBS + 2] = (double)sweep_acc[c] / g.n_links;
    }
}

__global__ void mark_refresh(int n_chains, int R, const int* since, int* list) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_chains) return;
    if (since[c] >= R) {
        int k = atomicAdd(&list[0], 1);
        list[1 + k] = c;
    }
}

}  // namespace

ggf_status ggf_flush(ggf_ctx* ctx, cudaStream_t st);
ggf_status ggf_flush_tc(ggf_ctx* ctx, cudaStream_t st, int* launches);

size_t ggf_ratio_smem(int P, int r) {
    return (size_t)(2 * P * r * r + NWARP * 4 * r * r + P + NWARP * r) * sizeof(cxd);
}

ggf_status ggf_link_step_ex(ggf_ctx* ctx, int link, cudaStream_t st, const int* link_of_chain, const double* forced,
                            int forced_k, int* dead);

ggf_status ggf_link_step(ggf_ctx* ctx, int link, cudaStream_t st) {
    return ggf_link_step_ex(ctx, link, st, nullptr, nullptr, 0, nullptr);
}

// One proposal per chain.  Block moves pass a per-chain link, the proposed
// angles (forced, slot forced_k) and dead flags; the flush cadence then stays
// with the caller.
ggf_status ggf_link_step_ex(ggf_ctx* ctx, int link, cudaStream_t st, const int* link_of_chain, const double* forced,
                            int forced_k, int* dead) {
    Chains& ch = ctx->ch;
    const Geometry& g = ctx->g;
    SweepArgs a;
    a.dc = ctx->dc();
    a.n_chains = ch.n;
    a.d_sweep = ch.d_sweep;
    a.link = link;
    a.seed = ch.opts.seed;
    a.coff = ch.opts.chain_offset;
    a.width = ch.opts.width;
    a.links = ch.links;
    a.Wr = ch.Wr;
    a.Wc = ch.Wc;
    a.ell = ch.ell;
    a.zbuf = (cxd*)ch.zbuf;
    const bool fp64 = ch.opts.precision == GGF_FP64;
    size_t rsz = fp64 ? sizeof(double) : sizeof(float);
    a.ybuf_r = ch.ybuf;
    a.ybuf_c = (unsigned char*)ch.ybuf + (size_t)ch.n * ctx->K * 2 * g.r * g.N * rsz;
    a.accept = ch.accept;
    a.since_refresh = ch.since_refresh;
    a.sweep_acc = ch.sweep_acc;
    a.counters = ch.counters;
    a.Pr = ch.Pr; a.Pc = ch.Pc;
    a.link_of_chain = link_of_chain;
    a.forced = forced;
    a.forced_k = forced_k;
    a.dead = dead;
    a.pend = ch.pend;
    a.kmax = ch.kmax;
    size_t smem = ggf_ratio_smem(ctx->P, g.r);
    const int ev0 = ctx->prof_mark(st);
    ctx->launches += 2 + (ctx->Kc ? 1 : 0);
    if (g.group == GGF_SU2) {
        if (fp64) ratio_kernel<double, cxd, true><<<ch.n, NWARP * 32, smem, st>>>(a);
        else ratio_kernel<float, cxf, true><<<ch.n, NWARP * 32, smem, st>>>(a);
    } else {
        if (fp64) ratio_kernel<double, cxd, false><<<ch.n, NWARP * 32, smem, st>>>(a);
        else ratio_kernel<float, cxf, false><<<ch.n, NWARP * 32, smem, st>>>(a);
    }
    GGF_CK(cudaGetLastError());
    const int ev1 = ctx->prof_mark(st);
    ctx->prof_pair(GGF_KT_RATIO, ev0, ev1);
    const int N = g.N;
    if (ch.kmax > 1) {
        dim3 gg((N + 127) / 128, ctx->K, ch.n), gc2((N + 127) / 128, ctx->Kc, ch.n);
#define GGF_GATH(T, R_, grid, fam, off, Wp, Pp)                                                               \
    gather_kernel<T, R_><<<grid, 128, (2 * ch.kmax * R_ * R_ + R_ * R_ + 2 * 128 * (128 / sizeof(T) + 1)) * sizeof(T), st>>>( \
        g, ctx->P, fam, off, link, link_of_chain, (const T*)(Wp), (typename Sc<T>::R*)(Pp), a.zbuf, ch.accept, \
        ch.pend, ch.kmax)
        if (g.r == 4) {
            if (fp64) {
                GGF_GATH(double, 4, gg, ctx->K, 0, ch.Wr, ch.Pr);
                if (ctx->Kc) GGF_GATH(cxd, 4, gc2, ctx->Kc, ctx->K, ch.Wc, ch.Pc);
            } else {
                GGF_GATH(float, 4, gg, ctx->K, 0, ch.Wr, ch.Pr);
                if (ctx->Kc) GGF_GATH(cxf, 4, gc2, ctx->Kc, ctx->K, ch.Wc, ch.Pc);
            }
        } else {
            if (fp64) {
                GGF_GATH(double, 8, gg, ctx->K, 0, ch.Wr, ch.Pr);
                if (ctx->Kc) GGF_GATH(cxd, 8, gc2, ctx->Kc, ctx->K, ch.Wc, ch.Pc);
            } else {
                GGF_GATH(float, 8, gg, ctx->K, 0, ch.Wr, ch.Pr);
                if (ctx->Kc) GGF_GATH(cxf, 8, gc2, ctx->Kc, ctx->K, ch.Wc, ch.Pc);
            }
        }
#undef GGF_GATH
        GGF_CK(cudaGetLastError());
        ctx->prof_pair(GGF_KT_UPDATE, ev1, ctx->prof_mark(st));
        if (forced) { ++ch.steps_since_flush; return GGF_OK; }
        if (++ch.steps_since_flush >= ch.kmax) GGF_TRY(ggf_flush(ctx, st));
        return GGF_OK;
    }
    const int TI = 8;
    dim3 gr((N + TI - 1) / TI, ctx->K, ch.n);
    dim3 gc((N + TI - 1) / TI, ctx->Kc, ch.n);
#define GGF_UPD(T, R_, grid, fam, off, Wp, Yp)                                                         \
    update_kernel<T, R_><<<grid, 256, (R_ * R_ + TI * R_) * sizeof(T), st>>>(N, ctx->P, fam, off, (T*)(Wp), \
                                                                              (const T*)(Yp), a.zbuf, ch.accept, TI)
    if (g.r == 4) {
        if (fp64) {
            GGF_UPD(double, 4, gr, ctx->K, 0, ch.Wr, a.ybuf_r);
            if (ctx->Kc) GGF_UPD(cxd, 4, gc, ctx->Kc, ctx->K, ch.Wc, a.ybuf_c);
        } else {
            GGF_UPD(float, 4, gr, ctx->K, 0, ch.Wr, a.ybuf_r);
            if (ctx->Kc) GGF_UPD(cxf, 4, gc, ctx->Kc, ctx->K, ch.Wc, a.ybuf_c);
        }
    } else {
        if (fp64) {
            GGF_UPD(double, 8, gr, ctx->K, 0, ch.Wr, a.ybuf_r);
            if (ctx->Kc) GGF_UPD(cxd, 8, gc, ctx->Kc, ctx->K, ch.Wc, a.ybuf_c);
        } else {
            GGF_UPD(float, 8, gr, ctx->K, 0, ch.Wr, a.ybuf_r);
            if (ctx->Kc) GGF_UPD(cxf, 8, gc, ctx->Kc, ctx->K, ch.Wc, a.ybuf_c);
        }
    }
#undef GGF_UPD
    GGF_CK(cudaGetLastError());
    ctx->prof_pair(GGF_KT_UPDATE, ev1, ctx->prof_mark(st));
    return GGF_OK;
}

ggf_status ggf_flush(ggf_ctx* ctx, cudaStream_t st) {
    Chains& ch = ctx->ch;
    const Geometry& g = ctx->g;
    if (ch.kmax <= 1 || ch.steps_since_flush == 0) return GGF_OK;
    const bool fp64 = ch.opts.precision == GGF_FP64;
    const int N = g.N, tiles = (N + 63) / 64;
    const int ev0 = ctx->prof_mark(st);
    dim3 gr(tiles * tiles, ctx->K, ch.n), gc(tiles * tiles, ctx->Kc, ch.n);
#define GGF_FL(T, R_, grid, fam, Wp, Pp) \
    flush_kernel<T, R_><<<grid, 256, 0, st>>>(N, fam, (T*)(Wp), (const typename Sc<T>::R*)(Pp), ch.pend, ch.kmax, tiles)
    int nl = 1 + (ctx->Kc ? 1 : 0);
    if (!fp64 && ctx->use_tc) {
        nl = 0;
        GGF_TRY(ggf_flush_tc(ctx, st, &nl));
    } else if (g.r == 4) {
        if (fp64) { GGF_FL(double, 4, gr, ctx->K, ch.Wr, ch.Pr); if (ctx->Kc) GGF_FL(cxd, 4, gc, ctx->Kc, ch.Wc, ch.Pc); }
        else { GGF_FL(float, 4, gr, ctx->K, ch.Wr, ch.Pr); if (ctx->Kc) GGF_FL(cxf, 4, gc, ctx->Kc, ch.Wc, ch.Pc); }
    } else {
        if (fp64) { GGF_FL(double, 8, gr, ctx->K, ch.Wr, ch.Pr); if (ctx->Kc) GGF_FL(cxd, 8, gc, ctx->Kc, ch.Wc, ch.Pc); }
        else { GGF_FL(float, 8, gr, ctx->K, ch.Wr, ch.Pr); if (ctx->Kc) GGF_FL(cxf, 8, gc, ctx->Kc, ch.Wc, ch.Pc); }
    }
#undef GGF_FL
    ctx->prof_pair(GGF_KT_FLUSH, ev0, ctx->prof_mark(st));
    reset_pend<<<(ch.n + 127) / 128, 128, 0, st>>>(ch.n, ch.pend);
    ctx->launches += nl + 1;
    GGF_CK(cudaGetLastError());
    ch.steps_since_flush = 0;
    return GGF_OK;
}

__global__ void bump_sweep(unsigned long long* s) { *s += 1ULL; }

// Kernel attributes are set once per context before any launch, so that no
// attribute call happens while a sweep is being captured into a graph.
// The attribute is a per-function cap shared by every context in the
// process, so it is raised once to the device's opt-in maximum.
ggf_status ggf_prepare_sampler(ggf_ctx* ctx) {
    static bool done[64] = {false};
    if (ctx->device >= 0 && ctx->device < 64 && done[ctx->device]) return GGF_OK;
    int mx = 0;
    GGF_CK(cudaDeviceGetAttribute(&mx, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device));
    if (ggf_ratio_smem(36, 8) > (size_t)mx) return ggf_fail(ctx, GGF_EINVAL, "shared memory too small for K = 8");
    // dynamic cap = opt-in limit minus the kernel's static shared memory
    auto cap = [&](const void* fn) -> ggf_status {
        cudaFuncAttributes fa;
        GGF_CK(cudaFuncGetAttributes(&fa, fn));
        GGF_CK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, mx - (int)fa.sharedSizeBytes));
        return GGF_OK;
    };
    GGF_TRY(cap((const void*)ratio_kernel<double, cxd, false>));
    GGF_TRY(cap((const void*)ratio_kernel<float, cxf, false>));
    GGF_TRY(cap((const void*)ratio_kernel<double, cxd, true>));
    GGF_TRY(cap((const void*)ratio_kernel<float, cxf, true>));
    GGF_TRY(cap((const void*)gather_kernel<double, 4>));
    GGF_TRY(cap((const void*)gather_kernel<double, 8>));
    GGF_TRY(cap((const void*)gather_kernel<float, 4>));
    GGF_TRY(cap((const void*)gather_kernel<float, 8>));
    GGF_TRY(cap((const void*)gather_kernel<cxd, 4>));
    GGF_TRY(cap((const void*)gather_kernel<cxd, 8>));
    GGF_TRY(cap((const void*)gather_kernel<cxf, 4>));
    GGF_TRY(cap((const void*)gather_kernel<cxf, 8>));
    if (ctx->device >= 0 && ctx->device < 64) done[ctx->device] = true;
    return GGF_OK;
}

ggf_status ggf_bump_sweep(ggf_ctx* ctx, cudaStream_t st) {
    bump_sweep<<<1, 1, 0, st>>>(ctx->ch.d_sweep);
    ctx->launches += 1;
    GGF_CK(cudaGetLastError());
    return GGF_OK;
}

ggf_status ggf_observe(ggf_ctx* ctx, double* d_obs, cudaStream_t st) {
    Chains& ch = ctx->ch;
    ctx->launches += 1;
    observe_kernel<<<ch.n, 256, 0, st>>>(ctx->dc(), ch.n, ch.links, ch.ell, ch.sweep_acc, d_obs);
    GGF_CK(cudaGetLastError());
    return GGF_OK;
}

ggf_status ggf_mark_refresh(ggf_ctx* ctx, cudaStream_t st) {
    Chains& ch = ctx->ch;
    GGF_CK(cudaMemsetAsync(ch.refresh_list, 0, sizeof(int), st));
    ctx->launches += 1;
    mark_refresh<<<(ch.n + 127) / 128, 128, 0, st>>>(ch.n, ch.opts.refresh_every, ch.since_refresh, ch.refresh_list);
    GGF_CK(cudaGetLastError());
    return GGF_OK;
}
