// Batched (submatrix) delayed updates for local Metropolis sweeps
// (Sec. 5.1 sampling of p(G); the blocking of the Sherman-Morrison-Woodbury
// updates is this library's design, not the paper's).
//
// A batch is kb consecutive links l0 .. l0 + kb - 1 of the sweep order.  Every
// link end belongs to exactly one link, so the batch's Majorana sets S_j are
// disjoint and T = S_0 u ... u S_{kb-1} has exactly kb r elements (position
// j r + xi of T is Majorana xi of link l0 + j).  Every proposal of the batch
// needs only the block of the current inverse on T.  With W the inverse at
// the start of the batch, C = W[:, T], Y = W[T, :], G0 = W[T, T]:
//   batch_gather  C -> U panel, Y^T -> V^T panel, G := G0, X := 0 (C read as
//                 the true columns: -Y^T, equal in exact arithmetic, makes
//                 the rounding error grow geometrically)
//   batch_steps   one CTA per chain runs the kb link steps on the small
//                 matrices: ratio from G[S_j, S_j], decision, and on accept,
//                 with Z = (1 + Delta G[S, S])^{-1} Delta,
//                   G[F, F] -= G[F, S] Z G[S, F]   (F: the later links' rows)
//                   X       += P Z Q,  P = E_S - X G0[:, S],
//                                      Q = E_S^T - G0[S, :] X,
//                 so that the exact inverse after the batch is W - C X Y
//                 (each step is the rank-r update W' = W - W[:, S] Z W[S, :]
//                 with W[:, S] = C P and W[S, :] = Q Y).
//   batch_apply   V^T <- V^T X^T  (V = X Y)
// followed by the flush W <- W - U V (tcgen05 tensor cores for FP32 chains).
// Per batch and pair this reads C and Y once (2 N kb r elements) instead of
// two N-long panel products per accepted link, and folds kb links into one
// pass over W.
#include "ggf_sweep.cuh"

// 1: the X product of FP32 batches runs on the tensor cores (k_apply_tc.cu)
#ifndef GGF_APPLY_TC
#define GGF_APPLY_TC 1
#endif

namespace {

// ---- gather -------------------------------------------------------------------
// Grid (ceil(N / BR), family pairs, chains), 256 threads.  Rows i0 .. i0+BR-1
// of the U panel (C = W[:, T]) and of the V^T panel (Y^T = W[T, :]^T); the
// rows of G := W[T, T] whose T index falls in the block; X := 0 there.
template <class T>
__global__ void __launch_bounds__(256) batch_gather(Geometry g, int l0, int kb, int fam_pairs, int KRM, int BR,
                                                    const T* W, typename Sc<T>::R* Pan, T* Sm) {
    typedef typename Sc<T>::R RR;
    const int c = blockIdx.z, p = blockIdx.y, N = g.N, r = g.r, kr = kb * r;
    extern __shared__ unsigned char smraw[];
    int* Tl = (int*)smraw;                                   // [kr]
    T* tile = (T*)(smraw + ((kr * sizeof(int) + 15) & ~(size_t)15));   // [BR][kr + 1]
    for (int q = threadIdx.x; q < kr; q += blockDim.x) {
        int a0, b0;
        link_ends(g, l0 + q / r, a0, b0);
        Tl[q] = link_majorana(g, a0, b0, q % r);
    }
    __syncthreads();
    const int i0 = blockIdx.x * BR, nb = min(BR, N - i0), ld = kr + 1;
    const size_t NK = panel_plane(N, KRM), base = (size_t)c * fam_pairs + p;
    const int NP = panel_rows(N);
    const T* Wp = W + base * N * N;
    RR* U = Pan + base * 2 * PanelIO<T>::PLANES * NK;
    RR* Vt = U + PanelIO<T>::PLANES * NK;
    T* Gm = Sm + base * 2 * KRM * KRM;
    T* Xm = Gm + (size_t)KRM * KRM;
    // V^T rows: tile[ii][q] = W[T_q][i0 + ii], read along rows of W
    for (int e = threadIdx.x; e < kr * BR; e += blockDim.x) {
        int q = e / BR, ii = e - q * BR;
        tile[ii * ld + q] = ii < nb ? Wp[(size_t)Tl[q] * N + i0 + ii] : Sc<T>::zero();
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nb * kr; e += blockDim.x) {
        int ii = e / kr, q = e - ii * kr;
        PanelIO<T>::st(Vt, NK, pidx(i0 + ii, q, NP), tile[ii * ld + q]);
    }
    __syncthreads();
    // U rows: the true columns W[i0 + ii][T_q].  Replacing them by -Y^T (equal
    // for an exactly antisymmetric W) lets the rounding error grow
    // geometrically from batch to batch.
    for (int e = threadIdx.x; e < nb * kr; e += blockDim.x) {
        int ii = e / kr, q = e - ii * kr;
        T v = Wp[(size_t)(i0 + ii) * N + Tl[q]];
        tile[ii * ld + q] = v;
        PanelIO<T>::st(U, NK, pidx(i0 + ii, q, NP), v);
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int a = warp; a < kr; a += nw) {
        const int ii = Tl[a] - i0;
        if (ii < 0 || ii >= nb) continue;
        for (int q = lane; q < kr; q += 32) {
            Gm[(size_t)a * KRM + q] = tile[ii * ld + q];   // W[T_a][T_q] = U[T_a][q]
            Xm[(size_t)a * KRM + q] = Sc<T>::zero();
        }
    }
}

// ---- link steps on the small matrices ----------------------------------------
struct BatchArgs {
    DevConst dc;
    const unsigned long long* d_sweep;
    int l0, kb, KRM;
    uint64_t seed;
    uint64_t coff;         // Philox key word 1 = coff + chain
    double width;
    void* links;
    cxd* ell;
    int* since_refresh;
    int* sweep_acc;
    unsigned long long* counters;
    int* pend;
    const void* Pr;   // U panels: G0 = U[T, 0 .. kr)
    const void* Pc;
    void* Sr;         // small matrices [n][K][2][KRM][KRM]: G then X
    void* Sc_;        // [n][Kc][2][KRM][KRM]
};

// Rank-r update of one pair's small matrices after link j of the batch was
// accepted (all threads of the CTA).  Gm, Xm: KRM x KRM; U: the pair's U
// panel (planes of N x KRM); Z: r x r (FP64); st: 4 KRM r scratch scalars.
template <class T, int r>
__device__ __forceinline__ void small_update(T* Gm, T* Xm, const typename Sc<T>::R* U, size_t NK, int NP,
                                             const int* Tl, int j, int kb, int KRM, const cxd* Z, T* st) {
    const int jr = j * r, m = jr + r, kr = kb * r, nf = kr - m;
    T* A1 = st;                    // G[F, S] Z, later G0[0:jr, S], later P Z
    T* A2 = A1 + (size_t)KRM * r;  // G[S, F], later G0[S, 0:jr]
    T* A3 = A2 + (size_t)KRM * r;  // P  (m x r)
    T* A4 = A3 + (size_t)KRM * r;  // Q  (r x m)
    // (a) later links: G[F, F] -= (G[F, S] Z) G[S, F]
    if (nf > 0) {
        for (int e = threadIdx.x; e < nf * r; e += blockDim.x) {
            int i = e / r, b = e - i * r;
            T acc = Sc<T>::zero();
            for (int a = 0; a < r; ++a) acc += Gm[(size_t)(m + i) * KRM + jr + a] * Sc<T>::from(Z[a * r + b]);
            A1[e] = acc;
        }
        for (int e = threadIdx.x; e < r * nf; e += blockDim.x) {
            int b = e / nf, jj = e - b * nf;
            A2[e] = Gm[(size_t)(jr + b) * KRM + m + jj];
        }
        __syncthreads();
        for (int e = threadIdx.x; e < nf * nf; e += blockDim.x) {
            int i = e / nf, jj = e - i * nf;
            T* gp = Gm + (size_t)(m + i) * KRM + m + jj;
            T acc = *gp;
            for (int b = 0; b < r; ++b) acc -= A1[i * r + b] * A2[b * nf + jj];
            *gp = acc;
        }
        __syncthreads();
    }
    // (b) X += P Z Q on the leading m x m block
    for (int e = threadIdx.x; e < jr * r; e += blockDim.x) {
        int a = e / r, b = e - a * r;
        A1[e] = PanelIO<T>::ld(U, NK, pidx(Tl[a], jr + b, NP));        // G0[a][S_b]
        A2[b * jr + a] = PanelIO<T>::ld(U, NK, pidx(Tl[jr + b], a, NP));   // G0[S_b][a]
    }
    __syncthreads();
    // P (m x r): rows a < jr are -X[a, 0:jr] G0[0:jr, S], rows jr.. the identity;
    // Q (r x m): columns cc < jr are -G0[S, 0:jr] X[0:jr, cc], then the identity.
    // One thread per row a of P (resp. column cc of Q) keeps its r outputs in
    // registers, so every element of X is loaded once per product.
    const T one = Sc<T>::from(cxd{1.0, 0.0});
    for (int a = threadIdx.x; a < m; a += blockDim.x) {
        T acc[r];
#pragma unroll
        for (int b = 0; b < r; ++b) acc[b] = Sc<T>::zero();
        if (a < jr) {
            const T* xr = Xm + (size_t)a * KRM;
            for (int q = 0; q < jr; ++q) {
                const T x = xr[q];
#pragma unroll
                for (int b = 0; b < r; ++b) acc[b] -= x * A1[q * r + b];
            }
        }
#pragma unroll
        for (int b = 0; b < r; ++b) A3[a * r + b] = (a >= jr && b == a - jr) ? one : acc[b];
    }
    for (int cc = threadIdx.x; cc < m; cc += blockDim.x) {
        T acc[r];
#pragma unroll
        for (int b = 0; b < r; ++b) acc[b] = Sc<T>::zero();
        if (cc < jr) {
            for (int q = 0; q < jr; ++q) {
                const T x = Xm[(size_t)q * KRM + cc];
#pragma unroll
                for (int b = 0; b < r; ++b) acc[b] -= A2[b * jr + q] * x;
            }
        }
#pragma unroll
        for (int b = 0; b < r; ++b) A4[b * m + cc] = (cc >= jr && b == cc - jr) ? one : acc[b];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < m * r; e += blockDim.x) {
        int a = e / r, b = e - a * r;
        T acc = Sc<T>::zero();
        for (int q = 0; q < r; ++q) acc += A3[a * r + q] * Sc<T>::from(Z[q * r + b]);
        A1[e] = acc;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
        int a = e / m, cc = e - a * m;
        T* xp = Xm + (size_t)a * KRM + cc;
        T acc = *xp;
        for (int b = 0; b < r; ++b) acc += A1[a * r + b] * A4[b * m + cc];
        *xp = acc;
    }
    __syncthreads();
}

// One CTA (NWARP warps) per chain runs the batch's kb link steps in order.
// SU2: SU(2) links (quaternion proposal and doublet twist); the Z2 and U(1)
// instantiations (SU2 = false) do not contain that code.
template <class RW, class CW, bool SU2>
__global__ void __launch_bounds__(NWARP * 32, 2) batch_steps(BatchArgs a) {
    extern __shared__ cxd sm[];
    const Geometry& g = a.dc.g;
    const int P = a.dc.P, K = a.dc.K, Kc = P - K, r = g.r, N = g.N, KRM = a.KRM;
    const int c = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // the ratio phase's arrays and the update scratch share the front of
    // shared memory; Z and the T list follow
    const size_t front_ratio = (size_t)(2 * P * r * r + NWARP * 4 * r * r + P + NWARP * r);
    const size_t front_upd = (4 * (size_t)KRM * r * sizeof(CW) + sizeof(cxd) - 1) / sizeof(cxd);
    const size_t front = front_ratio > front_upd ? front_ratio : front_upd;
    cxd* Delta = sm;                       // [P][r][r]
    cxd* Wss = Delta + P * r * r;          // [P][r][r]
    cxd* Bord = Wss + P * r * r;           // [NWARP][2r][2r]
    cxd* rho = Bord + NWARP * 4 * r * r;   // [P]
    cxd* fcol = rho + P;                   // [NWARP][r]
    cxd* Zs = sm + front;                  // [P][r][r]
    int* Tl = (int*)(Zs + P * r * r);      // [kb r]
    __shared__ Proposal s_q;
    __shared__ double s_cs[8];
    __shared__ double s_su2[36];          // SU2: new quaternion, old and new doublet rotations
    __shared__ int s_accept, s_any;
    typedef typename Sc<RW>::R RR;
    const size_t NK = panel_plane(N, KRM), SS = (size_t)KRM * KRM;
    const int NP = panel_rows(N);
    const int kr = a.kb * r;
    for (int q = threadIdx.x; q < kr; q += blockDim.x) {
        int a0, b0;
        link_ends(g, a.l0 + q / r, a0, b0);
        Tl[q] = link_majorana(g, a0, b0, q % r);
    }
    if (threadIdx.x == 0) s_any = 0;
    __syncthreads();
    const unsigned long long sweep = *a.d_sweep;

    for (int j = 0; j < a.kb; ++j) {
        const int l = a.l0 + j, jr = j * r;
        if constexpr (SU2) {
            if (threadIdx.x == 0) {
                Proposal qq{};
                qq.u_acc = draw_su2(g, a.links, c, l, sweep, a.seed, a.width, s_su2, s_su2 + 4, s_su2 + 20,
                                   a.coff);
                s_q = qq;
            }
        } else {
            if (threadIdx.x == 0) s_q = draw_proposal(g, a.links, c, l, sweep, a.seed, a.width, a.coff);
        }
        __syncthreads();
        const Proposal q = s_q;
        if constexpr (!SU2) twist_table(g, q, s_cs);
        __syncthreads();
        for (int p = warp; p < P; p += NWARP) {
            cxd* D = Delta + p * r * r;
            cxd* Ws = Wss + p * r * r;
            if constexpr (SU2) pair_delta_su2(a.dc, p, l, s_su2 + 4, s_su2 + 20, D);
            else pair_delta(a.dc, p, l, q, s_cs, D);
            for (int e = lane; e < r * r; e += 32) {
                const size_t off = (size_t)(jr + e / r) * KRM + jr + e % r;
                if (p < K) Ws[e] = loadc((const RW*)a.Sr + ((size_t)c * K + p) * 2 * SS + off);
                else Ws[e] = loadc((const CW*)a.Sc_ + ((size_t)c * Kc + (p - K)) * 2 * SS + off);
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
            const int acc = (sn > 0.0 && so > 0.0 && q.u_acc < sn / so) ? 1 : 0;
            atomicAdd(&a.counters[0], 1ULL);
            s_accept = acc;
            if (acc) {
                s_any = 1;
                atomicAdd(&a.counters[1], 1ULL);
                a.since_refresh[c] += 1;
                a.sweep_acc[c] += 1;
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
        if (!s_accept) continue;
        for (int p = warp; p < P; p += NWARP) {
            pair_z(Delta + p * r * r, Wss + p * r * r, Bord + warp * 4 * r * r, fcol + warp * r, r, Zs + p * r * r);
            if (lane == 0) ell_add(a.ell[(size_t)c * P + p], rho[p], p < K);
            __syncwarp();
        }
        __syncthreads();
        for (int p = 0; p < K; ++p) {
            RW* Gm = (RW*)a.Sr + ((size_t)c * K + p) * 2 * SS;
            const RR* U = (const RR*)a.Pr + ((size_t)c * K + p) * 2 * PanelIO<RW>::PLANES * NK;
            if (r == 4) small_update<RW, 4>(Gm, Gm + SS, U, NK, NP, Tl, j, a.kb, KRM, Zs + p * r * r, (RW*)sm);
            else small_update<RW, 8>(Gm, Gm + SS, U, NK, NP, Tl, j, a.kb, KRM, Zs + p * r * r, (RW*)sm);
        }
        for (int p = 0; p < Kc; ++p) {
            CW* Gm = (CW*)a.Sc_ + ((size_t)c * Kc + p) * 2 * SS;
            const RR* U = (const RR*)a.Pc + ((size_t)c * Kc + p) * 2 * PanelIO<CW>::PLANES * NK;
            if (r == 4) small_update<CW, 4>(Gm, Gm + SS, U, NK, NP, Tl, j, a.kb, KRM, Zs + (K + p) * r * r, (CW*)sm);
            else small_update<CW, 8>(Gm, Gm + SS, U, NK, NP, Tl, j, a.kb, KRM, Zs + (K + p) * r * r, (CW*)sm);
        }
    }
    if (threadIdx.x == 0) a.pend[c] = s_any ? a.kb : 0;
}

size_t steps_smem(int P, int r, int KRM, size_t cw_bytes) {
    size_t front = std::max((size_t)(2 * P * r * r + NWARP * 4 * r * r + P + NWARP * r),
                            (4 * (size_t)KRM * r * cw_bytes + sizeof(cxd) - 1) / sizeof(cxd));
    return (front + (size_t)P * r * r) * sizeof(cxd) + (size_t)KRM * sizeof(int);
}

// ---- V^T <- V^T X^T -----------------------------------------------------------
// Grid (ceil(N / RB), family pairs, chains) with RB = 16 RPT rows per CTA,
// 256 threads as 16 x 16.  A CTA stages its RB rows of V^T in shared memory
// and rewrites them in place; per 128-wide output chunk, thread (ty, tx)
// accumulates rows ty RPT .. + RPT - 1 x outputs tx + 16 t (t = 0 .. 7) over
// the rank, with X^T staged 16 columns at a time.  Interleaved outputs make
// the 16 threads of a row read 16 consecutive elements of a staged X^T row
// (contiguous blocks of 8 per thread put them 8 elements apart: 4- to 16-way
// bank conflicts) and write 8 consecutive rank columns of a panel chunk.
constexpr int AP_LDX = 132;   // X^T stage row length (128 outputs + pad, 16-byte rows)

template <class T, int RPT>
__global__ void __launch_bounds__(256) batch_apply(int N, int fam_pairs, int KRM, int kr, typename Sc<T>::R* Pan,
                                                   const T* Sm, const int* pend) {
    typedef typename Sc<T>::R RR;
    constexpr int RB = 16 * RPT;
    const int c = blockIdx.z;
    if (pend[c] == 0) return;
    const int p = blockIdx.y;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int ld = kr + 1;
    T* Xs = (T*)smraw;           // [16][AP_LDX]  X^T chunk: Xs[bb][aa] = X[a0 + aa][b0 + bb]
    T* Vs = Xs + 16 * AP_LDX;    // [RB][kr + 1]
    const size_t NK = panel_plane(N, KRM), base = (size_t)c * fam_pairs + p;
    const int NP = panel_rows(N);
    RR* Vt = Pan + base * 2 * PanelIO<T>::PLANES * NK + PanelIO<T>::PLANES * NK;
    const T* Xm = Sm + base * 2 * KRM * KRM + (size_t)KRM * KRM;
    const int i0 = blockIdx.x * RB, nb = min(RB, N - i0);
    for (int e = threadIdx.x; e < RB * kr; e += blockDim.x) {
        int ii = e / kr, q = e - ii * kr;
        Vs[ii * ld + q] = ii < nb ? PanelIO<T>::ld(Vt, NK, pidx(i0 + ii, q, NP)) : Sc<T>::zero();
    }
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    for (int a0 = 0; a0 < kr; a0 += 128) {
        T acc[RPT][8];
#pragma unroll
        for (int u = 0; u < RPT; ++u)
#pragma unroll
            for (int t = 0; t < 8; ++t) acc[u][t] = Sc<T>::zero();
        // X chunks are loaded into registers one chunk ahead (8 values per
        // thread), so their global loads overlap the previous chunk's products
        T xn[8];
#pragma unroll
        for (int w = 0; w < 8; ++w) {
            const int e = threadIdx.x + w * 256, aa = e >> 4, bb = e & 15;
            xn[w] = (a0 + aa < kr && bb < kr) ? Xm[(size_t)(a0 + aa) * KRM + bb] : Sc<T>::zero();
        }
        for (int b0 = 0; b0 < kr; b0 += 16) {
            __syncthreads();
#pragma unroll
            for (int w = 0; w < 8; ++w) {
                const int e = threadIdx.x + w * 256;
                Xs[(e & 15) * AP_LDX + (e >> 4)] = xn[w];
            }
            __syncthreads();
            if (b0 + 16 < kr) {
#pragma unroll
                for (int w = 0; w < 8; ++w) {
                    const int e = threadIdx.x + w * 256, aa = e >> 4, bb = b0 + 16 + (e & 15);
                    xn[w] = (a0 + aa < kr && bb < kr) ? Xm[(size_t)(a0 + aa) * KRM + bb] : Sc<T>::zero();
                }
            }
            const int bn = min(16, kr - b0);
            for (int bb = 0; bb < bn; ++bb) {
                T v[RPT], x[8];
#pragma unroll
                for (int u = 0; u < RPT; ++u) v[u] = Vs[(ty * RPT + u) * ld + b0 + bb];
#pragma unroll
                for (int t = 0; t < 8; ++t) x[t] = Xs[bb * AP_LDX + tx + 16 * t];
#pragma unroll
                for (int u = 0; u < RPT; ++u)
#pragma unroll
                    for (int t = 0; t < 8; ++t) acc[u][t] += v[u] * x[t];
            }
        }
#pragma unroll
        for (int u = 0; u < RPT; ++u) {
            const int ii = ty * RPT + u;
            if (ii >= nb) continue;
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const int aa = a0 + tx + 16 * t;
                if (aa < kr) PanelIO<T>::st(Vt, NK, pidx(i0 + ii, aa, NP), acc[u][t]);
            }
        }
    }
}

size_t apply_smem(int RPT, int kr, size_t tb) { return (16 * AP_LDX + (size_t)16 * RPT * (kr + 1)) * tb; }

int gather_rows(int kr, size_t tb) {
    int br = 32;
    while (br > 4 && (size_t)br * (kr + 1) * tb > 96 * 1024) br >>= 1;
    return br;
}

}  // namespace

ggf_status ggf_flush(ggf_ctx* ctx, cudaStream_t st);
ggf_status ggf_apply_tc(ggf_ctx* ctx, bool cplx, int fam_pairs, int kr, float* Pan, const float* Sm, cudaStream_t st);

// Shared-memory caps of the batch kernels (once per device, like the other
// sampler kernels), and the largest batch that fits.
ggf_status ggf_prepare_batch(ggf_ctx* ctx) {
    static bool done[64] = {false};
    if (ctx->device >= 0 && ctx->device < 64 && done[ctx->device]) return GGF_OK;
    int mx = 0;
    GGF_CK(cudaDeviceGetAttribute(&mx, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device));
    auto cap = [&](const void* fn) -> ggf_status {
        cudaFuncAttributes fa;
        GGF_CK(cudaFuncGetAttributes(&fa, fn));
        GGF_CK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, mx - (int)fa.sharedSizeBytes));
        return GGF_OK;
    };
    GGF_TRY(cap((const void*)batch_gather<double>));
    GGF_TRY(cap((const void*)batch_gather<float>));
    GGF_TRY(cap((const void*)batch_gather<cxd>));
    GGF_TRY(cap((const void*)batch_gather<cxf>));
    GGF_TRY(cap((const void*)batch_steps<double, cxd, false>));
    GGF_TRY(cap((const void*)batch_steps<float, cxf, false>));
    GGF_TRY(cap((const void*)batch_steps<double, cxd, true>));
    GGF_TRY(cap((const void*)batch_steps<float, cxf, true>));
    GGF_TRY(cap((const void*)batch_apply<double, 4>));
    GGF_TRY(cap((const void*)batch_apply<float, 4>));
    GGF_TRY(cap((const void*)batch_apply<cxd, 4>));
    GGF_TRY(cap((const void*)batch_apply<cxf, 4>));
    GGF_TRY(cap((const void*)batch_apply<double, 2>));
    GGF_TRY(cap((const void*)batch_apply<float, 2>));
    GGF_TRY(cap((const void*)batch_apply<cxd, 2>));
    GGF_TRY(cap((const void*)batch_apply<cxf, 2>));
    if (ctx->device >= 0 && ctx->device < 64) done[ctx->device] = true;
    return GGF_OK;
}

// Shared memory the batch kernels need for batches of kmax links; EINVAL if
// it exceeds the device's per-block limit.
ggf_status ggf_check_batch(ggf_ctx* ctx, int kmax, bool fp64) {
    int mx = 0;
    GGF_CK(cudaDeviceGetAttribute(&mx, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device));
    const int r = ctx->g.r, KRM = kmax * r;
    const size_t cw = fp64 ? sizeof(cxd) : sizeof(cxf);
    const size_t need_steps = steps_smem(ctx->P, r, KRM, cw) + 1024;
    const size_t need_apply = apply_smem(2, KRM, cw) + 1024;
    if (need_steps > (size_t)mx || need_apply > (size_t)mx)
        return ggf_fail(ctx, GGF_EINVAL, "delay too large: batch kernels need more shared memory than the device has");
    return GGF_OK;
}

// Run links l0 .. l0 + kb - 1 of the sweep as one batch (gather, link steps,
// X applied to the V panel, flush).
ggf_status ggf_batch(ggf_ctx* ctx, int l0, int kb, cudaStream_t st) {
    Chains& ch = ctx->ch;
    const Geometry& g = ctx->g;
    const bool fp64 = ch.opts.precision == GGF_FP64;
    const int N = g.N, r = g.r, KRM = ch.kmax * r, kr = kb * r;
    const size_t rsz = fp64 ? sizeof(double) : sizeof(float);
    const size_t ssz = (size_t)ch.n * 2 * KRM * KRM * rsz;   // one family pair's small matrices, all chains
    void* Sr = ch.Sm;
    void* Sc_ = (unsigned char*)ch.Sm + ssz * ctx->K;
    const int ev0 = ctx->prof_mark(st);
    {
        const int br_r = gather_rows(kr, rsz), br_c = gather_rows(kr, 2 * rsz);
        dim3 gr((N + br_r - 1) / br_r, ctx->K, ch.n), gc((N + br_c - 1) / br_c, ctx->Kc, ch.n);
        const size_t t0 = (kr * sizeof(int) + 15) & ~(size_t)15;
        if (fp64) {
            batch_gather<double><<<gr, 256, t0 + (size_t)br_r * (kr + 1) * rsz, st>>>(
                g, l0, kb, ctx->K, KRM, br_r, (const double*)ch.Wr, (double*)ch.Pr, (double*)Sr);
            if (ctx->Kc)
                batch_gather<cxd><<<gc, 256, t0 + (size_t)br_c * (kr + 1) * 2 * rsz, st>>>(
                    g, l0, kb, ctx->Kc, KRM, br_c, (const cxd*)ch.Wc, (double*)ch.Pc, (cxd*)Sc_);
        } else {
            batch_gather<float><<<gr, 256, t0 + (size_t)br_r * (kr + 1) * rsz, st>>>(
                g, l0, kb, ctx->K, KRM, br_r, (const float*)ch.Wr, (float*)ch.Pr, (float*)Sr);
            if (ctx->Kc)
                batch_gather<cxf><<<gc, 256, t0 + (size_t)br_c * (kr + 1) * 2 * rsz, st>>>(
                    g, l0, kb, ctx->Kc, KRM, br_c, (const cxf*)ch.Wc, (float*)ch.Pc, (cxf*)Sc_);
        }
        GGF_CK(cudaGetLastError());
    }
    const int ev1 = ctx->prof_mark(st);
    ctx->prof_pair(GGF_KT_GATHER, ev0, ev1);
    {
        BatchArgs a;
        a.dc = ctx->dc();
        a.d_sweep = ch.d_sweep;
        a.l0 = l0;
        a.kb = kb;
        a.KRM = KRM;
        a.seed = ch.opts.seed;
        a.coff = ch.opts.chain_offset;
        a.width = ch.opts.width;
        a.links = ch.links;
        a.ell = ch.ell;
        a.since_refresh = ch.since_refresh;
        a.sweep_acc = ch.sweep_acc;
        a.counters = ch.counters;
        a.pend = ch.pend;
        a.Pr = ch.Pr;
        a.Pc = ch.Pc;
        a.Sr = Sr;
        a.Sc_ = Sc_;
        const size_t smem = steps_smem(ctx->P, r, KRM, fp64 ? sizeof(cxd) : sizeof(cxf));
        if (g.group == GGF_SU2) {
            if (fp64) batch_steps<double, cxd, true><<<ch.n, NWARP * 32, smem, st>>>(a);
            else batch_steps<float, cxf, true><<<ch.n, NWARP * 32, smem, st>>>(a);
        } else {
            if (fp64) batch_steps<double, cxd, false><<<ch.n, NWARP * 32, smem, st>>>(a);
            else batch_steps<float, cxf, false><<<ch.n, NWARP * 32, smem, st>>>(a);
        }
        GGF_CK(cudaGetLastError());
    }
    const int ev2 = ctx->prof_mark(st);
    ctx->prof_pair(GGF_KT_RATIO, ev1, ev2);
    {
        int mx = 0;
        GGF_CK(cudaDeviceGetAttribute(&mx, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device));
        // 64-row blocks where they fit in shared memory, else 32
        const int rpt_r = apply_smem(4, kr, rsz) + 1024 <= (size_t)mx ? 4 : 2;
        const int rpt_c = apply_smem(4, kr, 2 * rsz) + 1024 <= (size_t)mx ? 4 : 2;
        dim3 gr((N + 16 * rpt_r - 1) / (16 * rpt_r), ctx->K, ch.n), gc((N + 16 * rpt_c - 1) / (16 * rpt_c), ctx->Kc, ch.n);
        const size_t sr = apply_smem(rpt_r, kr, rsz), sc = apply_smem(rpt_c, kr, 2 * rsz);
#define GGF_APPLY(T, RPT, grid, smem, fam, Pp, Sp) \
    batch_apply<T, RPT><<<grid, 256, smem, st>>>(N, fam, KRM, kr, (typename Sc<T>::R*)(Pp), (const T*)(Sp), ch.pend)
        if (GGF_APPLY_TC && !fp64 && ctx->use_tc && kr <= 256 && g.group != GGF_Z2) {
            // FP32 chains: the X product on the tensor cores (TF32 split).  Z2
            // chains keep the FMA-pipe product: a flip is a large change, and
            // the tensor-core accumulation doubled their FP32 drift (measured
            // 3.3e-6 against 1.7e-6 per accept at 16 x 16), while the small
            // moves of U(1) and SU(2) chains are unaffected (1e-8 per accept)
            GGF_TRY(ggf_apply_tc(ctx, false, ctx->K, kr, (float*)ch.Pr, (const float*)Sr, st));
            GGF_TRY(ggf_apply_tc(ctx, true, ctx->Kc, kr, (float*)ch.Pc, (const float*)Sc_, st));
        } else if (fp64) {
            if (rpt_r == 4) GGF_APPLY(double, 4, gr, sr, ctx->K, ch.Pr, Sr); else GGF_APPLY(double, 2, gr, sr, ctx->K, ch.Pr, Sr);
            if (ctx->Kc) {
                if (rpt_c == 4) GGF_APPLY(cxd, 4, gc, sc, ctx->Kc, ch.Pc, Sc_); else GGF_APPLY(cxd, 2, gc, sc, ctx->Kc, ch.Pc, Sc_);
            }
        } else {
            if (rpt_r == 4) GGF_APPLY(float, 4, gr, sr, ctx->K, ch.Pr, Sr); else GGF_APPLY(float, 2, gr, sr, ctx->K, ch.Pr, Sr);
            if (ctx->Kc) {
                if (rpt_c == 4) GGF_APPLY(cxf, 4, gc, sc, ctx->Kc, ch.Pc, Sc_); else GGF_APPLY(cxf, 2, gc, sc, ctx->Kc, ch.Pc, Sc_);
            }
        }
#undef GGF_APPLY
        GGF_CK(cudaGetLastError());
    }
    ctx->prof_pair(GGF_KT_APPLY, ev2, ctx->prof_mark(st));
    ctx->launches += 1 + 2 * (1 + (ctx->Kc ? 1 : 0));
    ch.steps_since_flush = kb;
    return ggf_flush(ctx, st);
}
