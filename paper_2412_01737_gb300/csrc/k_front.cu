// FP64 log-Pfaffian of M_nm(G) (Sec. 5: N_nm(G) = c_nm Pf(M_nm(G))) by a
// site-by-site elimination that follows the lattice.
//
// M = D + O(G) Gamma_X O(G)^T couples a virtual Majorana only to the other
// Majoranas of its own site (the block D and the link block of its own end)
// and to the partner end of its link.  Sites are added in index order
// s = 0 .. V-1; after adding site s, every Majorana whose site and link
// partner are both added is "closed": no later site couples to it, so it can
// be eliminated from the dense "front" (the Schur complement of M on the
// added, not yet eliminated Majoranas).  With M = [[A, B], [-B^T, C]] and A
// the block of one eliminated pair (k, p),
//     Pf(M) = M_kp Pf(C + (v u^T - u v^T) / M_kp),   u = M[k, rest], v = M[p, rest]
// (Schur complement of a skew matrix), after moving k, p to the front, which
// multiplies Pf by the sign of that permutation.  Pairs are chosen within the
// closed set by the largest |entry| (pivoting restricted to the closed set).
//
// The front of a periodic L x L lattice holds two rows of link ends (the
// +y ends of the last L sites and the -y ends of row 0, which wait for the
// periodic wrap) plus a few ends of the current row: at 16 x 16, n_v = 2 at
// most 152 of the N = 4096 Majoranas, so one matrix costs ~4e7 FP64 FMAs
// instead of the N^3/6 ~ 1.1e10 of a dense Pfaffian.  The front lives in
// shared memory as a packed upper triangle (skew-symmetric storage), one CTA
// per (configuration, pair) item; fronts too large for shared memory use a
// global-memory slice per CTA.
//
// Sign: Pf(M) = sgn(sigma) prod_t M^(t)_{k_t p_t} with sigma the elimination
// sequence (k_1, p_1, k_2, p_2, ...).  The parity of sigma is accumulated as
// the number of earlier-eliminated Majoranas with a larger index, for each
// eliminated one: with all Majoranas of sites > s still to come (their
// indices are larger), that count is (N - 1 - v) - #(front entries > v) -
// (N - (s + 1) B).
#include <algorithm>
#include <map>
#include <vector>
#include "ggf_ctx.h"
#include "ggf_geom.cuh"

namespace {

constexpr int FT = 512;                 // threads per CTA
constexpr int FW = FT / 32;

__device__ __forceinline__ int tri_row(int i, int F) { return i * (2 * F - i - 1) / 2 - i - 1; }

template <class T> __device__ __forceinline__ T fzero();
template <> __device__ __forceinline__ double fzero<double>() { return 0.0; }
template <> __device__ __forceinline__ cxd fzero<cxd>() { return {0.0, 0.0}; }
__device__ __forceinline__ double fmag(double v) { return fabs(v); }
__device__ __forceinline__ double fmag(cxd v) { return hypot(v.x, v.y); }
__device__ __forceinline__ bool fnz(double v) { return v != 0.0; }
__device__ __forceinline__ bool fnz(cxd v) { return v.x != 0.0 || v.y != 0.0; }
__device__ __forceinline__ double fneg(double v) { return -v; }
__device__ __forceinline__ cxd fneg(cxd v) { return {-v.x, -v.y}; }
__device__ __forceinline__ double fdiv(double a, double b) { return a / b; }
__device__ __forceinline__ cxd fdiv(cxd a, cxd b) { return a / b; }
__device__ __forceinline__ cxd funit(double v) { return {v >= 0 ? 1.0 : -1.0, 0.0}; }
__device__ __forceinline__ cxd funit(cxd v) {
    double m = hypot(v.x, v.y);
    return {v.x / m, v.y / m};
}
// r += a * b - c * d
__device__ __forceinline__ void frank2(double& r, double a, double b, double c, double d) {
    r = fma(a, b, r);
    r = fma(-c, d, r);
}
__device__ __forceinline__ void frank2(cxd& r, cxd a, cxd b, cxd c, cxd d) {
    double x = r.x, y = r.y;
    x = fma(a.x, b.x, x); x = fma(-a.y, b.y, x); x = fma(-c.x, d.x, x); x = fma(c.y, d.y, x);
    y = fma(a.x, b.y, y); y = fma(a.y, b.x, y); y = fma(-c.x, d.y, y); y = fma(-c.y, d.x, y);
    r = {x, y};
}

// S(a, b) of the packed strict upper triangle, skew-symmetric
template <class T>
__device__ __forceinline__ T sget(const T* S, int F, int a, int b) {
    if (a < b) return S[tri_row(a, F) + b];
    if (a > b) return fneg(S[tri_row(b, F) + a]);
    return fzero<T>();
}

struct FrontArgs {
    int F;              // slots of the front
    int N, B, V;
    const int* slot;    // [N] slot of Majorana i (fixed by the schedule)
    const int* eoff;    // [V + 1] offsets into elim
    const int* elim;    // slots eliminated after adding site s
};

// One CTA per item (grid-stride over items).  Dynamic shared memory: u[F],
// v[F] (T), idx[F], es[F] (int), then the packed triangle when it fits.
template <class T>
__global__ void __launch_bounds__(FT, 1)
front_pf_kernel(DevConst dc, FrontArgs fa, int n_items, const int* item_cfg, const int* item_pair, const void* links,
                cxd* logpf, cxd* phase, int* flag, T* gws, size_t tri_elems, int in_smem) {
    extern __shared__ __align__(16) unsigned char fsm[];
    __shared__ int s_k, s_p, s_bad;
    const int F = fa.F, N = fa.N, B = fa.B, V = fa.V;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    T* u = (T*)fsm;
    T* v = u + F;
    int* idx = (int*)(v + F);
    int* es = idx + F;
    T* S = in_smem ? (T*)(fsm + (((size_t)F * (2 * sizeof(T) + 2 * sizeof(int)) + 15) / 16) * 16)
                   : gws + (size_t)blockIdx.x * tri_elems;
    const Geometry& g = dc.g;
    for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int cfg = item_cfg[item], pair = item_pair[item];
        for (int a = tid; a < F; a += FT) idx[a] = -1;
        if (tid == 0) s_bad = 0;
        double logabs = 0.0;   // meaningful in thread 0
        cxd ph = {1.0, 0.0};
        int par = 0;
        __syncthreads();
        for (int s = 0; s < V && !s_bad; ++s) {
            // ---- add site s: its B Majoranas take their slots, their rows are M's entries
            for (int k = tid; k < B; k += FT) idx[fa.slot[s * B + k]] = s * B + k;
            __syncthreads();
            for (int w = tid; w < B * F; w += FT) {
                const int k = w / F, b = w - k * F;
                const int a = fa.slot[s * B + k];
                const int jb = idx[b];
                if (b == a || jb < 0) continue;
                if (jb >= s * B && b < a) continue;        // new-new pair: written once, by the lower slot's row
                const int lo = min(a, b), hi = max(a, b);
                const int i = idx[lo], j = idx[hi];
                T val = fzero<T>();
                const int si = i / B, sj = j / B;
                int li, pi, lj, pj;
                link_of(g, i, li, pi);
                link_of(g, j, lj, pj);
                if (si == sj || li == lj) val = assemble_elem<T>(dc, links, cfg, pair, i, j);
                S[tri_row(lo, F) + hi] = val;
            }
            // ---- eliminate the closed Majoranas in pivoted pairs
            const int e0 = fa.eoff[s], e1 = fa.eoff[s + 1];
            for (int t = tid; t < e1 - e0; t += FT) es[t] = fa.elim[e0 + t];
            __syncthreads();
            for (int t = 0; t < e1 - e0; t += 2) {
                if (warp == 0) {
                    const int ne = e1 - e0 - t;
                    double best = -1.0;
                    int bq = 0;
                    for (int q = lane; q < ne * ne; q += 32) {
                        const int x = q / ne, y = q - x * ne;
                        if (x >= y) continue;
                        const double m = fmag(sget(S, F, es[t + x], es[t + y]));
                        if (m > best) { best = m; bq = q; }
                    }
                    for (int o = 16; o > 0; o >>= 1) {
                        const double ob = __shfl_down_sync(0xffffffffu, best, o);
                        const int oq = __shfl_down_sync(0xffffffffu, bq, o);
                        if (ob > best || (ob == best && oq < bq)) { best = ob; bq = oq; }
                    }
                    if (lane == 0) {
                        const int x = bq / ne, y = bq - (bq / ne) * ne;
                        const int k = es[t + x], p = es[t + y];
                        if (!(best > 1e-8) || !isfinite(best)) s_bad = 1;   // no usable pivot: refactor densely
                        // move the pair to positions t, t + 1 of the closed list (x < y,
                        // so the first swap leaves position t + y alone)
                        es[t + x] = es[t];
                        es[t] = k;
                        es[t + y] = es[t + 1];
                        es[t + 1] = p;
                        s_k = k;
                        s_p = p;
                    }
                }
                __syncthreads();
                if (s_bad) break;
                const int k = s_k, p = s_p;
                const T akp = sget(S, F, k, p);
                if (warp == 0) {
                    // parity of the elimination sequence: k, then p
                    const int vk = idx[k], vp = idx[p];
                    int ck = 0, cp = 0;
                    for (int b = lane; b < F; b += 32) {
                        const int j = idx[b];
                        if (j < 0 || b == k) continue;
                        ck += j > vk;
                        if (b != p) cp += j > vp;
                    }
                    for (int o = 16; o > 0; o >>= 1) {
                        ck += __shfl_down_sync(0xffffffffu, ck, o);
                        cp += __shfl_down_sync(0xffffffffu, cp, o);
                    }
                    if (lane == 0) {
                        const int later = N - (s + 1) * B;
                        par ^= ((N - 1 - vk) - ck - later) & 1;
                        par ^= ((N - 1 - vp) - cp - later) & 1;
                        logabs += log(fmag(akp));
                        ph = ph * funit(akp);
                    }
                }
                for (int b = tid; b < F; b += FT) {
                    const bool live = idx[b] >= 0 && b != k && b != p;
                    u[b] = live ? fdiv(sget(S, F, k, b), akp) : fzero<T>();
                    v[b] = live ? sget(S, F, p, b) : fzero<T>();
                }
                __syncthreads();
                if (tid == 0) { idx[k] = -1; idx[p] = -1; }
                // C += v u^T - u v^T on the strict upper triangle
                for (int i = warp; i < F - 1; i += FW) {
                    const T vi = v[i], ui = u[i];
                    if (!fnz(vi) && !fnz(ui)) continue;
                    T* row = S + tri_row(i, F);
                    for (int j = i + 1 + lane; j < F; j += 32) frank2(row[j], vi, u[j], ui, v[j]);
                }
                __syncthreads();
            }
        }
        if (tid == 0) {
            flag[item] = s_bad;
            if (s_bad) {
                logpf[item] = {NAN, 0.0};
                phase[item] = {0.0, 0.0};
            } else {
                logpf[item] = {logabs, 0.0};
                phase[item] = par ? cxd{-ph.x, -ph.y} : ph;
            }
        }
        __syncthreads();
    }
}

// Elimination schedule for an L x L lattice with B virtual Majoranas per
// site: slot of every Majorana and the slots closed after each site.
void build_schedule(const Geometry& g, int& F, std::vector<int>& slot, std::vector<int>& eoff,
                    std::vector<int>& elim) {
    const int B = g.B, V = g.V, N = g.N, L = g.L;
    slot.assign(N, -1);
    eoff.assign(V + 1, 0);
    elim.clear();
    auto partner_site = [&](int s, int e) {
        const int x = s % L, y = s / L, d = e >> 1;
        if (e & 1) return d == 0 ? y * L + (x + 1) % L : ((y + 1) % L) * L + x;
        return d == 0 ? y * L + (x + L - 1) % L : ((y + L - 1) % L) * L + x;
    };
    std::vector<int> free_slots, front;
    int next = 0;
    F = 0;
    for (int s = 0; s < V; ++s) {
        for (int k = 0; k < B; ++k) {
            int sl;
            if (!free_slots.empty()) {
                auto it = std::min_element(free_slots.begin(), free_slots.end());
                sl = *it;
                free_slots.erase(it);
            } else {
                sl = next++;
            }
            slot[s * B + k] = sl;
            front.push_back(s * B + k);
        }
        F = std::max(F, next);
        std::vector<int> keep;
        for (int i : front) {
            const int si = i / B, e = (i % B) / g.h2;
            if (partner_site(si, e) <= s) {
                elim.push_back(slot[i]);
                free_slots.push_back(slot[i]);
            } else {
                keep.push_back(i);
            }
        }
        front.swap(keep);
        eoff[s + 1] = (int)elim.size();
    }
}

}  // namespace

// Shared memory of the front kernel for F slots (without / with the triangle).
static size_t front_smem(int F, size_t elem, bool tri) {
    size_t b = (((size_t)F * (2 * elem + 2 * sizeof(int)) + 15) / 16) * 16;
    if (tri) b += (size_t)F * (F - 1) / 2 * elem;
    return b;
}

// opt-in shared memory per CTA (227 KB) less a margin for the static variables
static const size_t kSmemMax = 227 * 1024 - 1024;

ggf_status ggf_front_prepare(ggf_ctx* ctx) {
    const Geometry& g = ctx->g;
    if (ctx->d_front && ctx->front_L == g.L && ctx->front_B == g.B) return GGF_OK;
    if (ctx->d_front) cudaFree(ctx->d_front);
    ctx->d_front = nullptr;
    int F = 0;
    std::vector<int> slot, eoff, elim;
    build_schedule(g, F, slot, eoff, elim);
    if ((int)elim.size() != g.N) return ggf_fail(ctx, GGF_ESTATE, "front schedule does not close every Majorana");
    std::vector<int> all;
    all.insert(all.end(), slot.begin(), slot.end());
    all.insert(all.end(), eoff.begin(), eoff.end());
    all.insert(all.end(), elim.begin(), elim.end());
    GGF_CK(cudaMalloc(&ctx->d_front, all.size() * sizeof(int)));
    GGF_CK(cudaMemcpy(ctx->d_front, all.data(), all.size() * sizeof(int), cudaMemcpyHostToDevice));
    ctx->front_F = F;
    ctx->front_L = g.L;
    ctx->front_B = g.B;
    static bool attr_done[64] = {false};
    if (ctx->device >= 0 && ctx->device < 64 && !attr_done[ctx->device]) {
        GGF_CK(cudaFuncSetAttribute(front_pf_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemMax));
        GGF_CK(cudaFuncSetAttribute(front_pf_kernel<cxd>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemMax));
        attr_done[ctx->device] = true;
    }
    return GGF_OK;
}

void ggf_front_free(ggf_ctx* ctx) {
    if (ctx->d_front) cudaFree(ctx->d_front);
    if (ctx->front_ws) cudaFree(ctx->front_ws);
    ctx->d_front = nullptr;
    ctx->front_ws = nullptr;
    ctx->front_ws_bytes = 0;
    ctx->front_L = ctx->front_B = -1;
}

int ggf_front_slots(ggf_ctx* ctx) { return ctx->front_F; }

// log Pf(M_nm(G)) of n_items (configuration, pair-within-family) items:
// d_logpf[item] = (log|Pf|, 0), d_phase[item] = Pf/|Pf|, d_flag[item] = 1
// where a closed set had no usable pivot (the caller refactors those items
// densely).  Links are device configurations indexed by d_item_cfg.
ggf_status ggf_front_pfaffian(ggf_ctx* ctx, bool cplx, int n_items, const int* d_item_cfg, const int* d_item_pair,
                              const void* d_links, cxd* d_logpf, cxd* d_phase, int* d_flag, cudaStream_t st) {
    if (n_items == 0) return GGF_OK;
    GGF_TRY(ggf_front_prepare(ctx));
    const Geometry& g = ctx->g;
    const int F = ctx->front_F;
    FrontArgs fa;
    fa.F = F;
    fa.N = g.N;
    fa.B = g.B;
    fa.V = g.V;
    fa.slot = ctx->d_front;
    fa.eoff = ctx->d_front + g.N;
    fa.elim = ctx->d_front + g.N + g.V + 1;
    const size_t elem = cplx ? sizeof(cxd) : sizeof(double);
    const bool in_smem = front_smem(F, elem, true) <= kSmemMax;
    const size_t tri = (size_t)F * (F - 1) / 2;
    int grid = std::min(n_items, 65535);
    void* ws = nullptr;
    if (!in_smem) {
        const int sms = ctx->n_sms > 0 ? ctx->n_sms : 152;
        grid = std::min(n_items, 2 * sms);
        const size_t need = (size_t)grid * tri * elem;
        if (need > ctx->front_ws_bytes) {
            if (ctx->front_ws) cudaFree(ctx->front_ws);
            ctx->front_ws = nullptr;
            ctx->front_ws_bytes = 0;
            GGF_CK(cudaMalloc(&ctx->front_ws, need));
            ctx->front_ws_bytes = need;
        }
        ws = ctx->front_ws;
    }
    const size_t smem = front_smem(F, elem, in_smem);
    ctx->launches += 1;
    if (cplx)
        front_pf_kernel<cxd><<<grid, FT, smem, st>>>(ctx->dc(), fa, n_items, d_item_cfg, d_item_pair, d_links, d_logpf,
                                                     d_phase, d_flag, (cxd*)ws, tri, in_smem ? 1 : 0);
    else
        front_pf_kernel<double><<<grid, FT, smem, st>>>(ctx->dc(), fa, n_items, d_item_cfg, d_item_pair, d_links,
                                                        d_logpf, d_phase, d_flag, (double*)ws, tri, in_smem ? 1 : 0);
    GGF_CK(cudaGetLastError());
    return GGF_OK;
}
