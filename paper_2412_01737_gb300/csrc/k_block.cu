// Block moves with the learned proposal (U(1) chains, delayed updates with
// room for 32 pending rank-r updates).
//
// One move per chain, all chains in lockstep:
//  1. fold pending updates into W;
//  2. block origin per chain (Philox, counter (move, 0, 21, 0), key (seed, chain));
//  3. network: new angles for the 32 block links and log q(new) - log q(old);
//  4. the 32 links are changed one after another as tentative rank-r updates
//     of the effective inverse (pending panels, W untouched); the product of
//     their Pfaffian ratios is the block's Pf(M')/Pf(M) for every pair, and the
//     tracked log-weights follow it;
//  5. Metropolis-Hastings: accept iff u < [N(G')/N(G)] q(old)/q(new)
//     (u from counter (move, 0, 23, 0)); a rejected move restores the links
//     and log-weights and drops the tentative panel entries;
//  6. fold the accepted updates into W.
#include "ggf_ctx.h"
#include "ggf_net.h"

ggf_status ggf_link_step_ex(ggf_ctx* ctx, int link, cudaStream_t st, const int* link_of_chain, const double* forced,
                            int forced_k, int* dead);
ggf_status ggf_flush(ggf_ctx* ctx, cudaStream_t st);
ggf_status ggf_observe(ggf_ctx* ctx, double* d_obs, cudaStream_t st);
ggf_status ggf_mark_refresh(ggf_ctx* ctx, cudaStream_t st);

namespace {

__global__ void block_origin(int n, int L, uint64_t seed, uint64_t koff, uint64_t move, int* blocks) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    uint64_t c4[4] = {move, 0, 21, 0}, o4[4];
    philox4x64_10(c4, seed, koff + (uint64_t)c, o4);
    blocks[2 * c] = min(L - 1, (int)(u53(o4[0]) * L));
    blocks[2 * c + 1] = min(L - 1, (int)(u53(o4[1]) * L));
}

// links of block step k for every chain, and the saved state
__global__ void block_prepare(int n, int L, int P, const int* blocks, const double* links, const cxd* ell,
                              int* link_k, double* old_links, cxd* ell_save, int* dead) {
    int c = blockIdx.x;
    if (c >= n) return;
    const int bx = blocks[2 * c], by = blocks[2 * c + 1];
    const int nl = 2 * L * L;
    for (int k = threadIdx.x; k < 32; k += blockDim.x) {
        int d = k & 1, q = k >> 1, i = q & 3, j = q >> 2;
        int s = ((by + j) % L) * L + (bx + i) % L;
        int l = 2 * s + d;
        link_k[(size_t)k * n + c] = l;
        old_links[(size_t)c * 32 + k] = links[(size_t)c * nl + l];
    }
    for (int p = threadIdx.x; p < P; p += blockDim.x) ell_save[(size_t)c * P + p] = ell[(size_t)c * P + p];
    if (threadIdx.x == 0) dead[c] = 0;
}

__device__ double combine_log(const DevConst& dc, const cxd* ell, double amax, bool* ok) {
    double s = 0.0;
    for (int p = 0; p < dc.P; ++p) {
        cxd e = dc.logc[p] + ell[p];
        if (p < dc.K) e.y = 0.0;
        e.x -= amax;
        s += (dc.w[p] * cexp_(e)).x;
    }
    *ok = s > 0.0;
    return s > 0.0 ? log(s) : -INFINITY;
}

__global__ void block_decide(DevConst dc, int n, const int* link_k, const double* lq, const double* old_links,
                             const cxd* ell_save, cxd* ell, double* links, int* pend, const int* dead,
                             int* since_refresh, int* sweep_acc, unsigned long long* counters, uint64_t seed,
                             uint64_t koff, uint64_t move) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    const int P = dc.P, nl = dc.g.n_links;
    const cxd* e0 = ell_save + (size_t)c * P;
    cxd* e1 = ell + (size_t)c * P;
    double amax = -INFINITY;
    for (int p = 0; p < P; ++p) amax = fmax(amax, fmax(dc.logc[p].x + e0[p].x, dc.logc[p].x + e1[p].x));
    bool ok0, ok1;
    double l0 = combine_log(dc, e0, amax, &ok0), l1 = combine_log(dc, e1, amax, &ok1);
    uint64_t c4[4] = {move, 0, 23, 0}, o4[4];
    philox4x64_10(c4, seed, koff + (uint64_t)c, o4);
    double u = u53(o4[0]);
    double logR = l1 - l0 - lq[c];
    bool acc = !dead[c] && ok0 && ok1 && (logR >= 0.0 || u < exp(logR));
    atomicAdd(&counters[4], 1ULL);
    if (acc) {
        atomicAdd(&counters[5], 1ULL);
        since_refresh[c] += 32;
        sweep_acc[c] = nl;
    } else {
        for (int k = 0; k < 32; ++k) links[(size_t)c * nl + link_k[(size_t)k * n + c]] = old_links[(size_t)c * 32 + k];
        for (int p = 0; p < P; ++p) e1[p] = e0[p];
        pend[c] = 0;   // drop the tentative panel entries (the move started with none pending)
        sweep_acc[c] = 0;
    }
}

}  // namespace

extern "C" ggf_status ggf_sample_blocks(ggf_ctx* ctx, ggf_net* net, int n_moves, double* obs, int mem, void* stream) {
    if (!ctx || !net) return GGF_EINVAL;
    if (!ctx->have_gauss || ctx->ch.n == 0) return ggf_fail(ctx, GGF_ESTATE, "chains not initialised");
    Chains& ch = ctx->ch;
    const Geometry& g = ctx->g;
    if (g.group != GGF_U1) return ggf_fail(ctx, GGF_EINVAL, "block moves are defined for U(1) links");
    if (ch.kmax < 32) return ggf_fail(ctx, GGF_EINVAL, "block moves need chains initialised with delay >= 32");
    if (ggf_net_L(net) != g.L) return ggf_fail(ctx, GGF_EINVAL, "network lattice size differs from the context's");
    if (g.L < 4) return ggf_fail(ctx, GGF_EINVAL, "block moves need L >= 4");
    if (n_moves < 0) return ggf_fail(ctx, GGF_EINVAL, "n_moves < 0");
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int n = ch.n, P = ctx->P;
    // scratch for the move (owned by the call)
    int *blocks = nullptr, *link_k = nullptr, *dead = nullptr;
    double *lq = nullptr, *prop = nullptr, *old_links = nullptr, *dobs = nullptr;
    cxd* ell_save = nullptr;
    ggf_status rc = GGF_OK;
    auto fail_cuda = [&](cudaError_t e, const char* w) { if (rc == GGF_OK) rc = ggf_cuda(ctx, e, w); };
    cudaError_t e;
    if ((e = cudaMalloc(&blocks, n * 2 * sizeof(int))) != cudaSuccess) fail_cuda(e, "alloc");
    if ((e = cudaMalloc(&link_k, (size_t)32 * n * sizeof(int))) != cudaSuccess) fail_cuda(e, "alloc");
    if ((e = cudaMalloc(&dead, n * sizeof(int))) != cudaSuccess) fail_cuda(e, "alloc");
    if ((e = cudaMalloc(&lq, n * sizeof(double))) != cudaSuccess) fail_cuda(e, "alloc");
    if ((e = cudaMalloc(&prop, (size_t)n * 32 * sizeof(double))) != cudaSuccess) fail_cuda(e, "alloc");
    if ((e = cudaMalloc(&old_links, (size_t)n * 32 * sizeof(double))) != cudaSuccess) fail_cuda(e, "alloc");
    if ((e = cudaMalloc(&ell_save, (size_t)n * P * sizeof(cxd))) != cudaSuccess) fail_cuda(e, "alloc");
    if (obs && mem == GGF_MEM_HOST && (e = cudaMalloc(&dobs, (size_t)n * GGF_N_OBS * sizeof(double))) != cudaSuccess)
        fail_cuda(e, "alloc");
    for (int mv = 0; mv < n_moves && rc == GGF_OK; ++mv) {
        const uint64_t move = ch.block_moves;
        if ((rc = ggf_flush(ctx, st)) != GGF_OK) break;
        block_origin<<<(n + 127) / 128, 128, 0, st>>>(n, g.L, ch.opts.seed, ch.opts.chain_offset, move, blocks);
        block_prepare<<<n, 32, 0, st>>>(n, g.L, P, blocks, (const double*)ch.links, ch.ell, link_k, old_links,
                                        ell_save, dead);
        if ((e = cudaGetLastError()) != cudaSuccess) { fail_cuda(e, "block_prepare"); break; }
        rc = ggf_net_head(net, n, 2, (const double*)ch.links, nullptr, blocks, lq, prop, ch.opts.seed, move, st,
                          ch.opts.chain_offset);
        if (rc != GGF_OK) { ctx->err = ggf_net_last_error(net); break; }
        for (int k = 0; k < 32 && rc == GGF_OK; ++k)
            rc = ggf_link_step_ex(ctx, -1, st, link_k + (size_t)k * n, prop, k, dead);
        if (rc != GGF_OK) break;
        block_decide<<<(n + 127) / 128, 128, 0, st>>>(ctx->dc(), n, link_k, lq, old_links, ell_save, ch.ell,
                                                      (double*)ch.links, ch.pend, dead, ch.since_refresh,
                                                      ch.sweep_acc, ch.counters, ch.opts.seed, ch.opts.chain_offset,
                                                      move);
        if ((e = cudaGetLastError()) != cudaSuccess) { fail_cuda(e, "block_decide"); break; }
        if ((rc = ggf_flush(ctx, st)) != GGF_OK) break;
        ctx->launches += 4;
        if (obs) {
            double* dst = mem == GGF_MEM_HOST ? dobs : obs + (size_t)mv * n * GGF_N_OBS;
            if ((rc = ggf_observe(ctx, dst, st)) != GGF_OK) break;
            if (mem == GGF_MEM_HOST &&
                (e = cudaMemcpyAsync(obs + (size_t)mv * n * GGF_N_OBS, dobs, (size_t)n * GGF_N_OBS * sizeof(double),
                                     cudaMemcpyDeviceToHost, st)) != cudaSuccess) { fail_cuda(e, "obs copy"); break; }
        }
        ch.block_moves += 1;
    }
    if (rc == GGF_OK && (e = cudaStreamSynchronize(st)) != cudaSuccess) fail_cuda(e, "sample_blocks sync");
    if (rc == GGF_OK && (rc = ggf_net_check(net)) != GGF_OK) ctx->err = ggf_net_last_error(net);
    if (rc == GGF_OK && ctx->prof) {   // timing of the tentative link steps and flushes
        for (size_t k = 0; k + 2 < ctx->ev_cat.size(); k += 3) {
            float ms = 0;
            if (cudaEventElapsedTime(&ms, ctx->ev[ctx->ev_cat[k + 1]], ctx->ev[ctx->ev_cat[k + 2]]) == cudaSuccess) {
                ctx->kt_ms[ctx->ev_cat[k]] += ms;
                ctx->kt_n[ctx->ev_cat[k]] += 1;
            }
        }
    }
    ctx->ev_cat.clear();
    ctx->ev_used = 0;
    void* ps[] = {blocks, link_k, dead, lq, prop, old_links, ell_save, dobs};
    for (void* q : ps) if (q) cudaFree(q);
    return rc;
}
