// C ABI entry points of libggf (see include/ggf.h for the contract).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>
#include "ggf_ctx.h"

size_t ggf_factor_tmp_bytes(int n, int batch);
size_t ggf_refine_bytes(int N, bool cplx);
ggf_status ggf_refine_inverse(ggf_ctx* ctx, bool cplx, const void* d_links, int cfg, int pair, float* W, void* ws,
                              int terms, double* rmax, cudaStream_t st);
// Newton refinement policy for FP32 inverses (largest |I - M W| entry r):
// r <= kRefineFloor is the FP32 floor (no step); r <= kRefineOne takes one
// step with one TF32 product; r <= kRefineTol takes three-product steps.
// Steps repeat (at most three) while each halves r; the inverse is kept when
// r ends at most kRefineOne (a matrix whose FP32 floor lies above
// kRefineFloor stalls there), else the chain is refactored by Gauss-Jordan.
static const double kRefineFloor = 4e-6, kRefineOne = 1e-4, kRefineTol = 5e-2;
ggf_status ggf_link_step(ggf_ctx* ctx, int link, cudaStream_t st);
ggf_status ggf_observe(ggf_ctx* ctx, double* d_obs, cudaStream_t st);
ggf_status ggf_mark_refresh(ggf_ctx* ctx, cudaStream_t st);
ggf_status ggf_flush(ggf_ctx* ctx, cudaStream_t st);
ggf_status ggf_prepare_sampler(ggf_ctx* ctx);
ggf_status ggf_prepare_flush_tc(ggf_ctx* ctx);
ggf_status ggf_prepare_batch(ggf_ctx* ctx);
ggf_status ggf_check_batch(ggf_ctx* ctx, int kmax, bool fp64);
size_t ggf_flush_ps_chain_bytes(ggf_ctx* ctx, int KRM);
size_t ggf_flush_ps_newton_bytes(ggf_ctx* ctx);
ggf_status ggf_batch(ggf_ctx* ctx, int l0, int kb, cudaStream_t st);
ggf_status ggf_bump_sweep(ggf_ctx* ctx, cudaStream_t st);
ggf_status ggf_electric(ggf_ctx* ctx, cxd* d_out, cxd* d_pairs, cudaStream_t st, bool field = false);
ggf_status ggf_fermion(ggf_ctx* ctx, cxd* d_site, cxd* d_link, cxd* d_pair_site, cxd* d_pair_link,
                       cudaStream_t st);
ggf_status ggf_pair_norm(ggf_ctx* ctx, cxd* d_out, cudaStream_t st);
ggf_status ggf_score(ggf_ctx* ctx, double* d_out, cudaStream_t st);
ggf_status ggf_fermion4(ggf_ctx* ctx, cxd* d_out, cudaStream_t st, cxd* d_pairs = nullptr);
ggf_status ggf_link_score(ggf_ctx* ctx, cxd* d_out, cudaStream_t st);
ggf_status ggf_link_terms(ggf_ctx* ctx, const int* d_q, cxd* d_blk, cxd* d_pair_blk, cxd* d_out, cxd* d_pair_out,
                          cudaStream_t st);

ggf_status ggf_fail(ggf_ctx* ctx, ggf_status st, const std::string& msg) {
    if (ctx) ctx->err = msg;
    return st;
}

ggf_status ggf_cuda(ggf_ctx* ctx, cudaError_t e, const char* what) {
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) return ggf_fail(ctx, GGF_ENOMEM, m);
    return ggf_fail(ctx, GGF_ECUDA, m);
}

ggf_status ggf_workspace(ggf_ctx* ctx, size_t bytes) {
    if (bytes <= ctx->work_bytes) return GGF_OK;
    if (ctx->work) cudaFree(ctx->work);
    ctx->work = nullptr;
    ctx->work_bytes = 0;
    GGF_CK(cudaMalloc(&ctx->work, bytes));
    ctx->work_bytes = bytes;
    return GGF_OK;
}

void ggf_free_chains(ggf_ctx* ctx) {
    Chains& c = ctx->ch;
    if (c.gexec) cudaGraphExecDestroy(c.gexec);
    if (c.graph) cudaGraphDestroy(c.graph);
    if (c.gexec_t) cudaGraphExecDestroy(c.gexec_t);
    if (c.graph_t) cudaGraphDestroy(c.graph_t);
    if (c.cs) cudaStreamDestroy(c.cs);
    if (c.join) cudaEventDestroy(c.join);
    if (c.d_sweep) cudaFree(c.d_sweep);
    if (c.d_obs_stage) cudaFree(c.d_obs_stage);
    void* ptrs[] = {c.links, c.Wr, c.Wc, c.ell, c.zbuf, c.ybuf, c.accept, c.since_refresh,
                    c.sweep_acc, c.counters, c.drift, c.refresh_list, c.Pr, c.Pc, c.pend, c.Sm, c.flags, c.ps};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    ggf_chain_opts o = c.opts;
    c = Chains();
    c.opts = o;
}

void ggf_free_consts(ggf_ctx* ctx) {
    void* ptrs[] = {ctx->d_D, ctx->d_Gr, ctx->d_Gc, ctx->d_logc, ctx->d_w, ctx->d_Ap, ctx->d_Bp};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    ctx->d_D = nullptr; ctx->d_Ap = nullptr; ctx->d_Bp = nullptr; ctx->d_Gr = nullptr; ctx->d_Gc = nullptr; ctx->d_logc = nullptr; ctx->d_w = nullptr;
    ctx->have_gauss = false;
}

namespace {

// Z2: int8 g; U(1): double theta; SU(2): four doubles (unit quaternion)
size_t link_bytes(const Geometry& g) {
    return g.group == GGF_Z2 ? 1 : g.group == GGF_SU2 ? 4 * sizeof(double) : sizeof(double);
}

// scoped device buffer
struct DBuf {
    void* p = nullptr;
    ~DBuf() { if (p) cudaFree(p); }
};

ggf_status dalloc(ggf_ctx* ctx, DBuf& b, size_t bytes) {
    GGF_CK(cudaMalloc(&b.p, std::max<size_t>(bytes, 16)));
    return GGF_OK;
}

size_t budget_bytes() {
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    size_t cap = (size_t)8 << 30;
    return std::max<size_t>(std::min(cap, fr / 2), (size_t)64 << 20);
}

// logpf/phase of dense refactorisations back to their item positions
__global__ void scatter_pf_kernel(int n, const int* idx, const cxd* lp, const cxd* ph, cxd* logpf, cxd* phase) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    logpf[idx[i]] = lp[i];
    phase[idx[i]] = ph[i];
}

// ell[cfg][pair_off + pair] of items with explicit (cfg, pair)
__global__ void write_items_kernel(int n_items, const int* cfg, const int* pair, int pair_off, int P, bool cplx,
                                   const cxd* logpf, const cxd* phase, cxd* ell) {
    int it = blockIdx.x * blockDim.x + threadIdx.x;
    if (it >= n_items) return;
    cxd v = {logpf[it].x, 0.0};
    if (cplx) v.y = atan2(phase[it].y, phase[it].x);
    ell[(size_t)cfg[it] * P + pair_off + pair[it]] = v;
}

// W[chain][p] <- convert(A[item]) and log-weight bookkeeping after a factorisation
template <class TD>
__global__ void scatter_kernel(int N, int fam_pairs, const int* item_chain, const int* item_pair, const void* A,
                               bool cplx, TD* W) {
    int it = blockIdx.y;
    size_t NN = (size_t)N * N;
    size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= NN) return;
    int c = item_chain[it], p = item_pair[it];
    cxd v = cplx ? ((const cxd*)A)[(size_t)it * NN + e] : cxd{((const double*)A)[(size_t)it * NN + e], 0.0};
    W[((size_t)c * fam_pairs + p) * NN + e] = Sc<TD>::from(v);
}

// log Pf(M_nm(G)) of explicit (configuration, pair-within-family) items
// (host lists hc, hp) into d_logpf / d_phase, by the site-by-site FP64
// elimination; items whose closed sets had no usable pivot are refactored by
// the dense FP64 Parlett-Reid Pfaffian.  d_cfg, d_pair, d_flag hold
// hc.size() entries (overwritten).
ggf_status pf_items(ggf_ctx* ctx, bool cplx, const std::vector<int>& hc, const std::vector<int>& hp,
                    const void* d_links, int* d_cfg, int* d_pair, int* d_flag, cxd* d_logpf, cxd* d_phase,
                    cudaStream_t st) {
    const int items = (int)hc.size();
    if (items == 0) return GGF_OK;
    const int N = ctx->g.N;
    const size_t NN = (size_t)N * N;
    GGF_CK(cudaMemcpyAsync(d_cfg, hc.data(), items * sizeof(int), cudaMemcpyHostToDevice, st));
    GGF_CK(cudaMemcpyAsync(d_pair, hp.data(), items * sizeof(int), cudaMemcpyHostToDevice, st));
    GGF_TRY(ggf_front_pfaffian(ctx, cplx, items, d_cfg, d_pair, d_links, d_logpf, d_phase, d_flag, st));
    std::vector<int> hf(items);
    GGF_CK(cudaMemcpyAsync(hf.data(), d_flag, items * sizeof(int), cudaMemcpyDeviceToHost, st));
    GGF_CK(cudaStreamSynchronize(st));
    std::vector<int> fi, fc, fp;
    for (int i = 0; i < items; ++i)
        if (hf[i]) { fi.push_back(i); fc.push_back(hc[i]); fp.push_back(hp[i]); }
    ctx->dense_pfaffians += fi.size();
    if (fi.empty()) return GGF_OK;
    const size_t elem = cplx ? sizeof(cxd) : sizeof(double);
    const int nf = (int)fi.size();
    const int per = (int)std::max<size_t>(1, std::min<size_t>(nf, budget_bytes() / (NN * elem)));
    const size_t tmp = ggf_factor_tmp_bytes(N, per);
    GGF_TRY(ggf_workspace(ctx, NN * elem * per + tmp + (size_t)per * (3 * sizeof(int) + 2 * sizeof(cxd)) + 1024));
    unsigned char* q = (unsigned char*)ctx->work;
    void* A = q;
    q += (NN * elem * per + 255) / 256 * 256;
    void* ftmp = q;
    q += (tmp + 255) / 256 * 256;
    cxd* f_logpf = (cxd*)q; q += (size_t)per * sizeof(cxd);
    cxd* f_phase = (cxd*)q; q += (size_t)per * sizeof(cxd);
    int* f_cfg = (int*)q; q += (size_t)per * sizeof(int);
    int* f_pair = (int*)q; q += (size_t)per * sizeof(int);
    int* f_idx = (int*)q;
    for (int f0 = 0; f0 < nf; f0 += per) {
        const int nb = std::min(per, nf - f0);
        GGF_CK(cudaMemcpyAsync(f_cfg, fc.data() + f0, nb * sizeof(int), cudaMemcpyHostToDevice, st));
        GGF_CK(cudaMemcpyAsync(f_pair, fp.data() + f0, nb * sizeof(int), cudaMemcpyHostToDevice, st));
        GGF_CK(cudaMemcpyAsync(f_idx, fi.data() + f0, nb * sizeof(int), cudaMemcpyHostToDevice, st));
        GGF_TRY(ggf_assemble(ctx, !cplx, nb, f_cfg, f_pair, d_links, A, st));
        GGF_TRY(ggf_pfaffian_batched(ctx, cplx, N, nb, A, f_logpf, f_phase, ftmp, st));
        scatter_pf_kernel<<<(nb + 127) / 128, 128, 0, st>>>(nb, f_idx, f_logpf, f_phase, d_logpf, d_phase);
        GGF_CK(cudaGetLastError());
        GGF_CK(cudaStreamSynchronize(st));
    }
    return GGF_OK;
}

// log Pf of every (configuration, pair) item of one family into ell[cfg][P].
ggf_status front_family(ggf_ctx* ctx, bool cplx, int n_cfg, int npf, const void* d_links, cxd* ell, cudaStream_t st) {
    const int P = ctx->P;
    const long long total = (long long)n_cfg * npf;
    const int chunk = (int)std::min<long long>(total, 1 << 20);
    DBuf tab;
    GGF_TRY(dalloc(ctx, tab, (size_t)chunk * (2 * sizeof(cxd) + 3 * sizeof(int)) + 256));
    cxd* d_logpf = (cxd*)tab.p;
    cxd* d_phase = d_logpf + chunk;
    int* d_cfg = (int*)(d_phase + chunk);
    int* d_pair = d_cfg + chunk;
    int* d_flag = d_pair + chunk;
    std::vector<int> hc, hp;
    for (long long i0 = 0; i0 < total; i0 += chunk) {
        const int items = (int)std::min<long long>(chunk, total - i0);
        hc.resize(items); hp.resize(items);
        for (int i = 0; i < items; ++i) { hc[i] = (int)((i0 + i) / npf); hp[i] = (int)((i0 + i) % npf); }
        GGF_TRY(pf_items(ctx, cplx, hc, hp, d_links, d_cfg, d_pair, d_flag, d_logpf, d_phase, st));
        GGF_CK(cudaMemcpyAsync(d_cfg, hc.data(), items * sizeof(int), cudaMemcpyHostToDevice, st));
        GGF_CK(cudaMemcpyAsync(d_pair, hp.data(), items * sizeof(int), cudaMemcpyHostToDevice, st));
        write_items_kernel<<<(items + 127) / 128, 128, 0, st>>>(items, d_cfg, d_pair, cplx ? ctx->K : 0, P, cplx,
                                                                 d_logpf, d_phase, ell);
        GGF_CK(cudaGetLastError());
        GGF_CK(cudaStreamSynchronize(st));
    }
    return GGF_OK;
}

// Log-weights of (chain, pair) items from a fresh factorisation: init sets
// them; a refresh records |l_tracked - l_fresh| (log magnitude plus phase
// mod 2 pi) as drift and replaces them.  Resets the accept count since the
// last refresh.
__global__ void ell_set_kernel(int n_items, int pair_off, int P, bool cplx, bool init, const int* item_chain,
                               const int* item_pair, const cxd* logpf, const cxd* phase, cxd* ell, double* drift,
                               int* since, unsigned long long* counters, int* flags) {
    int it = blockIdx.x * blockDim.x + threadIdx.x;
    if (it >= n_items) return;
    int c = item_chain[it], p = pair_off + item_pair[it];
    cxd& el = ell[(size_t)c * P + p];
    cxd v = {logpf[it].x, 0.0};
    if (cplx) v.y = atan2(phase[it].y, phase[it].x);
    if (!isfinite(v.x)) {
        atomicAdd(&counters[3], 1ULL);
        atomicOr(&flags[c], 1);
    }
    if (!init) {
        double d = fabs(v.x - el.x);
        if (cplx) d += fabs(remainder(v.y - el.y, 2 * M_PI));
        if (!(d <= drift[c])) drift[c] = d;
    }
    el = v;
    since[c] = 0;
}

__global__ void count_singular_kernel(int n_items, const int* item_chain, const cxd* logdet,
                                      unsigned long long* counters, int* flags) {
    int it = blockIdx.x * blockDim.x + threadIdx.x;
    if (it < n_items && !isfinite(logdet[it].x)) {
        atomicAdd(&counters[3], 1ULL);
        atomicOr(&flags[item_chain[it]], 1);
    }
}

// Per-chain status: singular factorisation or non-finite tracked log-weight
// -> GGF_ESINGULAR; drift above tol (tol > 0) -> GGF_EDRIFT; else GGF_OK.
__global__ void status_kernel(int n, int P, const cxd* ell, const double* drift, const int* flags, double tol,
                              int32_t* status) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    bool bad = (flags[c] & 1) != 0;
    for (int p = 0; p < P; ++p) {
        const cxd e = ell[(size_t)c * P + p];
        bad |= !isfinite(e.x) || !isfinite(e.y);
    }
    status[c] = bad ? GGF_ESINGULAR : (tol > 0.0 && !(drift[c] <= tol)) ? GGF_EDRIFT : GGF_OK;
}

// FP64 Gauss-Jordan inverses of the listed chains' M_nm(G), converted into
// the chains' W storage.
ggf_status dense_inverse(ggf_ctx* ctx, const std::vector<int>& chains, cudaStream_t st) {
    if (chains.empty()) return GGF_OK;
    Chains& ch = ctx->ch;
    const int N = ctx->g.N;
    const size_t NN = (size_t)N * N;
    const bool fp64 = ch.opts.precision == GGF_FP64;
    for (int fam = 0; fam < 2; ++fam) {
        const bool cplx = fam == 1;
        const int npf = cplx ? ctx->Kc : ctx->K;
        if (npf == 0) continue;
        const size_t elem = cplx ? sizeof(cxd) : sizeof(double);
        const size_t per_item = NN * elem;
        int chunk_chains = (int)std::max<size_t>(1, budget_bytes() / (per_item * npf));
        chunk_chains = std::min<int>(chunk_chains, (int)chains.size());
        const int max_items = chunk_chains * npf;
        const size_t tmp = ggf_factor_tmp_bytes(N, max_items);
        const size_t small = (size_t)max_items * (2 * sizeof(int) + sizeof(cxd)) + 256;
        GGF_TRY(ggf_workspace(ctx, per_item * max_items + tmp + small + 1024));
        unsigned char* base = (unsigned char*)ctx->work;
        void* A = base;
        unsigned char* q = base + per_item * max_items;
        void* ftmp = q;
        q += (tmp + 255) / 256 * 256;
        int* d_chain = (int*)q; q += (size_t)max_items * sizeof(int);
        int* d_pair = (int*)q; q += (size_t)max_items * sizeof(int);
        q = (unsigned char*)(((uintptr_t)q + 15) / 16 * 16);
        cxd* d_logdet = (cxd*)q;
        std::vector<int> hc, hp;
        for (size_t c0 = 0; c0 < chains.size(); c0 += chunk_chains) {
            int nc = (int)std::min<size_t>(chunk_chains, chains.size() - c0);
            int items = nc * npf;
            hc.resize(items); hp.resize(items);
            for (int i = 0; i < nc; ++i)
                for (int p = 0; p < npf; ++p) { hc[i * npf + p] = chains[c0 + i]; hp[i * npf + p] = p; }
            GGF_CK(cudaMemcpyAsync(d_chain, hc.data(), items * sizeof(int), cudaMemcpyHostToDevice, st));
            GGF_CK(cudaMemcpyAsync(d_pair, hp.data(), items * sizeof(int), cudaMemcpyHostToDevice, st));
            GGF_TRY(ggf_assemble(ctx, !cplx, items, d_chain, d_pair, ch.links, A, st));
            GGF_TRY(ggf_invert_batched(ctx, cplx, N, items, A, d_logdet, ftmp, st));
            dim3 grid((unsigned)((NN + 255) / 256), items);
            if (!cplx) {
                if (fp64) scatter_kernel<double><<<grid, 256, 0, st>>>(N, npf, d_chain, d_pair, A, false, (double*)ch.Wr);
                else scatter_kernel<float><<<grid, 256, 0, st>>>(N, npf, d_chain, d_pair, A, false, (float*)ch.Wr);
            } else {
                if (fp64) scatter_kernel<cxd><<<grid, 256, 0, st>>>(N, npf, d_chain, d_pair, A, true, (cxd*)ch.Wc);
                else scatter_kernel<cxf><<<grid, 256, 0, st>>>(N, npf, d_chain, d_pair, A, true, (cxf*)ch.Wc);
            }
            count_singular_kernel<<<(items + 127) / 128, 128, 0, st>>>(items, d_chain, d_logdet, ch.counters,
                                                                       ch.flags);
            ctx->launches += 2;
            GGF_CK(cudaGetLastError());
            GGF_CK(cudaStreamSynchronize(st));  // hc/hp are reused by the next chunk
        }
    }
    return GGF_OK;
}

// Newton refinement of one FP32 inverse by the policy above; false when the
// residual is too large (or does not shrink) and the chain needs refactoring.
ggf_status refine_one(ggf_ctx* ctx, bool cplx, int c, int p, float* W, bool* ok, cudaStream_t st) {
    double r = 0.0;
    GGF_TRY(ggf_refine_inverse(ctx, cplx, ctx->ch.links, c, p, W, ctx->work, 0, &r, st));
    ctx->refine_rmax = std::max(ctx->refine_rmax, r);
    for (int step = 0; step < 3; ++step) {
        if (r <= kRefineFloor) { *ok = true; return GGF_OK; }
        if (!(r <= kRefineTol)) break;
        double unused = 0.0, after = 0.0;
        GGF_TRY(ggf_refine_inverse(ctx, cplx, ctx->ch.links, c, p, W, ctx->work, r <= kRefineOne ? 1 : 3, &unused, st));
        GGF_TRY(ggf_refine_inverse(ctx, cplx, ctx->ch.links, c, p, W, ctx->work, 0, &after, st));
        ctx->refine_steps += 1;
        // a step that no longer shrinks the residual has met this matrix's
        // FP32 floor (the rounded exact inverse has the same residual)
        if (!(after < 0.5 * r)) { r = std::min(r, after); *ok = r <= kRefineOne; return GGF_OK; }
        r = after;
    }
    *ok = r <= kRefineOne;
    return GGF_OK;
}

// Newton refinement of the listed FP32 chains' inverses (k_refine.cu); the
// chains whose residual is too large for it are returned in `dense`.
ggf_status newton_inverse(ggf_ctx* ctx, const std::vector<int>& chains, std::vector<int>& dense, cudaStream_t st) {
    Chains& ch = ctx->ch;
    const int N = ctx->g.N;
    const size_t NN = (size_t)N * N;
    GGF_TRY(ggf_workspace(ctx, ggf_refine_bytes(N, ctx->Kc > 0)));
    for (int c : chains) {
        bool ok = true;
        for (int fam = 0; fam < 2 && ok; ++fam) {
            const bool cplx = fam == 1;
            const int npf = cplx ? ctx->Kc : ctx->K;
            for (int p = 0; p < npf && ok; ++p) {
                float* W = cplx ? (float*)ch.Wc + ((size_t)c * ctx->Kc + p) * NN * 2
                                : (float*)ch.Wr + ((size_t)c * ctx->K + p) * NN;
                GGF_TRY(refine_one(ctx, cplx, c, p, W, &ok, st));
            }
        }
        if (!ok) dense.push_back(c);
    }
    GGF_CK(cudaStreamSynchronize(st));
    return GGF_OK;
}

// Log-weights of the listed chains from the site-by-site FP64 Pfaffian
// (dense fallback for items without a usable pivot).
ggf_status chain_ell(ggf_ctx* ctx, const std::vector<int>& chains, bool init, cudaStream_t st) {
    Chains& ch = ctx->ch;
    for (int fam = 0; fam < 2; ++fam) {
        const bool cplx = fam == 1;
        const int npf = cplx ? ctx->Kc : ctx->K;
        if (npf == 0) continue;
        const int items = (int)chains.size() * npf;
        std::vector<int> hc(items), hp(items);
        for (size_t i = 0; i < chains.size(); ++i)
            for (int p = 0; p < npf; ++p) { hc[i * npf + p] = chains[i]; hp[i * npf + p] = p; }
        DBuf tab;
        GGF_TRY(dalloc(ctx, tab, (size_t)items * (2 * sizeof(cxd) + 3 * sizeof(int)) + 256));
        cxd* d_logpf = (cxd*)tab.p;
        cxd* d_phase = d_logpf + items;
        int* d_chain = (int*)(d_phase + items);
        int* d_pair = d_chain + items;
        int* d_flag = d_pair + items;
        GGF_TRY(pf_items(ctx, cplx, hc, hp, ch.links, d_chain, d_pair, d_flag, d_logpf, d_phase, st));
        GGF_CK(cudaMemcpyAsync(d_chain, hc.data(), items * sizeof(int), cudaMemcpyHostToDevice, st));
        GGF_CK(cudaMemcpyAsync(d_pair, hp.data(), items * sizeof(int), cudaMemcpyHostToDevice, st));
        ell_set_kernel<<<(items + 127) / 128, 128, 0, st>>>(items, cplx ? ctx->K : 0, ctx->P, cplx, init, d_chain,
                                                            d_pair, d_logpf, d_phase, ch.ell, ch.drift,
                                                            ch.since_refresh, ch.counters, ch.flags);
        GGF_CK(cudaGetLastError());
        GGF_CK(cudaStreamSynchronize(st));
    }
    return GGF_OK;
}

// Factor the listed chains: log-weights from the site-by-site FP64 Pfaffian
// (init: set; refresh: drift recorded), inverses by FP64 Gauss-Jordan at the
// start and for FP64 chains, by a Newton step on the tensor cores for FP32
// chains (Gauss-Jordan where the residual is too large for it).
ggf_status factor_chains(ggf_ctx* ctx, const std::vector<int>& chains, bool init, cudaStream_t st) {
    if (chains.empty()) return GGF_OK;
    GGF_TRY(chain_ell(ctx, chains, init, st));
    const bool newton = !init && ctx->ch.opts.precision == GGF_FP32 && ctx->use_tc && ctx->g.N % 8 == 0;
    if (!newton) return dense_inverse(ctx, chains, st);
    std::vector<int> dense;
    GGF_TRY(newton_inverse(ctx, chains, dense, st));
    ctx->dense_refreshes += dense.size();
    return dense_inverse(ctx, dense, st);
}

ggf_status require(ggf_ctx* ctx, bool gauss, bool chains) {
    if (!ctx) return GGF_EINVAL;
    if (!ctx->have_lattice || !ctx->have_group) return ggf_fail(ctx, GGF_ESTATE, "lattice/group not initialised");
    if (gauss && !ctx->have_gauss) return ggf_fail(ctx, GGF_ESTATE, "Gaussians not initialised");
    if (chains && ctx->ch.n == 0) return ggf_fail(ctx, GGF_ESTATE, "chains not initialised");
    return GGF_OK;
}

}  // namespace

extern "C" {

ggf_status ggf_create(ggf_ctx** out, int device) {
    if (!out) return GGF_EINVAL;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || n == 0) return GGF_ECUDA;
    if (device < 0 || device >= n) return GGF_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) return GGF_ECUDA;
    ggf_ctx* c = new ggf_ctx();
    c->device = device;
    cudaDeviceGetAttribute(&c->n_sms, cudaDevAttrMultiProcessorCount, device);
    if (cudaMalloc(&c->d_err, sizeof(int)) != cudaSuccess || cudaMemset(c->d_err, 0, sizeof(int)) != cudaSuccess) {
        delete c;
        return GGF_ENOMEM;
    }
    c->ch.opts.precision = GGF_FP64;
    c->ch.opts.refresh_every = 64;
    c->ch.opts.width = 0.5;
    c->ch.opts.seed = 20241202ULL;
    *out = c;
    return GGF_OK;
}

void ggf_destroy(ggf_ctx* ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    ggf_free_chains(ctx);
    ggf_free_consts(ctx);
    ggf_front_free(ctx);
    if (ctx->work) cudaFree(ctx->work);
    if (ctx->d_err) cudaFree(ctx->d_err);
    for (cudaEvent_t e : ctx->ev) cudaEventDestroy(e);
    delete ctx;
}

const char* ggf_last_error(const ggf_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

ggf_status ggf_init_lattice(ggf_ctx* ctx, int L) {
    if (!ctx) return GGF_EINVAL;
    if (L < 1 || L > 64) return ggf_fail(ctx, GGF_EINVAL, "L must be in [1, 64]");
    cudaSetDevice(ctx->device);
    ggf_free_chains(ctx);
    ggf_free_consts(ctx);
    ctx->g = Geometry();
    ctx->g.L = L;
    ctx->g.V = L * L;
    ctx->g.n_links = 2 * L * L;
    ctx->have_lattice = true;
    ctx->have_group = false;
    return GGF_OK;
}

ggf_status ggf_init_group(ggf_ctx* ctx, int group, int n_v, const int* q_src) {
    if (!ctx) return GGF_EINVAL;
    if (!ctx->have_lattice) return ggf_fail(ctx, GGF_ESTATE, "call ggf_init_lattice first");
    if (group != GGF_Z2 && group != GGF_U1 && group != GGF_SU2)
        return ggf_fail(ctx, GGF_EINVAL, "group must be GGF_Z2, GGF_U1 or GGF_SU2");
    if (group == GGF_SU2 && n_v != 2) return ggf_fail(ctx, GGF_EINVAL, "SU(2) needs n_v = 2 (one doublet per link end)");
    if (n_v < 1 || n_v > 2) return ggf_fail(ctx, GGF_EINVAL, "n_v must be 1 or 2");
    if (group == GGF_U1 && !q_src) return ggf_fail(ctx, GGF_EINVAL, "U(1) needs q_src");
    cudaSetDevice(ctx->device);
    ggf_free_chains(ctx);
    ggf_free_consts(ctx);
    Geometry& g = ctx->g;
    g.group = group;
    g.n_v = n_v;
    g.B = 8 * n_v;
    g.h2 = 2 * n_v;
    g.r = 4 * n_v;
    g.N = g.B * g.V;
    for (int j = 0; j < 2; ++j) g.q[j] = (group == GGF_U1 && j < n_v) ? q_src[j] : 1;
    ctx->have_group = true;
    return GGF_OK;
}

ggf_status ggf_init_gaussians(ggf_ctx* ctx, const double* gamma_site, int K, const double* gamma_bond,
                              const double* lambda) {
    if (!ctx) return GGF_EINVAL;
    if (!ctx->have_group) return ggf_fail(ctx, GGF_ESTATE, "call ggf_init_group first");
    if (K < 1 || K > 8) return ggf_fail(ctx, GGF_EINVAL, "K must be in [1, 8]");
    if (!gamma_site || !gamma_bond || !lambda) return ggf_fail(ctx, GGF_EINVAL, "null input");
    cudaSetDevice(ctx->device);
    ggf_free_chains(ctx);
    return ggf_build_constants(ctx, gamma_site, K, gamma_bond, lambda);
}

ggf_status ggf_get_constants(const ggf_ctx* cctx, int* n_pairs, double* log_c, int* pairs) {
    if (!cctx || !cctx->have_gauss) return GGF_ESTATE;
    if (n_pairs) *n_pairs = cctx->P;
    for (int p = 0; p < cctx->P; ++p) {
        if (log_c) { log_c[2 * p] = cctx->logc[p].x; log_c[2 * p + 1] = cctx->logc[p].y; }
        if (pairs) { pairs[2 * p] = cctx->pair_n[p]; pairs[2 * p + 1] = cctx->pair_m[p]; }
    }
    return GGF_OK;
}

ggf_status ggf_logweight(ggf_ctx* ctx, int n_cfg, const void* links, double* logN, double* ell, int mem,
                         void* stream) {
    NvtxRange range("ggf_logweight");
    GGF_TRY(require(ctx, true, false));
    if (n_cfg < 0 || !links || !logN) return ggf_fail(ctx, GGF_EINVAL, "bad logweight arguments");
    if (n_cfg == 0) return GGF_OK;
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const Geometry& g = ctx->g;
    const int N = g.N, P = ctx->P;
    const size_t NN = (size_t)N * N;
    const size_t lbytes = (size_t)n_cfg * g.n_links * link_bytes(g);
    DBuf dl, dell, dlog;
    const void* d_links = links;
    if (mem == GGF_MEM_HOST) {
        GGF_TRY(dalloc(ctx, dl, lbytes));
        GGF_CK(cudaMemcpyAsync(dl.p, links, lbytes, cudaMemcpyHostToDevice, st));
        d_links = dl.p;
    }
    GGF_TRY(dalloc(ctx, dell, (size_t)n_cfg * P * sizeof(cxd)));
    for (int fam = 0; fam < 2; ++fam) {
        const bool cplx = fam == 1;
        const int npf = cplx ? ctx->Kc : ctx->K;
        if (npf == 0) continue;
        GGF_TRY(front_family(ctx, cplx, n_cfg, npf, d_links, (cxd*)dell.p, st));
    }
    double* d_logN = logN;
    if (mem == GGF_MEM_HOST) {
        GGF_TRY(dalloc(ctx, dlog, (size_t)n_cfg * sizeof(double)));
        d_logN = (double*)dlog.p;
    }
    GGF_TRY(ggf_combine(ctx, n_cfg, (const cxd*)dell.p, d_logN, st));
    if (mem == GGF_MEM_HOST) {
        GGF_CK(cudaMemcpyAsync(logN, d_logN, n_cfg * sizeof(double), cudaMemcpyDeviceToHost, st));
        if (ell) GGF_CK(cudaMemcpyAsync(ell, dell.p, (size_t)n_cfg * P * sizeof(cxd), cudaMemcpyDeviceToHost, st));
        GGF_CK(cudaStreamSynchronize(st));
    } else {
        if (ell) GGF_CK(cudaMemcpyAsync(ell, dell.p, (size_t)n_cfg * P * sizeof(cxd), cudaMemcpyDeviceToDevice, st));
        GGF_CK(cudaStreamSynchronize(st));  // scoped temporaries are freed on return
    }
    return GGF_OK;
}

ggf_status ggf_observable(ggf_ctx* ctx, int which, int n_cfg, const void* links, double* out, int mem,
                          void* stream) {
    GGF_TRY(require(ctx, false, false));
    if (which != GGF_OBS_PLAQUETTE) return ggf_fail(ctx, GGF_EINVAL, "unknown observable");
    if (n_cfg < 0 || !links || !out) return ggf_fail(ctx, GGF_EINVAL, "bad observable arguments");
    if (n_cfg == 0) return GGF_OK;
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const Geometry& g = ctx->g;
    if (mem == GGF_MEM_HOST) {
        DBuf dl, dout;
        size_t lb = (size_t)n_cfg * g.n_links * link_bytes(g);
        GGF_TRY(dalloc(ctx, dl, lb));
        GGF_TRY(dalloc(ctx, dout, n_cfg * sizeof(double)));
        GGF_CK(cudaMemcpyAsync(dl.p, links, lb, cudaMemcpyHostToDevice, st));
        GGF_TRY(ggf_plaquette(ctx, n_cfg, dl.p, (double*)dout.p, st));
        GGF_CK(cudaMemcpyAsync(out, dout.p, n_cfg * sizeof(double), cudaMemcpyDeviceToHost, st));
        GGF_CK(cudaStreamSynchronize(st));
        return GGF_OK;
    }
    return ggf_plaquette(ctx, n_cfg, links, out, st);
}

static ggf_status loops_entry(ggf_ctx* ctx, int R, int T, int mode, int n_cfg, const void* links, double* out, int mem,
                       void* stream) {
    GGF_TRY(require(ctx, false, false));
    if (n_cfg < 0 || !links || !out) return ggf_fail(ctx, GGF_EINVAL, "bad loop arguments");
    const Geometry& g = ctx->g;
    if (!mode && (R < 1 || T < 1 || R > g.L || T > g.L)) return ggf_fail(ctx, GGF_EINVAL, "need 1 <= R, T <= L");
    if (n_cfg == 0) return GGF_OK;
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (mem == GGF_MEM_HOST) {
        DBuf dl, dout;
        const size_t lb = (size_t)n_cfg * g.n_links * link_bytes(g);
        GGF_TRY(dalloc(ctx, dl, lb));
        GGF_TRY(dalloc(ctx, dout, n_cfg * sizeof(double)));
        GGF_CK(cudaMemcpyAsync(dl.p, links, lb, cudaMemcpyHostToDevice, st));
        GGF_TRY(ggf_loops(ctx, n_cfg, R, T, mode, dl.p, (double*)dout.p, st));
        GGF_CK(cudaMemcpyAsync(out, dout.p, n_cfg * sizeof(double), cudaMemcpyDeviceToHost, st));
        GGF_CK(cudaStreamSynchronize(st));
        return GGF_OK;
    }
    return ggf_loops(ctx, n_cfg, R, T, mode, links, out, st);
}

ggf_status ggf_wilson_loop(ggf_ctx* ctx, int R, int T, int n_cfg, const void* links, double* out, int mem,
                           void* stream) {
    return loops_entry(ctx, R, T, 0, n_cfg, links, out, mem, stream);
}

ggf_status ggf_polyakov_loop(ggf_ctx* ctx, int n_cfg, const void* links, double* out, int mem, void* stream) {
    return loops_entry(ctx, 0, 0, 1, n_cfg, links, out, mem, stream);
}

ggf_status ggf_chains_init(ggf_ctx* ctx, int n_chains, const void* links, const ggf_chain_opts* opts, int mem,
                           void* stream) {
    NvtxRange range("ggf_chains_init");
    GGF_TRY(require(ctx, true, false));
    if (n_chains < 1 || !links || !opts) return ggf_fail(ctx, GGF_EINVAL, "bad chains_init arguments");
    if (opts->precision != GGF_FP64 && opts->precision != GGF_FP32)
        return ggf_fail(ctx, GGF_EINVAL, "precision must be GGF_FP64 or GGF_FP32");
    if (opts->refresh_every < 1) return ggf_fail(ctx, GGF_EINVAL, "refresh_every must be >= 1");
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    ggf_free_chains(ctx);
    ctx->refine_rmax = 0.0;
    ctx->dense_refreshes = ctx->dense_pfaffians = ctx->refine_steps = 0;
    Chains& ch = ctx->ch;
    ch.opts = *opts;
    ch.n = n_chains;
    ch.sweep = 0;
    ch.block_moves = 0;
    const Geometry& g = ctx->g;
    const bool fp64 = opts->precision == GGF_FP64;
    const size_t rsz = fp64 ? sizeof(double) : sizeof(float);
    const size_t NN = (size_t)g.N * g.N;
    const size_t lb = (size_t)n_chains * g.n_links * link_bytes(g);
    GGF_CK(cudaMalloc(&ch.links, lb));
    GGF_CK(cudaMalloc(&ch.Wr, std::max<size_t>(16, (size_t)n_chains * ctx->K * NN * rsz)));
    GGF_CK(cudaMalloc(&ch.Wc, std::max<size_t>(16, (size_t)n_chains * ctx->Kc * NN * 2 * rsz)));
    GGF_CK(cudaMalloc(&ch.ell, (size_t)n_chains * ctx->P * sizeof(cxd)));
    GGF_CK(cudaMalloc(&ch.zbuf, (size_t)n_chains * ctx->P * g.r * g.r * sizeof(cxd)));
    ch.kmax = opts->delay > 1 ? opts->delay : 1;
    if (ch.kmax > 64) return ggf_fail(ctx, GGF_EINVAL, "delay must be <= 64");
    ch.steps_since_flush = 0;
    if (ch.kmax > 1) {
        const size_t pr = (size_t)n_chains * panel_plane(g.N, ch.kmax * g.r) * rsz;   // one plane per chain
        GGF_CK(cudaMalloc(&ch.Pr, std::max<size_t>(16, pr * 2 * ctx->K)));
        GGF_CK(cudaMalloc(&ch.Pc, std::max<size_t>(16, pr * 4 * ctx->Kc)));
        GGF_CK(cudaMalloc(&ch.ybuf, 16));
        GGF_TRY(ggf_check_batch(ctx, ch.kmax, fp64));
        const size_t KRM = (size_t)ch.kmax * g.r;
        GGF_CK(cudaMalloc(&ch.Sm, (size_t)n_chains * 2 * KRM * KRM * rsz * (ctx->K + 2 * ctx->Kc) + 16));
    } else {
        GGF_CK(cudaMalloc(&ch.ybuf, (size_t)n_chains * (ctx->K + 2 * ctx->Kc) * 2 * g.r * g.N * rsz + 16));
    }
    GGF_CK(cudaMalloc(&ch.pend, n_chains * sizeof(int)));
    GGF_CK(cudaMemsetAsync(ch.pend, 0, n_chains * sizeof(int), st));
    GGF_CK(cudaMalloc(&ch.d_sweep, sizeof(unsigned long long)));
    GGF_CK(cudaMemsetAsync(ch.d_sweep, 0, sizeof(unsigned long long), st));
    GGF_CK(cudaMalloc(&ch.d_obs_stage, (size_t)n_chains * GGF_N_OBS * sizeof(double)));
    GGF_CK(cudaStreamCreateWithFlags(&ch.cs, cudaStreamNonBlocking));
    GGF_CK(cudaEventCreateWithFlags(&ch.join, cudaEventDisableTiming));
    GGF_TRY(ggf_prepare_sampler(ctx));
    GGF_TRY(ggf_prepare_batch(ctx));
    GGF_TRY(ggf_prepare_flush_tc(ctx));
    GGF_CK(cudaMalloc(&ch.accept, n_chains * sizeof(int)));
    GGF_CK(cudaMalloc(&ch.since_refresh, n_chains * sizeof(int)));
    GGF_CK(cudaMalloc(&ch.sweep_acc, n_chains * sizeof(int)));
    GGF_CK(cudaMalloc(&ch.counters, 6 * sizeof(unsigned long long)));
    GGF_CK(cudaMalloc(&ch.drift, n_chains * sizeof(double)));
    GGF_CK(cudaMalloc(&ch.flags, n_chains * sizeof(int)));
    GGF_CK(cudaMemsetAsync(ch.flags, 0, n_chains * sizeof(int), st));
    GGF_CK(cudaMalloc(&ch.refresh_list, (n_chains + 1) * sizeof(int)));
    GGF_CK(cudaMemsetAsync(ch.accept, 0, n_chains * sizeof(int), st));
    GGF_CK(cudaMemsetAsync(ch.since_refresh, 0, n_chains * sizeof(int), st));
    GGF_CK(cudaMemsetAsync(ch.sweep_acc, 0, n_chains * sizeof(int), st));
    GGF_CK(cudaMemsetAsync(ch.counters, 0, 6 * sizeof(unsigned long long), st));
    GGF_CK(cudaMemsetAsync(ch.drift, 0, n_chains * sizeof(double), st));
    // host copy of the starting links to find identical configurations
    std::vector<unsigned char> hl(lb);
    if (mem == GGF_MEM_HOST) std::memcpy(hl.data(), links, lb);
    else GGF_CK(cudaMemcpy(hl.data(), links, lb, cudaMemcpyDeviceToHost));
    GGF_CK(cudaMemcpyAsync(ch.links, hl.data(), lb, cudaMemcpyHostToDevice, st));
    const size_t row = g.n_links * link_bytes(g);
    std::map<std::string, int> first;
    std::vector<int> reps, rep_of(n_chains);
    for (int c = 0; c < n_chains; ++c) {
        std::string key((const char*)hl.data() + (size_t)c * row, row);
        auto it = first.find(key);
        if (it == first.end()) { first[key] = c; reps.push_back(c); rep_of[c] = c; }
        else rep_of[c] = it->second;
    }
    GGF_TRY(factor_chains(ctx, reps, true, st));
    for (int c = 0; c < n_chains; ++c) {
        int r0 = rep_of[c];
        if (r0 == c) continue;
        GGF_CK(cudaMemcpyAsync((unsigned char*)ch.Wr + (size_t)c * ctx->K * NN * rsz,
                               (unsigned char*)ch.Wr + (size_t)r0 * ctx->K * NN * rsz, ctx->K * NN * rsz,
                               cudaMemcpyDeviceToDevice, st));
        if (ctx->Kc)
            GGF_CK(cudaMemcpyAsync((unsigned char*)ch.Wc + (size_t)c * ctx->Kc * NN * 2 * rsz,
                                   (unsigned char*)ch.Wc + (size_t)r0 * ctx->Kc * NN * 2 * rsz,
                                   ctx->Kc * NN * 2 * rsz, cudaMemcpyDeviceToDevice, st));
        GGF_CK(cudaMemcpyAsync(ch.ell + (size_t)c * ctx->P, ch.ell + (size_t)r0 * ctx->P, ctx->P * sizeof(cxd),
                               cudaMemcpyDeviceToDevice, st));
    }
    // the set-up's dense factorisation workspace can be large (up to 8 GiB);
    // a refresh grows its own again when it needs one
    if (ctx->work_bytes > ((size_t)1 << 30)) {
        GGF_CK(cudaStreamSynchronize(st));
        cudaFree(ctx->work);
        ctx->work = nullptr;
        ctx->work_bytes = 0;
    }
    // pre-split scratch of the tensor-core flush, after the set-up's own
    // workspace: waves of up to 2 GiB and a quarter of the free memory; within
    // that budget at least what the refresh's Newton product (rank N, one
    // pair) needs, so that it runs through the scratch too
    if (!fp64 && ch.kmax > 1 && ctx->use_tc) {
        const size_t per = ggf_flush_ps_chain_bytes(ctx, ch.kmax * g.r);
        size_t free_b = 0, total_b = 0;
        GGF_CK(cudaMemGetInfo(&free_b, &total_b));
        const size_t budget = std::min<size_t>((size_t)2 << 30, free_b / 4);
        ch.ps_wave = (int)std::max<size_t>(1, std::min<size_t>((size_t)n_chains, budget / std::max<size_t>(per, 1)));
        ch.ps_bytes = (size_t)ch.ps_wave * per;
        const size_t newton = ggf_flush_ps_newton_bytes(ctx);
        if (newton > ch.ps_bytes && newton <= budget) ch.ps_bytes = newton;
        if (cudaMalloc(&ch.ps, ch.ps_bytes) != cudaSuccess) {
            // memory is full: the flush splits its operands per tile instead
            cudaGetLastError();
            ch.ps = nullptr;
            ch.ps_wave = 0;
            ch.ps_bytes = 0;
        }
    }
    GGF_CK(cudaMemsetAsync(ch.counters, 0, 6 * sizeof(unsigned long long), st));
    GGF_CK(cudaStreamSynchronize(st));
    ctx->launches = 0;
    return GGF_OK;
}

}  // extern "C"

namespace {

// One sweep of every chain: link steps, pending flush, observables, refresh
// marks, sweep counter.  The same sequence is either launched eagerly or
// captured once into a CUDA graph and replayed.
ggf_status sweep_body(ggf_ctx* ctx, cudaStream_t st) {
    Chains& ch = ctx->ch;
    GGF_CK(cudaMemsetAsync(ch.sweep_acc, 0, ch.n * sizeof(int), st));
    const int nl = ctx->g.n_links;
    if (ch.kmax > 1) {
        for (int l0 = 0; l0 < nl; l0 += ch.kmax) GGF_TRY(ggf_batch(ctx, l0, std::min(ch.kmax, nl - l0), st));
    } else {
        for (int l = 0; l < nl; ++l) GGF_TRY(ggf_link_step(ctx, l, st));
    }
    GGF_TRY(ggf_flush(ctx, st));
    GGF_TRY(ggf_observe(ctx, ch.d_obs_stage, st));
    GGF_TRY(ggf_mark_refresh(ctx, st));
    GGF_TRY(ggf_bump_sweep(ctx, st));
    return GGF_OK;
}

void drop_graph(Chains& ch) {
    if (ch.gexec) cudaGraphExecDestroy(ch.gexec);
    if (ch.graph) cudaGraphDestroy(ch.graph);
    if (ch.gexec_t) cudaGraphExecDestroy(ch.gexec_t);
    if (ch.graph_t) cudaGraphDestroy(ch.graph_t);
    ch.gexec = nullptr;
    ch.graph = nullptr;
    ch.gexec_t = nullptr;
    ch.graph_t = nullptr;
    ch.gev_cat.clear();
    ch.gev_n = 0;
}

// Capture one sweep into a CUDA graph: the plain graph, or (timed = true) the
// same sweep with timing-event record nodes around its launch groups.
ggf_status ensure_graph(ggf_ctx* ctx, bool timed = false) {
    Chains& ch = ctx->ch;
    if (timed ? ch.gexec_t : ch.gexec) return GGF_OK;
    const bool prof = ctx->prof;
    if (timed) {
        // events are created before the capture: a sweep marks at most a few
        // events per link batch, link step or flush
        const size_t want = (size_t)8 * ctx->g.n_links + 64;
        while (ctx->ev.size() < want) {
            cudaEvent_t ev;
            GGF_CK(cudaEventCreate(&ev));
            ctx->ev.push_back(ev);
        }
    }
    ctx->prof = timed;
    ctx->ev_used = 0;
    ctx->ev_cat.clear();
    const unsigned long long l0 = ctx->launches;
    ctx->capturing = true;
    cudaError_t eb = cudaStreamBeginCapture(ch.cs, cudaStreamCaptureModeThreadLocal);
    if (eb != cudaSuccess) {
        ctx->prof = prof;
        ctx->capturing = false;
        return ggf_cuda(ctx, eb, "cudaStreamBeginCapture");
    }
    ggf_status s = sweep_body(ctx, ch.cs);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(ch.cs, &g);
    ctx->capturing = false;
    ctx->prof = prof;
    if (s != GGF_OK) {
        if (g) cudaGraphDestroy(g);
        return s;
    }
    if (e != cudaSuccess) return ggf_cuda(ctx, e, "cudaStreamEndCapture");
    if (timed) {
        ch.graph_t = g;
        GGF_CK(cudaGraphInstantiate(&ch.gexec_t, g, 0));
        ch.gev_cat = ctx->ev_cat;
        ch.gev_n = ctx->ev_used;
    } else {
        ch.graph = g;
        GGF_CK(cudaGraphInstantiate(&ch.gexec, g, 0));
    }
    ch.graph_launches = ctx->launches - l0;
    ctx->launches = l0;
    ctx->ev_cat.clear();
    ctx->ev_used = 0;
    return GGF_OK;
}

ggf_status accumulate_events(ggf_ctx* ctx, const std::vector<int>& cat, const std::vector<cudaEvent_t>& pool) {
    for (size_t k = 0; k + 2 < cat.size(); k += 3) {
        float ms = 0;
        GGF_CK(cudaEventElapsedTime(&ms, pool[cat[k + 1]], pool[cat[k + 2]]));
        ctx->kt_ms[cat[k]] += ms;
        ctx->kt_n[cat[k]] += 1;
    }
    return GGF_OK;
}

// After a sweep's kernels: observables out, refresh of the marked chains.
// With timing on, the events of the sweep (eager launch, or the timed graph's
// record nodes) are accumulated before the refresh records its own.
// launched: 0 eager sweep, 1 plain graph (no timing events), 2 timed graph.
ggf_status finish_sweep(ggf_ctx* ctx, double* obs_dst, int mem, int launched) {
    const bool graph_launched = launched != 0;
    Chains& ch = ctx->ch;
    cudaStream_t cs = ch.cs;
    if (obs_dst)
        GGF_CK(cudaMemcpyAsync(obs_dst, ch.d_obs_stage, (size_t)ch.n * GGF_N_OBS * sizeof(double),
                               mem == GGF_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, cs));
    int cnt = 0, derr = 0;
    GGF_CK(cudaMemcpyAsync(&cnt, ch.refresh_list, sizeof(int), cudaMemcpyDeviceToHost, cs));
    GGF_CK(cudaMemcpyAsync(&derr, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, cs));
    GGF_CK(cudaStreamSynchronize(cs));
    // a bounded device wait that ran out ends the call after this sweep
    if (derr) return ggf_fail(ctx, GGF_ETIMEOUT, "a bounded device wait ran out (tensor-core flush)");
    if (ctx->prof) {
        if (launched == 2) {
            GGF_TRY(accumulate_events(ctx, ch.gev_cat, ctx->ev));
            ctx->ev_used = ch.gev_n;     // the graph's events stay reserved for its next replay
        } else if (launched == 1) {
            ctx->ev_used = ch.gev_n;     // a plain replay records nothing
        } else {
            GGF_TRY(accumulate_events(ctx, ctx->ev_cat, ctx->ev));
            ctx->ev_used = 0;
        }
        ctx->ev_cat.clear();
    }
    if (cnt > 0) {
        std::vector<int> list(cnt);
        GGF_CK(cudaMemcpyAsync(list.data(), ch.refresh_list + 1, cnt * sizeof(int), cudaMemcpyDeviceToHost, cs));
        GGF_CK(cudaStreamSynchronize(cs));
        std::sort(list.begin(), list.end());
        const int r0 = ctx->prof_mark(cs);
        GGF_TRY(factor_chains(ctx, list, false, cs));
        ctx->prof_pair(GGF_KT_REFRESH, r0, ctx->prof_mark(cs));
        GGF_CK(cudaStreamSynchronize(cs));
        if (ctx->prof) {
            GGF_TRY(accumulate_events(ctx, ctx->ev_cat, ctx->ev));
            ctx->ev_cat.clear();
            ctx->ev_used = graph_launched ? ch.gev_n : 0;
        }
        unsigned long long h[4];
        GGF_CK(cudaMemcpy(h, ch.counters, sizeof(h), cudaMemcpyDeviceToHost));
        h[2] += cnt;
        GGF_CK(cudaMemcpy(ch.counters + 2, &h[2], sizeof(unsigned long long), cudaMemcpyHostToDevice));
    }
    ch.sweep += 1;
    return GGF_OK;
}

ggf_status check_err_word(ggf_ctx* ctx) {
    int herr = 0;
    GGF_CK(cudaMemcpy(&herr, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (herr) return ggf_fail(ctx, GGF_ETIMEOUT, "a bounded device wait ran out (tensor-core flush)");
    return GGF_OK;
}

}  // namespace

extern "C" {

ggf_status ggf_sample(ggf_ctx* ctx, int n_sweeps, double* obs, int mem, void* stream) {
    GGF_TRY(require(ctx, true, true));
    if (n_sweeps < 0) return ggf_fail(ctx, GGF_EINVAL, "n_sweeps < 0");
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    Chains& ch = ctx->ch;
    // the library stream waits for the caller's stream, and the caller's stream for it at the end
    GGF_CK(cudaEventRecord(ch.join, st));
    GGF_CK(cudaStreamWaitEvent(ch.cs, ch.join, 0));
    // graph mode replays the captured sweep; with per-kernel timing on, the
    // replayed graph is the same sweep with timing-event record nodes
    const bool use_graph = ch.opts.graph != 0;
    for (int s = 0; s < n_sweeps; ++s) {
        NvtxRange range("ggf_sample sweep");
        if (use_graph) {
            GGF_TRY(ensure_graph(ctx, ctx->prof));
            GGF_CK(cudaGraphLaunch(ctx->prof ? ch.gexec_t : ch.gexec, ch.cs));
            ctx->launches += ch.graph_launches;
        } else {
            ctx->ev_used = 0;
            ctx->ev_cat.clear();
            GGF_TRY(sweep_body(ctx, ch.cs));
        }
        GGF_TRY(finish_sweep(ctx, obs ? obs + (size_t)s * ch.n * GGF_N_OBS : nullptr, mem,
                             use_graph ? (ctx->prof ? 2 : 1) : 0));
    }
    GGF_CK(cudaEventRecord(ch.join, ch.cs));
    GGF_CK(cudaStreamWaitEvent(st, ch.join, 0));
    GGF_CK(cudaStreamSynchronize(st));
    return check_err_word(ctx);
}

ggf_status ggf_sample_group(ggf_ctx* const* ctxs, int n_ctx, int n_sweeps, double* const* obs, int mem,
                            void* stream) {
    NvtxRange range("ggf_sample_group");
    if (!ctxs || n_ctx < 1 || n_sweeps < 0) return GGF_EINVAL;
    for (int k = 0; k < n_ctx; ++k) {
        GGF_TRY(require(ctxs[k], true, true));
        if (ctxs[k]->device != ctxs[0]->device) return ggf_fail(ctxs[0], GGF_EINVAL, "contexts on different devices");
        if (!ctxs[k]->ch.opts.graph) return ggf_fail(ctxs[k], GGF_EINVAL, "group sampling needs graph mode");
        for (int m = 0; m < k; ++m)
            if (ctxs[m] == ctxs[k]) return ggf_fail(ctxs[k], GGF_EINVAL, "context listed twice");
    }
    ggf_ctx* ctx = ctxs[0];
    cudaSetDevice(ctx->device);
    for (int k = 0; k < n_ctx; ++k) GGF_TRY(ensure_graph(ctxs[k]));
    // one parent graph whose independent children are the contexts' sweeps
    cudaGraph_t pg = nullptr;
    cudaGraphExec_t pexec = nullptr;
    GGF_CK(cudaGraphCreate(&pg, 0));
    for (int k = 0; k < n_ctx; ++k) {
        cudaGraphNode_t node;
        cudaError_t e = cudaGraphAddChildGraphNode(&node, pg, nullptr, 0, ctxs[k]->ch.graph);
        if (e != cudaSuccess) { cudaGraphDestroy(pg); return ggf_cuda(ctx, e, "cudaGraphAddChildGraphNode"); }
    }
    cudaError_t e = cudaGraphInstantiate(&pexec, pg, 0);
    if (e != cudaSuccess) { cudaGraphDestroy(pg); return ggf_cuda(ctx, e, "cudaGraphInstantiate(group)"); }
    cudaStream_t st = (cudaStream_t)stream;
    cudaStream_t gs = ctx->ch.cs;
    ggf_status rc = GGF_OK;
    do {
        if (cudaEventRecord(ctx->ch.join, st) != cudaSuccess || cudaStreamWaitEvent(gs, ctx->ch.join, 0) != cudaSuccess) {
            rc = ggf_fail(ctx, GGF_ECUDA, "stream join failed");
            break;
        }
        for (int s = 0; s < n_sweeps && rc == GGF_OK; ++s) {
            e = cudaGraphLaunch(pexec, gs);
            if (e != cudaSuccess) { rc = ggf_cuda(ctx, e, "cudaGraphLaunch(group)"); break; }
            // the other contexts' streams see the group launch before their own copies and refreshes
            if (cudaEventRecord(ctx->ch.join, gs) != cudaSuccess) { rc = ggf_fail(ctx, GGF_ECUDA, "event"); break; }
            for (int k = 0; k < n_ctx && rc == GGF_OK; ++k) {
                ggf_ctx* c = ctxs[k];
                c->launches += c->ch.graph_launches;
                if (k > 0) cudaStreamWaitEvent(c->ch.cs, ctx->ch.join, 0);
                double* dst = (obs && obs[k]) ? obs[k] + (size_t)s * c->ch.n * GGF_N_OBS : nullptr;
                rc = finish_sweep(c, dst, mem, 1);   // no per-kernel timing in group mode
            }
        }
        if (rc == GGF_OK) {
            cudaEventRecord(ctx->ch.join, gs);
            cudaStreamWaitEvent(st, ctx->ch.join, 0);
            if (cudaStreamSynchronize(st) != cudaSuccess) rc = ggf_fail(ctx, GGF_ECUDA, "group sync failed");
        }
    } while (0);
    cudaGraphExecDestroy(pexec);
    cudaGraphDestroy(pg);
    for (int k = 0; k < n_ctx && rc == GGF_OK; ++k) {
        // each context's later work must also see the group's last sweep
        cudaStreamSynchronize(ctxs[k]->ch.cs);
        rc = check_err_word(ctxs[k]);
    }
    return rc;
}

ggf_status ggf_chains_links(ggf_ctx* ctx, void* links, int mem, void* stream) {
    GGF_TRY(require(ctx, true, true));
    if (!links) return ggf_fail(ctx, GGF_EINVAL, "null links");
    cudaSetDevice(ctx->device);
    size_t lb = (size_t)ctx->ch.n * ctx->g.n_links * link_bytes(ctx->g);
    cudaStream_t st = (cudaStream_t)stream;
    GGF_CK(cudaMemcpyAsync(links, ctx->ch.links, lb,
                           mem == GGF_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st));
    GGF_CK(cudaStreamSynchronize(st));
    return GGF_OK;
}

ggf_status ggf_chains_ell(ggf_ctx* ctx, double* ell, int mem, void* stream) {
    GGF_TRY(require(ctx, true, true));
    if (!ell) return ggf_fail(ctx, GGF_EINVAL, "null ell");
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    GGF_CK(cudaMemcpyAsync(ell, ctx->ch.ell, (size_t)ctx->ch.n * ctx->P * sizeof(cxd),
                           mem == GGF_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st));
    GGF_CK(cudaStreamSynchronize(st));
    return GGF_OK;
}

ggf_status ggf_chains_electric(ggf_ctx* ctx, double* out, int mem, void* stream) {
    GGF_TRY(require(ctx, true, true));
    if (!out) return ggf_fail(ctx, GGF_EINVAL, "null out");
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = (size_t)ctx->ch.n * ctx->g.n_links * sizeof(cxd);
    if (mem == GGF_MEM_HOST) {
        DBuf d;
        GGF_TRY(dalloc(ctx, d, bytes));
        GGF_TRY(ggf_electric(ctx, (cxd*)d.p, nullptr, st));
        GGF_CK(cudaMemcpyAsync(out, d.p, bytes, cudaMemcpyDeviceToHost, st));
        GGF_CK(cudaStreamSynchronize(st));
        return check_err_word(ctx);
    }
    GGF_TRY(ggf_electric(ctx, (cxd*)out, nullptr, st));
    return GGF_OK;
}

ggf_status ggf_chains_electric_field(ggf_ctx* ctx, double* out, int mem, void* stream) {
    GGF_TRY(require(ctx, true, true));
    if (!out) return ggf_fail(ctx, GGF_EINVAL, "null out");
    if (ctx->g.group != GGF_U1) return ggf_fail(ctx, GGF_EINVAL, "the electric field insertion is defined for U(1)");
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = (size_t)ctx->ch.n * ctx->g.n_links * sizeof(cxd);
    if (mem == GGF_MEM_HOST) {
        DBuf d;
        GGF_TRY(dalloc(ctx, d, bytes));
        GGF_TRY(ggf_electric(ctx, (cxd*)d.p, nullptr, st, true));
        GGF_CK(cudaMemcpyAsync(out, d.p, bytes, cudaMemcpyDeviceToHost, st));
        GGF_CK(cudaStreamSynchronize(st));
        return check_err_word(ctx);
    }
    GGF_TRY(ggf_electric(ctx, (cxd*)out, nullptr, st, true));
    return GGF_OK;
}

ggf_status ggf_chains_fermion(ggf_ctx* ctx, double* site, double* link, int mem, void* stream) {
    GGF_TRY(require(ctx, true, true));
    if (!site && !link) return ggf_fail(ctx, GGF_EINVAL, "site and link are both null");
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t sb = (size_t)ctx->ch.n * ctx->g.V * sizeof(cxd);
    const size_t lb = (size_t)ctx->ch.n * ctx->g.n_links * 4 * sizeof(cxd);
    if (mem == GGF_MEM_HOST) {
        DBuf ds, dl;
        if (site) GGF_TRY(dalloc(ctx, ds, sb));
        if (link) GGF_TRY(dalloc(ctx, dl, lb));
        GGF_TRY(ggf_fermion(ctx, (cxd*)ds.p, (cxd*)dl.p, nullptr, nullptr, st));
        if (site) GGF_CK(cudaMemcpyAsync(site, ds.p, sb, cudaMemcpyDeviceToHost, st));
        if (link) GGF_CK(cudaMemcpyAsync(link, dl.p, lb, cudaMemcpyDeviceToHost, st));
        GGF_CK(cudaStreamSynchronize(st));
        return check_err_word(ctx);
    }
    GGF_TRY(ggf_fermion(ctx, (cxd*)site, (cxd*)link, nullptr, nullptr, st));
    return GGF_OK;
}

ggf_status ggf_chains_link_terms(ggf_ctx* ctx, const int* charges, double* out, double* pair_out, int mem,
                                 void* stream) {
    GGF_TRY(require(ctx, true, true));
    if (!charges || (!out && !pair_out)) return ggf_fail(ctx, GGF_EINVAL, "need charges and an output");
    const Geometry& g = ctx->g;
    if (g.group != GGF_Z2 && g.group != GGF_U1)
        return ggf_fail(ctx, GGF_EINVAL, "link terms are defined for Z2 and U(1) chains");
    for (int s = 0; s < g.V; ++s)
        if (charges[s] == 0) return ggf_fail(ctx, GGF_EINVAL, "site charges must be nonzero");
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t ob = (size_t)ctx->ch.n * g.n_links * sizeof(cxd), pb = ob * ctx->K * ctx->K;
    DBuf dq, blk, pblk, dout, dpout;
    GGF_TRY(dalloc(ctx, dq, (size_t)g.V * sizeof(int)));
    GGF_CK(cudaMemcpyAsync(dq.p, charges, (size_t)g.V * sizeof(int), cudaMemcpyHostToDevice, st));
    if (out) GGF_TRY(dalloc(ctx, blk, 4 * ob));
    if (pair_out) GGF_TRY(dalloc(ctx, pblk, 4 * pb));
    cxd* o = (cxd*)out;
    cxd* po = (cxd*)pair_out;
    if (mem == GGF_MEM_HOST) {
        if (out) { GGF_TRY(dalloc(ctx, dout, ob)); o = (cxd*)dout.p; }
        if (pair_out) { GGF_TRY(dalloc(ctx, dpout, pb)); po = (cxd*)dpout.p; }
    }
    GGF_TRY(ggf_link_terms(ctx, (const int*)dq.p, (cxd*)blk.p, (cxd*)pblk.p, o, po, st));
    if (mem == GGF_MEM_HOST) {
        if (out) GGF_CK(cudaMemcpyAsync(out, o, ob, cudaMemcpyDeviceToHost, st));
        if (pair_out) GGF_CK(cudaMemcpyAsync(pair_out, po, pb, cudaMemcpyDeviceToHost, st));
    }
    // the scratch buffers are released on return
    GGF_CK(cudaStreamSynchronize(st));
    return check_err_word(ctx);
}

ggf_status ggf_chains_pairs(ggf_ctx* ctx, int what, double* out, int mem, void* stream) {
    GGF_TRY(require(ctx, true, true));
    if (!out) return ggf_fail(ctx, GGF_EINVAL, "null out");
    const Geometry& g = ctx->g;
    const size_t KK = (size_t)ctx->K * ctx->K, n = ctx->ch.n;
    size_t items;
    switch (what) {
        case GGF_PAIRS_NORM: items = 1; break;
        case GGF_PAIRS_ELECTRIC: items = g.n_links; break;
        case GGF_PAIRS_SITE: items = g.V; break;
        case GGF_PAIRS_LINK: items = (size_t)g.n_links * 4; break;
        case GGF_PAIRS_FOUR: items = g.n_links; break;
        case GGF_PAIRS_FIELD:
            if (g.group != GGF_U1) return ggf_fail(ctx, GGF_EINVAL, "the field's pair parts are defined for U(1)");
            items = g.n_links;
            break;
        default: return ggf_fail(ctx, GGF_EINVAL, "unknown pair quantity");
    }
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = n * items * KK * sizeof(cxd);
    DBuf d;
    cxd* dst = (cxd*)out;
    if (mem == GGF_MEM_HOST) {
        GGF_TRY(dalloc(ctx, d, bytes));
        dst = (cxd*)d.p;
    }
    if (what == GGF_PAIRS_NORM) GGF_TRY(ggf_pair_norm(ctx, dst, st));
    else if (what == GGF_PAIRS_ELECTRIC) GGF_TRY(ggf_electric(ctx, nullptr, dst, st));
    else if (what == GGF_PAIRS_FIELD) GGF_TRY(ggf_electric(ctx, nullptr, dst, st, true));
    else if (what == GGF_PAIRS_FOUR) GGF_TRY(ggf_fermion4(ctx, nullptr, st, dst));
    else if (what == GGF_PAIRS_SITE) GGF_TRY(ggf_fermion(ctx, nullptr, nullptr, dst, nullptr, st));
    else GGF_TRY(ggf_fermion(ctx, nullptr, nullptr, nullptr, dst, st));
    if (mem == GGF_MEM_HOST) {
        GGF_CK(cudaMemcpyAsync(out, dst, bytes, cudaMemcpyDeviceToHost, st));
        GGF_CK(cudaStreamSynchronize(st));
        return check_err_word(ctx);
    }
    return GGF_OK;
}

ggf_status ggf_chains_fermion4(ggf_ctx* ctx, double* out, int mem, void* stream) {
    GGF_TRY(require(ctx, true, true));
    if (!out) return ggf_fail(ctx, GGF_EINVAL, "null out");
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = (size_t)ctx->ch.n * ctx->g.n_links * sizeof(cxd);
    if (mem == GGF_MEM_HOST) {
        DBuf d;
        GGF_TRY(dalloc(ctx, d, bytes));
        GGF_TRY(ggf_fermion4(ctx, (cxd*)d.p, st));
        GGF_CK(cudaMemcpyAsync(out, d.p, bytes, cudaMemcpyDeviceToHost, st));
        GGF_CK(cudaStreamSynchronize(st));
        return check_err_word(ctx);
    }
    GGF_TRY(ggf_fermion4(ctx, (cxd*)out, st));
    return GGF_OK;
}

ggf_status ggf_chains_link_score(ggf_ctx* ctx, double* out, int mem, void* stream) {
    GGF_TRY(require(ctx, true, true));
    if (!out) return ggf_fail(ctx, GGF_EINVAL, "null out");
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = (size_t)ctx->ch.n * ctx->P * ctx->g.n_links * ctx->g.r * ctx->g.r * sizeof(cxd);
    if (mem == GGF_MEM_HOST) {
        DBuf d;
        GGF_TRY(dalloc(ctx, d, bytes));
        GGF_TRY(ggf_link_score(ctx, (cxd*)d.p, st));
        GGF_CK(cudaMemcpyAsync(out, d.p, bytes, cudaMemcpyDeviceToHost, st));
        GGF_CK(cudaStreamSynchronize(st));
        return check_err_word(ctx);
    }
    GGF_TRY(ggf_link_score(ctx, (cxd*)out, st));
    return GGF_OK;
}

ggf_status ggf_chains_score(ggf_ctx* ctx, double* out, int mem, void* stream) {
    GGF_TRY(require(ctx, true, true));
    if (!out) return ggf_fail(ctx, GGF_EINVAL, "null out");
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = (size_t)ctx->ch.n * ctx->g.V * ctx->g.B * ctx->g.B * sizeof(double);
    if (mem == GGF_MEM_HOST) {
        DBuf d;
        GGF_TRY(dalloc(ctx, d, bytes));
        GGF_TRY(ggf_score(ctx, (double*)d.p, st));
        GGF_CK(cudaMemcpyAsync(out, d.p, bytes, cudaMemcpyDeviceToHost, st));
        GGF_CK(cudaStreamSynchronize(st));
        return check_err_word(ctx);
    }
    GGF_TRY(ggf_score(ctx, out, st));
    return GGF_OK;
}

ggf_status ggf_debug_poison_inverse(ggf_ctx* ctx, int chain, int pair, int i, int j) {
    GGF_TRY(require(ctx, true, true));
    Chains& ch = ctx->ch;
    const int N = ctx->g.N;
    if (chain < 0 || chain >= ch.n || pair < 0 || pair >= ctx->P || i < 0 || i >= N || j < 0 || j >= N)
        return ggf_fail(ctx, GGF_EINVAL, "bad debug_poison_inverse arguments");
    cudaSetDevice(ctx->device);
    const bool fp64 = ch.opts.precision == GGF_FP64;
    const size_t rsz = fp64 ? sizeof(double) : sizeof(float);
    const bool cplx = pair >= ctx->K;
    const size_t esz = cplx ? 2 * rsz : rsz;
    const size_t NN = (size_t)N * N, e = (size_t)i * N + j;
    unsigned char* base = cplx ? (unsigned char*)ch.Wc + ((size_t)chain * ctx->Kc + (pair - ctx->K)) * NN * esz
                               : (unsigned char*)ch.Wr + ((size_t)chain * ctx->K + pair) * NN * esz;
    const double nd = NAN;
    const float nf = NAN;
    GGF_CK(cudaDeviceSynchronize());
    GGF_CK(cudaMemcpy(base + e * esz, fp64 ? (const void*)&nd : (const void*)&nf, rsz, cudaMemcpyHostToDevice));
    return GGF_OK;
}

}  // extern "C"

namespace {
__global__ void scale_kernel(float* W, size_t n, float f) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) W[i] *= f;
}
}  // namespace

extern "C" {

ggf_status ggf_debug_scale_inverse(ggf_ctx* ctx, int chain, int pair, double factor) {
    GGF_TRY(require(ctx, true, true));
    Chains& ch = ctx->ch;
    if (chain < 0 || chain >= ch.n || pair < 0 || pair >= ctx->P)
        return ggf_fail(ctx, GGF_EINVAL, "bad debug_scale_inverse arguments");
    if (ch.opts.precision != GGF_FP32) return ggf_fail(ctx, GGF_EINVAL, "debug_scale_inverse: FP32 chains only");
    cudaSetDevice(ctx->device);
    const size_t NN = (size_t)ctx->g.N * ctx->g.N;
    const bool cplx = pair >= ctx->K;
    const int p = cplx ? pair - ctx->K : pair;
    float* W = cplx ? (float*)ch.Wc + ((size_t)chain * ctx->Kc + p) * NN * 2
                    : (float*)ch.Wr + ((size_t)chain * ctx->K + p) * NN;
    const size_t n = NN * (cplx ? 2 : 1);
    GGF_CK(cudaDeviceSynchronize());
    scale_kernel<<<(unsigned)((n + 255) / 256), 256>>>(W, n, (float)factor);
    GGF_CK(cudaGetLastError());
    GGF_CK(cudaDeviceSynchronize());
    return GGF_OK;
}

ggf_status ggf_chains_refine(ggf_ctx* ctx, int chain, int pair, int apply, double* rmax) {
    GGF_TRY(require(ctx, true, true));
    Chains& ch = ctx->ch;
    if (chain < 0 || chain >= ch.n || pair < 0 || pair >= ctx->P || !rmax)
        return ggf_fail(ctx, GGF_EINVAL, "bad chains_refine arguments");
    if (ch.opts.precision != GGF_FP32) return ggf_fail(ctx, GGF_EINVAL, "chains_refine: FP32 chains only");
    cudaSetDevice(ctx->device);
    const int N = ctx->g.N;
    const size_t NN = (size_t)N * N;
    const bool cplx = pair >= ctx->K;
    const int p = cplx ? pair - ctx->K : pair;
    float* W = cplx ? (float*)ch.Wc + ((size_t)chain * ctx->Kc + p) * NN * 2
                    : (float*)ch.Wr + ((size_t)chain * ctx->K + p) * NN;
    GGF_CK(cudaDeviceSynchronize());
    GGF_TRY(ggf_workspace(ctx, ggf_refine_bytes(N, cplx)));
    GGF_TRY(ggf_refine_inverse(ctx, cplx, ch.links, chain, p, W, ctx->work, 0, rmax, 0));
    if (apply && *rmax <= kRefineTol) {
        double unused = 0.0;
        GGF_TRY(ggf_refine_inverse(ctx, cplx, ch.links, chain, p, W, ctx->work, *rmax <= kRefineOne ? 1 : 3, &unused, 0));
    }
    GGF_CK(cudaDeviceSynchronize());
    return GGF_OK;
}

ggf_status ggf_chains_inverse(ggf_ctx* ctx, int chain, int pair, double* out, int mem, void* stream) {
    GGF_TRY(require(ctx, true, true));
    Chains& ch = ctx->ch;
    if (chain < 0 || chain >= ch.n || pair < 0 || pair >= ctx->P || !out)
        return ggf_fail(ctx, GGF_EINVAL, "bad chains_inverse arguments");
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t NN = (size_t)ctx->g.N * ctx->g.N;
    const bool fp64 = ch.opts.precision == GGF_FP64;
    const size_t rsz = fp64 ? sizeof(double) : sizeof(float);
    const bool cplx = pair >= ctx->K;
    const size_t esz = cplx ? 2 * rsz : rsz;
    const unsigned char* src = cplx ? (const unsigned char*)ch.Wc + ((size_t)chain * ctx->Kc + (pair - ctx->K)) * NN * esz
                                    : (const unsigned char*)ch.Wr + ((size_t)chain * ctx->K + pair) * NN * esz;
    std::vector<unsigned char> h(NN * esz);
    GGF_CK(cudaStreamSynchronize(st));
    GGF_CK(cudaMemcpy(h.data(), src, h.size(), cudaMemcpyDeviceToHost));
    std::vector<double> o(2 * NN);
    for (size_t e = 0; e < NN; ++e) {
        double re, im = 0.0;
        if (fp64) { const double* d = (const double*)h.data(); re = cplx ? d[2 * e] : d[e]; if (cplx) im = d[2 * e + 1]; }
        else { const float* f = (const float*)h.data(); re = cplx ? f[2 * e] : f[e]; if (cplx) im = f[2 * e + 1]; }
        o[2 * e] = re; o[2 * e + 1] = im;
    }
    GGF_CK(cudaMemcpy(out, o.data(), o.size() * sizeof(double), mem == GGF_MEM_HOST ? cudaMemcpyHostToHost : cudaMemcpyHostToDevice));
    return GGF_OK;
}

ggf_status ggf_chains_status(ggf_ctx* ctx, double drift_tol, int32_t* status, int mem, void* stream) {
    GGF_TRY(require(ctx, true, true));
    if (!status) return ggf_fail(ctx, GGF_EINVAL, "null status");
    cudaSetDevice(ctx->device);
    Chains& ch = ctx->ch;
    cudaStream_t st = (cudaStream_t)stream;
    int32_t* d = status;
    DBuf tmp;
    if (mem == GGF_MEM_HOST) {
        GGF_TRY(dalloc(ctx, tmp, (size_t)ch.n * sizeof(int32_t)));
        d = (int32_t*)tmp.p;
    }
    status_kernel<<<(ch.n + 127) / 128, 128, 0, st>>>(ch.n, ctx->P, ch.ell, ch.drift, ch.flags, drift_tol, d);
    GGF_CK(cudaGetLastError());
    if (mem == GGF_MEM_HOST)
        GGF_CK(cudaMemcpyAsync(status, d, (size_t)ch.n * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    GGF_CK(cudaStreamSynchronize(st));
    return GGF_OK;
}

ggf_status ggf_chains_stats(ggf_ctx* ctx, ggf_chain_stats* out) {
    GGF_TRY(require(ctx, true, true));
    if (!out) return ggf_fail(ctx, GGF_EINVAL, "null stats");
    cudaSetDevice(ctx->device);
    unsigned long long h[6];
    GGF_CK(cudaMemcpy(h, ctx->ch.counters, sizeof(h), cudaMemcpyDeviceToHost));
    std::vector<double> d(ctx->ch.n);
    GGF_CK(cudaMemcpy(d.data(), ctx->ch.drift, d.size() * sizeof(double), cudaMemcpyDeviceToHost));
    out->proposals = h[0];
    out->accepts = h[1];
    out->refreshes = h[2];
    out->sweeps = ctx->ch.sweep;
    out->max_drift = d.empty() ? 0.0 : *std::max_element(d.begin(), d.end());
    out->n_chains = ctx->ch.n;
    out->launches = ctx->launches;
    out->block_proposals = h[4];
    out->block_accepts = h[5];
    out->n_pairs = ctx->P;
    out->max_resid = ctx->refine_rmax;
    out->dense_refreshes = ctx->dense_refreshes;
    out->refine_steps = ctx->refine_steps;
    out->dense_pfaffians = ctx->dense_pfaffians;
    out->flush_wave = ctx->ch.ps ? (uint64_t)ctx->ch.ps_wave : 0;
    if (h[3]) return ggf_fail(ctx, GGF_ESINGULAR, "a refresh met a singular M(G)");
    return GGF_OK;
}

// In-memory chain state (residency waves): header, then the device arrays.
struct StateHeader {
    char magic[8];
    int geo[8];                 // L, group, n_v, K, n, P, precision, kmax
    ggf_chain_opts opts;
    uint64_t sweep, block_moves;
    unsigned long long counters[6];
};

struct StatePart {
    void* dev;
    size_t bytes;
};

static std::vector<StatePart> state_parts(ggf_ctx* ctx) {
    Chains& ch = ctx->ch;
    const Geometry& g = ctx->g;
    const size_t rsz = ch.opts.precision == GGF_FP64 ? sizeof(double) : sizeof(float);
    const size_t NN = (size_t)g.N * g.N;
    return {{ch.links, (size_t)ch.n * g.n_links * link_bytes(g)},
            {ch.Wr, (size_t)ch.n * ctx->K * NN * rsz},
            {ch.Wc, (size_t)ch.n * ctx->Kc * NN * 2 * rsz},
            {ch.ell, (size_t)ch.n * ctx->P * sizeof(cxd)},
            {ch.since_refresh, (size_t)ch.n * sizeof(int)},
            {ch.drift, (size_t)ch.n * sizeof(double)},
            {ch.flags, (size_t)ch.n * sizeof(int)}};
}

static size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

ggf_status ggf_chains_state_size(ggf_ctx* ctx, uint64_t* bytes) {
    GGF_TRY(require(ctx, true, true));
    if (!bytes) return ggf_fail(ctx, GGF_EINVAL, "null bytes");
    size_t total = align_up(sizeof(StateHeader));
    for (const StatePart& q : state_parts(ctx)) total += align_up(q.bytes);
    *bytes = total;
    return GGF_OK;
}

ggf_status ggf_chains_save_state(ggf_ctx* ctx, void* dst, int mem, void* stream) {
    GGF_TRY(require(ctx, true, true));
    if (!dst) return ggf_fail(ctx, GGF_EINVAL, "null dst");
    cudaSetDevice(ctx->device);
    Chains& ch = ctx->ch;
    const Geometry& g = ctx->g;
    cudaStream_t st = (cudaStream_t)stream;
    GGF_TRY(ggf_flush(ctx, st));
    GGF_CK(cudaStreamSynchronize(st));
    GGF_CK(cudaStreamSynchronize(ch.cs));
    StateHeader h{};
    std::memcpy(h.magic, "GGFSTAT2", 8);
    const int geo[8] = {g.L, g.group, g.n_v, ctx->K, ch.n, ctx->P, ch.opts.precision, ch.kmax};
    std::memcpy(h.geo, geo, sizeof(geo));
    h.opts = ch.opts;
    h.sweep = ch.sweep;
    h.block_moves = ch.block_moves;
    GGF_CK(cudaMemcpy(h.counters, ch.counters, sizeof(h.counters), cudaMemcpyDeviceToHost));
    const cudaMemcpyKind down = mem == GGF_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    unsigned char* out = (unsigned char*)dst;
    GGF_CK(cudaMemcpy(out, &h, sizeof(h), mem == GGF_MEM_HOST ? cudaMemcpyHostToHost : cudaMemcpyHostToDevice));
    size_t off = align_up(sizeof(StateHeader));
    for (const StatePart& q : state_parts(ctx)) {
        if (q.bytes) GGF_CK(cudaMemcpyAsync(out + off, q.dev, q.bytes, down, st));
        off += align_up(q.bytes);
    }
    GGF_CK(cudaStreamSynchronize(st));
    return GGF_OK;
}

ggf_status ggf_chains_load_state(ggf_ctx* ctx, const void* src, int mem, void* stream) {
    GGF_TRY(require(ctx, true, true));
    if (!src) return ggf_fail(ctx, GGF_EINVAL, "null src");
    cudaSetDevice(ctx->device);
    Chains& ch = ctx->ch;
    const Geometry& g = ctx->g;
    cudaStream_t st = (cudaStream_t)stream;
    StateHeader h;
    GGF_CK(cudaMemcpy(&h, src, sizeof(h), mem == GGF_MEM_HOST ? cudaMemcpyHostToHost : cudaMemcpyDeviceToHost));
    const int geo[8] = {g.L, g.group, g.n_v, ctx->K, ch.n, ctx->P, ch.opts.precision, ch.kmax};
    if (std::memcmp(h.magic, "GGFSTAT2", 8) != 0 || std::memcmp(h.geo, geo, sizeof(geo)) != 0)
        return ggf_fail(ctx, GGF_EINVAL, "state does not match the context's problem, chains, precision or delay");
    GGF_CK(cudaStreamSynchronize(st));
    GGF_CK(cudaStreamSynchronize(ch.cs));
    const cudaMemcpyKind up = mem == GGF_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    const unsigned char* in = (const unsigned char*)src;
    size_t off = align_up(sizeof(StateHeader));
    for (const StatePart& q : state_parts(ctx)) {
        if (q.bytes) GGF_CK(cudaMemcpyAsync(q.dev, in + off, q.bytes, up, st));
        off += align_up(q.bytes);
    }
    GGF_CK(cudaMemcpyAsync(ch.counters, h.counters, sizeof(h.counters), cudaMemcpyHostToDevice, st));
    unsigned long long sw = h.sweep;
    GGF_CK(cudaMemcpyAsync(ch.d_sweep, &sw, sizeof(sw), cudaMemcpyHostToDevice, st));
    GGF_CK(cudaMemsetAsync(ch.pend, 0, (size_t)ch.n * sizeof(int), st));
    GGF_CK(cudaStreamSynchronize(st));
    ch.opts = h.opts;              // seed, width, refresh cadence of the saved chains
    ch.sweep = h.sweep;
    ch.block_moves = h.block_moves;
    ch.steps_since_flush = 0;
    drop_graph(ch);                // the captured sweep holds the previous options
    return GGF_OK;
}

ggf_status ggf_checkpoint(ggf_ctx* ctx, const char* path) {
    GGF_TRY(require(ctx, true, true));
    if (!path) return ggf_fail(ctx, GGF_EINVAL, "null path");
    cudaSetDevice(ctx->device);
    Chains& ch = ctx->ch;
    const Geometry& g = ctx->g;
    size_t lb = (size_t)ch.n * g.n_links * link_bytes(g);
    std::vector<unsigned char> hl(lb);
    std::vector<cxd> he((size_t)ch.n * ctx->P);
    std::vector<int> hs(ch.n);
    unsigned long long cnt[4];
    GGF_CK(cudaDeviceSynchronize());
    GGF_CK(cudaMemcpy(hl.data(), ch.links, lb, cudaMemcpyDeviceToHost));
    GGF_CK(cudaMemcpy(he.data(), ch.ell, he.size() * sizeof(cxd), cudaMemcpyDeviceToHost));
    GGF_CK(cudaMemcpy(hs.data(), ch.since_refresh, hs.size() * sizeof(int), cudaMemcpyDeviceToHost));
    GGF_CK(cudaMemcpy(cnt, ch.counters, sizeof(cnt), cudaMemcpyDeviceToHost));
    FILE* f = fopen(path, "wb");
    if (!f) return ggf_fail(ctx, GGF_EIO, std::string("cannot open ") + path);
    const char magic[8] = {'G', 'G', 'F', 'C', 'K', 'P', 'T', '3'};
    int hdr[8] = {g.L, g.group, g.n_v, ctx->K, ch.n, ctx->P, 0, 0};
    bool ok = fwrite(magic, 1, 8, f) == 8 && fwrite(hdr, sizeof(hdr), 1, f) == 1 &&
              fwrite(&ch.opts, sizeof(ch.opts), 1, f) == 1 && fwrite(&ch.sweep, sizeof(ch.sweep), 1, f) == 1 &&
              fwrite(cnt, sizeof(cnt), 1, f) == 1 && fwrite(hl.data(), 1, lb, f) == lb &&
              fwrite(he.data(), sizeof(cxd), he.size(), f) == he.size() &&
              fwrite(hs.data(), sizeof(int), hs.size(), f) == hs.size();
    ok = (fclose(f) == 0) && ok;
    if (!ok) return ggf_fail(ctx, GGF_EIO, "checkpoint write failed");
    return GGF_OK;
}

ggf_status ggf_resume(ggf_ctx* ctx, const char* path, void* stream) {
    GGF_TRY(require(ctx, true, false));
    if (!path) return ggf_fail(ctx, GGF_EINVAL, "null path");
    FILE* f = fopen(path, "rb");
    if (!f) return ggf_fail(ctx, GGF_EIO, std::string("cannot open ") + path);
    char magic[8];
    int hdr[8];
    ggf_chain_opts o;
    uint64_t sweep;
    unsigned long long cnt[4];
    bool ok = fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "GGFCKPT3", 8) == 0 &&
              fread(hdr, sizeof(hdr), 1, f) == 1 && fread(&o, sizeof(o), 1, f) == 1 &&
              fread(&sweep, sizeof(sweep), 1, f) == 1 && fread(cnt, sizeof(cnt), 1, f) == 1;
    const Geometry& g = ctx->g;
    if (!ok || hdr[0] != g.L || hdr[1] != g.group || hdr[2] != g.n_v || hdr[3] != ctx->K || hdr[5] != ctx->P) {
        fclose(f);
        return ggf_fail(ctx, GGF_EIO, "checkpoint does not match the context (or is corrupt)");
    }
    int n = hdr[4];
    if (n < 1) { fclose(f); return ggf_fail(ctx, GGF_EIO, "corrupt checkpoint"); }
    size_t lb = (size_t)n * g.n_links * link_bytes(g);
    std::vector<unsigned char> hl(lb);
    std::vector<cxd> he((size_t)n * ctx->P);
    std::vector<int> hs(n);
    ok = fread(hl.data(), 1, lb, f) == lb && fread(he.data(), sizeof(cxd), he.size(), f) == he.size() &&
         fread(hs.data(), sizeof(int), hs.size(), f) == hs.size();
    fclose(f);
    if (!ok) return ggf_fail(ctx, GGF_EIO, "truncated checkpoint");
    GGF_TRY(ggf_chains_init(ctx, n, hl.data(), &o, GGF_MEM_HOST, stream));
    Chains& ch = ctx->ch;
    cudaStream_t st = (cudaStream_t)stream;
    // restore the tracked log-weights: the rebuilt ones agree to rounding, and the
    // tracked values keep the run bit-identical to an uninterrupted one
    GGF_CK(cudaMemcpyAsync(ch.ell, he.data(), he.size() * sizeof(cxd), cudaMemcpyHostToDevice, st));
    GGF_CK(cudaMemcpyAsync(ch.since_refresh, hs.data(), hs.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    GGF_CK(cudaMemcpyAsync(ch.counters, cnt, sizeof(cnt), cudaMemcpyHostToDevice, st));
    unsigned long long sw = sweep;
    GGF_CK(cudaMemcpyAsync(ch.d_sweep, &sw, sizeof(sw), cudaMemcpyHostToDevice, st));
    GGF_CK(cudaStreamSynchronize(st));
    ch.sweep = sweep;
    return GGF_OK;
}

ggf_status ggf_profile(ggf_ctx* ctx, int enable) {
    if (!ctx) return GGF_EINVAL;
    ctx->prof = enable != 0;
    for (int k = 0; k < GGF_KT_N; ++k) { ctx->kt_ms[k] = 0; ctx->kt_n[k] = 0; }
    ctx->ev_cat.clear();
    ctx->ev_used = 0;
    return GGF_OK;
}

ggf_status ggf_kernel_time(ggf_ctx* ctx, int which, double* ms, uint64_t* launches) {
    if (!ctx || which < 0 || which >= GGF_KT_N) return GGF_EINVAL;
    if (ms) *ms = ctx->kt_ms[which];
    if (launches) *launches = ctx->kt_n[which];
    return GGF_OK;
}

ggf_status ggf_sync(ggf_ctx* ctx, void* stream) {
    if (!ctx) return GGF_EINVAL;
    cudaSetDevice(ctx->device);
    GGF_CK(cudaStreamSynchronize((cudaStream_t)stream));
    GGF_CK(cudaGetLastError());
    int herr = 0;
    GGF_CK(cudaMemcpy(&herr, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (herr) return ggf_fail(ctx, GGF_ETIMEOUT, "a bounded device wait ran out (tensor-core flush)");
    return GGF_OK;
}

}  // extern "C"
