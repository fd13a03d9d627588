// Allocation-free variant of ggf_logweight.
//
// Some callers cannot allocate device memory at the point where they need
// log N(G): real-time or embedded hosts whose memory is budgeted once at
// start, a process that shares the GPU under an allocator that forbids
// further cudaMalloc calls, or a loop that cannot pay the implicit device
// synchronisation of cudaFree.  ggf_logweight itself grows a workspace with cudaMalloc,
// so this entry point instead works in one fixed scratch array that lives in
// the library image (a file-scope __device__ array, 32 MiB, held by every GPU
// that loads the library until the process exits).
//
// The scratch is shared by all calls on a device: two calls whose work
// overlaps on the GPU (different streams, or host threads racing) corrupt each
// other's results; serialise them.  Every element the kernels read is written
// first in the same call (the Pfaffian accumulators are set by their own
// initialisation kernel), so nothing depends on what a previous call left.
#include <mutex>
#include "ggf_ctx.h"

namespace {

constexpr size_t kScratchBytes = (size_t)32 << 20;   // 32 MiB
constexpr int kMaxN = 1024;                          // largest M_nm handled (N = 8 n_v L^2)

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void* g_scratch_dev[64] = {nullptr};                // device address per device ordinal

// Host code may not take the address of g_scratch directly (that is a host
// shadow, not device memory): look it up once per device, device current.
ggf_status scratch_for(ggf_ctx* ctx, void** out) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (ctx->device < 0 || ctx->device >= 64) return ggf_fail(ctx, GGF_EINVAL, "device ordinal out of range");
    if (!g_scratch_dev[ctx->device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) return ggf_cuda(ctx, e, "cudaGetSymbolAddress(scratch)");
        g_scratch_dev[ctx->device] = p;
    }
    *out = g_scratch_dev[ctx->device];
    return GGF_OK;
}

// Items i0 .. i0 + n_items - 1 of one family, item = cfg * npf + pair (cfg
// counted from the start of the current chunk of configurations).
__global__ void na_items(int i0, int n_items, int npf, int* cfg, int* pair) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_items) { cfg[i] = (i0 + i) / npf; pair[i] = (i0 + i) % npf; }
}

__global__ void na_write_ell(int i0, int n_items, int npf, int pair_off, int P, bool cplx, const cxd* logpf,
                             const cxd* phase, cxd* ell) {
    int it = blockIdx.x * blockDim.x + threadIdx.x;
    if (it >= n_items) return;
    int c = (i0 + it) / npf, p = (i0 + it) % npf;
    cxd v = {logpf[it].x, 0.0};
    if (cplx) v.y = atan2(phase[it].y, phase[it].x);
    ell[(size_t)c * P + pair_off + p] = v;
}

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

}  // namespace

size_t ggf_factor_tmp_bytes(int n, int batch);

extern "C" ggf_status ggf_logweight_noalloc(ggf_ctx* ctx, int n_cfg, const void* links, double* logN,
                                            void* stream) {
    if (!ctx) return GGF_EINVAL;
    if (!ctx->have_lattice || !ctx->have_group || !ctx->have_gauss)
        return ggf_fail(ctx, GGF_ESTATE, "lattice, group and Gaussians must be initialised");
    if (n_cfg < 0 || !links || !logN) return ggf_fail(ctx, GGF_EINVAL, "bad logweight_noalloc arguments");
    const Geometry& g = ctx->g;
    const int N = g.N, P = ctx->P;
    if (N > kMaxN)
        return ggf_fail(ctx, GGF_EINVAL, "ggf_logweight_noalloc: M is " + std::to_string(N) + " x " +
                                             std::to_string(N) + ", above the fixed-scratch maximum " +
                                             std::to_string(kMaxN) + " (use ggf_logweight)");
    if (n_cfg == 0) return GGF_OK;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return ggf_fail(ctx, GGF_ECUDA, "cudaSetDevice failed");
    cudaStream_t st = (cudaStream_t)stream;
    void* base = nullptr;
    GGF_TRY(scratch_for(ctx, &base));
    const size_t NN = (size_t)N * N;
    // Configurations are taken in chunks whose log-Pfaffians (P per
    // configuration) stay in the scratch until they are combined; within a
    // chunk each family's (configuration, pair) items are factored in groups
    // sized to the rest of the scratch (real items at 8 B per entry, complex
    // at 16 B), so a single item of the largest M (N = kMaxN) always fits.
    const int cfg_chunk = std::min(n_cfg, 4096);
    const size_t ell_bytes = align256((size_t)cfg_chunk * P * sizeof(cxd));
    auto item_bytes = [&](int items, size_t elem) {
        return align256(NN * elem * items) + align256(ggf_factor_tmp_bytes(N, items)) +
               2 * align256((size_t)items * sizeof(int)) + 2 * align256((size_t)items * sizeof(cxd));
    };
    unsigned char* s0 = (unsigned char*)base;
    const size_t lrow = (size_t)g.n_links * (g.group == GGF_Z2 ? 1 : g.group == GGF_SU2 ? 4 * sizeof(double) : sizeof(double));
    for (int c0 = 0; c0 < n_cfg; c0 += cfg_chunk) {
        const int nc = std::min(cfg_chunk, n_cfg - c0);
        const void* lk = (const unsigned char*)links + (size_t)c0 * lrow;
        cxd* ell = (cxd*)s0;
        unsigned char* fam_base = s0 + ell_bytes;
        for (int fam = 0; fam < 2; ++fam) {
            const bool cplx = fam == 1;
            const int npf = cplx ? ctx->Kc : ctx->K;
            if (npf == 0) continue;
            const size_t elem = cplx ? sizeof(cxd) : sizeof(double);
            const int total = nc * npf;
            int group = 0;
            for (int it = total; it >= 1; it = it > 1 ? it / 2 : 0)
                if (ell_bytes + item_bytes(it, elem) <= kScratchBytes) { group = it; break; }
            if (group == 0)
                return ggf_fail(ctx, GGF_EINVAL, "ggf_logweight_noalloc: one item does not fit the scratch");
            for (int i0 = 0; i0 < total; i0 += group) {
                const int items = std::min(group, total - i0);
                unsigned char* q = fam_base;
                void* A = q;
                q += align256(NN * elem * items);
                void* ftmp = q;
                q += align256(ggf_factor_tmp_bytes(N, items));
                int* d_cfg = (int*)q;
                q += align256((size_t)items * sizeof(int));
                int* d_pair = (int*)q;
                q += align256((size_t)items * sizeof(int));
                cxd* d_logpf = (cxd*)q;
                q += align256((size_t)items * sizeof(cxd));
                cxd* d_phase = (cxd*)q;
                na_items<<<(items + 127) / 128, 128, 0, st>>>(i0, items, npf, d_cfg, d_pair);
                GGF_CK(cudaGetLastError());
                GGF_TRY(ggf_assemble(ctx, !cplx, items, d_cfg, d_pair, lk, A, st));
                GGF_TRY(ggf_pfaffian_batched(ctx, cplx, N, items, A, d_logpf, d_phase, ftmp, st));
                na_write_ell<<<(items + 127) / 128, 128, 0, st>>>(i0, items, npf, cplx ? ctx->K : 0, P, cplx,
                                                                  d_logpf, d_phase, ell);
                GGF_CK(cudaGetLastError());
            }
        }
        GGF_TRY(ggf_combine(ctx, nc, ell, logN + c0, st));
    }
    return GGF_OK;
}
