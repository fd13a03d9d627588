// Internal state of a libggf context (not part of the ABI).
#pragma once
#include <string>
#include <vector>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include "ggf_common.cuh"
#include "../../include/ggf.h"

struct Geometry {
    int L = 0, V = 0, n_links = 0;
    int group = -1, n_v = 0;
    int B = 0;    // virtual Majoranas per site, 8 n_v
    int h2 = 0;   // Majoranas per link end, 2 n_v
    int r = 0;    // Majoranas per link, 4 n_v
    int N = 0;    // virtual Majoranas on the lattice, B V
    int q[2] = {0, 0};  // U(1) charges of source-end modes
};

// Read-only data the kernels need, passed by value.
struct DevConst {
    Geometry g;
    int K, P, Kc;                 // Gaussians, pairs, complex pairs (P = K + Kc)
    const double* D;              // [V][B][B]
    const double* Ap;             // [V][2][2]   physical block of each site
    const double* Bp;             // [V][2][B]   physical-virtual coupling of each site
    const double* Gr;             // [K][n_links][r][r]   diagonal pairs
    const cxd* Gc;                // [Kc][n_links][r][r]  pairs n < m
    const cxd* logc;              // [P]
    const cxd* w;                 // [P] combine weights
};

struct Chains {
    int n = 0;
    ggf_chain_opts opts{};
    uint64_t sweep = 0;
    void* links = nullptr;        // int8 or double [n][n_links]
    void* Wr = nullptr;           // [n][K][N][N]   double or float
    void* Wc = nullptr;           // [n][Kc][N][N]  cxd or cxf
    cxd* ell = nullptr;           // [n][P]
    void* zbuf = nullptr;         // [n][P][r][r]  W-precision scalars (complex slot size)
    void* ybuf = nullptr;         // [n][P][r][N]
    int* accept = nullptr;        // [n]
    int* since_refresh = nullptr; // [n]
    int* sweep_acc = nullptr;     // [n]
    unsigned long long* counters = nullptr;  // [6]: proposals, accepts, refreshes, singular, block proposals, block accepts
    double* drift = nullptr;      // [n] max drift seen
    int* flags = nullptr;         // [n] bit 0: a factorisation of this chain met a singular M
    int* refresh_list = nullptr;  // [n + 1]
    // delayed updates (opts.delay > 1): per chain and pair, U^T and V panels
    // [n][pairs][kmax r][N] in W precision, pending count per chain
    void* Pr = nullptr;   // real-family panels [n][K][2][N][kmax r]
    void* Pc = nullptr;   // complex-family panels [n][Kc][2][2][N][kmax r]
    int* pend = nullptr;          // [n]
    // batched delayed updates: small matrices G = W_eff[T, T] and X per chain
    // and pair, real family [n][K][2][kmax r][kmax r] then complex family
    // [n][Kc][2][kmax r][kmax r] (W precision)
    void* Sm = nullptr;
    int kmax = 1;
    int steps_since_flush = 0;
    // pre-split operand scratch of the tensor-core flush (FP32 delayed
    // modes): the flush runs in waves of ps_wave chains
    unsigned char* ps = nullptr;
    int ps_wave = 0;
    size_t ps_bytes = 0;
    unsigned long long block_moves = 0;      // learned-proposal moves made (Philox counter)
    // one sweep captured as a CUDA graph (opts.graph != 0)
    unsigned long long* d_sweep = nullptr;   // device copy of the sweep counter
    double* d_obs_stage = nullptr;           // [n][GGF_N_OBS] observables of the last sweep
    cudaStream_t cs = nullptr;               // library stream the graph runs on
    cudaEvent_t join = nullptr;              // stream-join event
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    unsigned long long graph_launches = 0;   // kernels per replay
    // the same sweep captured with timing-event record nodes around its launch
    // groups (per-kernel timing on, ggf_profile): events ev[0 .. gev_n) of the
    // context's pool and their (category, start, end) triples
    cudaGraph_t graph_t = nullptr;
    cudaGraphExec_t gexec_t = nullptr;
    std::vector<int> gev_cat;
    int gev_n = 0;
};

struct ggf_net;

struct ggf_ctx {
    int device = 0;
    std::string err;
    Geometry g;
    bool have_lattice = false, have_group = false, have_gauss = false;
    bool use_tc = true;        // FP32 delayed flush on tcgen05 tensor cores
    int* d_err = nullptr;      // device error word (bounded waits that ran out)
    int K = 0, P = 0, Kc = 0;
    std::vector<int> pair_n, pair_m;
    std::vector<cxd> logc, w;
    double* d_D = nullptr;
    double* d_Ap = nullptr;
    double* d_Bp = nullptr;
    double* d_Gr = nullptr;
    cxd* d_Gc = nullptr;
    cxd* d_logc = nullptr;
    cxd* d_w = nullptr;
    Chains ch;
    void* work = nullptr;
    size_t work_bytes = 0;
    // site-by-site Pfaffian (k_front.cu): schedule [slot N | eoff V+1 | elim N]
    // for the lattice it was built for, and a global front workspace for
    // fronts too large for shared memory
    int* d_front = nullptr;
    int front_F = 0, front_L = -1, front_B = -1;
    void* front_ws = nullptr;
    size_t front_ws_bytes = 0;
    // refresh bookkeeping since ggf_chains_init: largest Newton residual
    // |I - M W| seen, chains refreshed by dense Gauss-Jordan instead, and
    // Pfaffian items that fell back to the dense elimination
    double refine_rmax = 0.0;
    unsigned long long dense_refreshes = 0, dense_pfaffians = 0, refine_steps = 0;
    // event timing (ggf_profile)
    bool prof = false;
    std::vector<cudaEvent_t> ev;            // event pool
    std::vector<int> ev_cat;                // category of each recorded (start, end) pair
    int ev_used = 0;                        // events recorded this sweep
    bool capturing = false;                 // a sweep is being captured into a graph
    double kt_ms[GGF_KT_N] = {0, 0, 0, 0, 0, 0};
    unsigned long long kt_n[GGF_KT_N] = {0, 0, 0, 0, 0, 0};
    // record one event (returns its index, or -1 when profiling is off)
    int prof_mark(cudaStream_t st) {
        if (!prof) return -1;
        if (ev_used == (int)ev.size()) {
            if (capturing) return -1;    // the pool is grown before a capture
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return -1;
            ev.push_back(e);
        }
        // inside a capture the record becomes an event-record node of the graph
        cudaEventRecordWithFlags(ev[ev_used], st, capturing ? cudaEventRecordExternal : cudaEventRecordDefault);
        return ev_used++;
    }
    void prof_pair(int cat, int a, int b) {
        if (a < 0 || b < 0) return;
        ev_cat.push_back(cat); ev_cat.push_back(a); ev_cat.push_back(b);
    }
    unsigned long long launches = 0;   // kernels launched by ggf_sample
    int n_sms = 0;
    DevConst dc() const {
        DevConst c;
        c.g = g; c.K = K; c.P = P; c.Kc = Kc;
        c.D = d_D; c.Ap = d_Ap; c.Bp = d_Bp; c.Gr = d_Gr; c.Gc = d_Gc; c.logc = d_logc; c.w = d_w;
        return c;
    }
};

// NVTX range for the lifetime of a scope (a no-op unless a profiler is attached)
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// status helpers
ggf_status ggf_fail(ggf_ctx* ctx, ggf_status st, const std::string& msg);
ggf_status ggf_cuda(ggf_ctx* ctx, cudaError_t e, const char* what);
#define GGF_CK(call)                                                      \
    do {                                                                  \
        cudaError_t _e = (call);                                          \
        if (_e != cudaSuccess) return ggf_cuda(ctx, _e, #call);           \
    } while (0)
#define GGF_TRY(call)                                                     \
    do {                                                                  \
        ggf_status _s = (call);                                           \
        if (_s != GGF_OK) return _s;                                      \
    } while (0)

ggf_status ggf_workspace(ggf_ctx* ctx, size_t bytes);
void ggf_free_chains(ggf_ctx* ctx);
void ggf_free_consts(ggf_ctx* ctx);

// host init (ggf_init.cu)
ggf_status ggf_build_constants(ggf_ctx* ctx, const double* gamma_site, int K,
                               const double* gamma_bond, const double* lambda);

// linear algebra drivers (k_linalg.cu)
// Assemble FP64 M for items (cfg index, pair index) into dst (item-major, N*N each).
// real_family: pairs 0..K-1 (double) else complex pairs (cxd).
ggf_status ggf_assemble(ggf_ctx* ctx, bool real_family, int n_items, const int* d_item_cfg,
                        const int* d_item_pair, const void* d_links, void* dst, cudaStream_t st);
// Batched Pfaffian (destroys A): out[item] = (log|Pf|, phase as unit cxd)
ggf_status ggf_pfaffian_batched(ggf_ctx* ctx, bool cplx, int n, int batch, void* A, cxd* d_logpf,
                                cxd* d_phase, void* d_tmp, cudaStream_t st);
// Batched Gauss-Jordan inverse in place: logdet (log|det|, arg) per item.
ggf_status ggf_invert_batched(ggf_ctx* ctx, bool cplx, int n, int batch, void* A, cxd* d_logdet,
                              void* d_tmp, cudaStream_t st);
// log Pf(M_nm(G)) by site-by-site elimination along the lattice (FP64):
// (log|Pf|, 0) and the unit phase per item; flag[item] = 1 where no pivot was
// usable inside a closed set (refactor those items densely).
ggf_status ggf_front_pfaffian(ggf_ctx* ctx, bool cplx, int n_items, const int* d_item_cfg, const int* d_item_pair,
                              const void* d_links, cxd* d_logpf, cxd* d_phase, int* d_flag, cudaStream_t st);
void ggf_front_free(ggf_ctx* ctx);
// Combine per-config pair log-Pfaffians into log N (device, n_cfg items).
ggf_status ggf_combine(ggf_ctx* ctx, int n_cfg, const cxd* d_ell, double* d_logN, cudaStream_t st);
ggf_status ggf_plaquette(ggf_ctx* ctx, int n_cfg, const void* d_links, double* d_out, cudaStream_t st);
// Mean Wilson loops (mode 0: R x T rectangles; mode 1: loops winding along y).
ggf_status ggf_loops(ggf_ctx* ctx, int n_cfg, int R, int T, int mode, const void* d_links, double* d_out,
                     cudaStream_t st);
