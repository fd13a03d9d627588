// Batched dense kernels of libggf: assembly of M_nm(G) (Sec. 5), FP64
// Parlett-Reid Pfaffian and Gauss-Jordan inverse, combination of the pair
// terms into log N(G), plaquette Wilson loops (Sec. 2.3).
//
// The factorisations are right-looking and step-launched: every elimination
// step is one pivot launch (one CTA per matrix) plus one trailing-update
// launch whose grid covers the trailing block of every matrix in the batch,
// so a single large matrix still spreads over all SMs.
#include "ggf_ctx.h"
#include "ggf_geom.cuh"

namespace {

constexpr int TILE = 32;      // trailing-update tile (TILE x TILE per CTA)
constexpr int TROWS = 4;      // rows per thread (block 32 x 8)

struct PfAcc {
    double logabs;
    cxd phase;
    int singular;
    int pad;
};

template <class T>
__global__ void assemble_kernel(DevConst dc, const int* item_cfg, const int* item_pair, const void* links,
                                T* dst) {
    const Geometry& g = dc.g;
    const int item = blockIdx.y;
    const size_t NN = (size_t)g.N * g.N;
    size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= NN) return;
    int i = (int)(e / g.N), j = (int)(e - (size_t)i * g.N);
    dst[(size_t)item * NN + e] = assemble_elem<T>(dc, links, item_cfg[item], item_pair[item], i, j);
}

// ---- block reductions -----------------------------------------------------------
__device__ __forceinline__ void argmax_block(double v, int idx, double* sv, int* si, double& bv, int& bi) {
    for (int o = 16; o > 0; o >>= 1) {
        double ov = __shfl_down_sync(0xffffffffu, v, o);
        int oi = __shfl_down_sync(0xffffffffu, idx, o);
        if (ov > v || (ov == v && oi < idx)) { v = ov; idx = oi; }
    }
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { sv[w] = v; si[w] = idx; }
    __syncthreads();
    if (threadIdx.x == 0) {
        int nw = blockDim.x >> 5;
        bv = sv[0]; bi = si[0];
        for (int k = 1; k < nw; ++k)
            if (sv[k] > bv || (sv[k] == bv && si[k] < bi)) { bv = sv[k]; bi = si[k]; }
        sv[0] = bv; si[0] = bi;
    }
    __syncthreads();
    bv = sv[0]; bi = si[0];
}

__device__ __forceinline__ double mag(double v) { return fabs(v); }
__device__ __forceinline__ double mag(cxd v) { return hypot(v.x, v.y); }
__device__ __forceinline__ cxd unit(double v) { return {v >= 0 ? 1.0 : -1.0, 0.0}; }
__device__ __forceinline__ cxd unit(cxd v) { double m = hypot(v.x, v.y); return {v.x / m, v.y / m}; }
__device__ __forceinline__ double divs(double a, double b) { return a / b; }
__device__ __forceinline__ cxd divs(cxd a, cxd b) { return a / b; }

// ---- Pfaffian --------------------------------------------------------------------
template <class T>
__global__ void pf_pivot(T* A, int n, int k, T* tv, T* cv, PfAcc* acc) {
    __shared__ double sv[32];
    __shared__ int si[32];
    const int b = blockIdx.x;
    T* M = A + (size_t)b * n * n;
    T* t = tv + (size_t)b * n;
    T* c = cv + (size_t)b * n;
    if (acc[b].singular) return;
    double best = -1.0;
    int bi = k + 1;
    for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) {
        double m = mag(M[(size_t)i * n + k]);
        if (m > best) { best = m; bi = i; }
    }
    double bv;
    int p;
    argmax_block(best, bi, sv, si, bv, p);
    const int q = k + 1;
    if (p != q) {
        for (int j = k + threadIdx.x; j < n; j += blockDim.x) {
            T tmp = M[(size_t)q * n + j];
            M[(size_t)q * n + j] = M[(size_t)p * n + j];
            M[(size_t)p * n + j] = tmp;
        }
        __syncthreads();
        for (int i = k + threadIdx.x; i < n; i += blockDim.x) {
            T tmp = M[(size_t)i * n + q];
            M[(size_t)i * n + q] = M[(size_t)i * n + p];
            M[(size_t)i * n + p] = tmp;
        }
    }
    __syncthreads();
    T piv = M[(size_t)q * n + k];
    if (mag(piv) == 0.0) {
        if (threadIdx.x == 0) acc[b].singular = 1;
        return;
    }
    if (threadIdx.x == 0) {
        T akk1 = M[(size_t)k * n + q];
        acc[b].logabs += log(mag(akk1));
        cxd ph = acc[b].phase * unit(akk1);
        if (p != q) ph = -ph;
        acc[b].phase = ph;
    }
    for (int i = k + 2 + threadIdx.x; i < n; i += blockDim.x) {
        t[i] = divs(M[(size_t)i * n + k], piv);
        c[i] = M[(size_t)i * n + q];
    }
}

template <class T>
__global__ void pf_update(T* A, int n, int k, const T* tv, const T* cv, const PfAcc* acc, int tiles_x) {
    const int b = blockIdx.y;
    if (acc[b].singular) return;
    const int ty = blockIdx.x / tiles_x, tx = blockIdx.x - ty * tiles_x;
    const int j = k + 2 + tx * TILE + threadIdx.x;
    if (j >= n) return;
    T* M = A + (size_t)b * n * n;
    const T* t = tv + (size_t)b * n;
    const T* c = cv + (size_t)b * n;
    T tj = t[j], cj = c[j];
#pragma unroll
    for (int rr = 0; rr < TROWS; ++rr) {
        int i = k + 2 + ty * TILE + threadIdx.y + rr * 8;
        if (i < n) M[(size_t)i * n + j] += t[i] * cj - c[i] * tj;
    }
}

template <class T>
__global__ void pf_finish(const PfAcc* acc, cxd* logpf, cxd* phase, int batch) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= batch) return;
    if (acc[b].singular) {
        logpf[b] = {-INFINITY, 0.0};
        phase[b] = {0.0, 0.0};
    } else {
        logpf[b] = {acc[b].logabs, 0.0};
        phase[b] = acc[b].phase;
    }
}

__global__ void acc_init(PfAcc* acc, int batch) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < batch) { acc[b].logabs = 0.0; acc[b].phase = {1.0, 0.0}; acc[b].singular = 0; }
}

// ---- Gauss-Jordan inverse -----------------------------------------------------------
template <class T>
__global__ void gj_pivot(T* A, int n, int k, T* colk, int* piv, PfAcc* acc) {
    __shared__ double sv[32];
    __shared__ int si[32];
    const int b = blockIdx.x;
    if (acc[b].singular) return;
    T* M = A + (size_t)b * n * n;
    T* col = colk + (size_t)b * n;
    double best = -1.0;
    int bi = k;
    for (int i = k + threadIdx.x; i < n; i += blockDim.x) {
        double m = mag(M[(size_t)i * n + k]);
        if (m > best) { best = m; bi = i; }
    }
    double bv;
    int p;
    argmax_block(best, bi, sv, si, bv, p);
    if (p != k) {
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
            T tmp = M[(size_t)k * n + j];
            M[(size_t)k * n + j] = M[(size_t)p * n + j];
            M[(size_t)p * n + j] = tmp;
        }
    }
    __syncthreads();
    T d = M[(size_t)k * n + k];
    if (mag(d) == 0.0) {
        if (threadIdx.x == 0) acc[b].singular = 1;
        return;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) col[i] = (i == k) ? Sc<T>::zero() : M[(size_t)i * n + k];
    T one = Sc<T>::one();
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        T v = (j == k) ? one : M[(size_t)k * n + j];
        M[(size_t)k * n + j] = divs(v, d);
    }
    if (threadIdx.x == 0) {
        acc[b].logabs += log(mag(d));
        cxd ph = acc[b].phase * unit(d);
        if (p != k) ph = -ph;
        acc[b].phase = ph;
        piv[(size_t)b * n + k] = p;
    }
}

template <class T>
__global__ void gj_update(T* A, int n, int k, const T* colk, const PfAcc* acc, int tiles_x) {
    const int b = blockIdx.y;
    if (acc[b].singular) return;
    const int ty = blockIdx.x / tiles_x, tx = blockIdx.x - ty * tiles_x;
    const int j = tx * TILE + threadIdx.x;
    if (j >= n) return;
    T* M = A + (size_t)b * n * n;
    const T* col = colk + (size_t)b * n;
    T rk = M[(size_t)k * n + j];
#pragma unroll
    for (int rr = 0; rr < TROWS; ++rr) {
        int i = ty * TILE + threadIdx.y + rr * 8;
        if (i < n && i != k) {
            T a = (j == k) ? Sc<T>::zero() : M[(size_t)i * n + j];
            M[(size_t)i * n + j] = a - col[i] * rk;
        }
    }
}

template <class T>
__global__ void gj_unpivot(T* A, int n, const int* piv, const PfAcc* acc) {
    const int b = blockIdx.y;
    if (acc[b].singular) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    T* row = A + (size_t)b * n * n + (size_t)i * n;
    const int* pv = piv + (size_t)b * n;
    for (int k = n - 1; k >= 0; --k) {
        int p = pv[k];
        if (p != k) { T t = row[k]; row[k] = row[p]; row[p] = t; }
    }
}

template <class T>
__global__ void gj_finish(const PfAcc* acc, cxd* logdet, int batch) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= batch) return;
    if (acc[b].singular) logdet[b] = {-INFINITY, 0.0};
    else logdet[b] = {acc[b].logabs, atan2(acc[b].phase.y, acc[b].phase.x)};
}

// ---- combine and plaquettes --------------------------------------------------------
__global__ void combine_kernel(DevConst dc, int n_cfg, const cxd* ell, double* logN) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_cfg) return;
    double amax = -INFINITY;
    for (int p = 0; p < dc.P; ++p) {
        double a = dc.logc[p].x + ell[(size_t)c * dc.P + p].x;
        amax = fmax(amax, a);
    }
    if (!isfinite(amax)) { logN[c] = -INFINITY; return; }
    double s = 0.0;
    for (int p = 0; p < dc.P; ++p) {
        cxd a = dc.logc[p] + ell[(size_t)c * dc.P + p];
        if (p < dc.K) a.y = 0.0;
        a.x -= amax;
        cxd t = dc.w[p] * cexp_(a);
        s += t.x;
    }
    logN[c] = s > 0.0 ? amax + log(s) : -INFINITY;
}

__global__ void plaquette_kernel(Geometry g, int n_cfg, const void* links, double* out) {
    __shared__ double red[256];
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
    if (threadIdx.x == 0) out[c] = red[0] / g.V;
}

// Mean of loop_value over the loop positions (mode 0: the V corners of R x T
// rectangles; mode 1: the L winding loops); one block per configuration.
__global__ void loop_kernel(Geometry g, int n_cfg, int R, int T, int mode, const void* links, double* out) {
    __shared__ double red[256];
    const int c = blockIdx.x;
    const int items = mode ? g.L : g.V;
    double acc = 0.0;
    for (int s = threadIdx.x; s < items; s += blockDim.x) acc += loop_value(g, links, c, s, R, T, mode);
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[c] = red[0] / items;
}

template <class T>
ggf_status run_pfaffian(ggf_ctx* ctx, int n, int batch, T* A, cxd* logpf, cxd* phase, void* tmp,
                        cudaStream_t st) {
    T* tv = (T*)tmp;
    T* cv = tv + (size_t)batch * n;
    PfAcc* acc = (PfAcc*)(cv + (size_t)batch * n);
    acc_init<<<(batch + 127) / 128, 128, 0, st>>>(acc, batch);
    ctx->launches += 2 + (n / 2) + (n / 2 - 1);
    for (int k = 0; k < n - 1; k += 2) {
        pf_pivot<T><<<batch, 256, 0, st>>>(A, n, k, tv, cv, acc);
        int m = n - k - 2;
        if (m > 0) {
            int tiles = (m + TILE - 1) / TILE;
            dim3 grid(tiles * tiles, batch);
            pf_update<T><<<grid, dim3(32, 8), 0, st>>>(A, n, k, tv, cv, acc, tiles);
        }
    }
    pf_finish<T><<<(batch + 127) / 128, 128, 0, st>>>(acc, logpf, phase, batch);
    GGF_CK(cudaGetLastError());
    return GGF_OK;
}

template <class T>
ggf_status run_invert(ggf_ctx* ctx, int n, int batch, T* A, cxd* logdet, void* tmp, cudaStream_t st) {
    T* col = (T*)tmp;
    int* piv = (int*)(col + (size_t)batch * n);
    PfAcc* acc = (PfAcc*)(piv + (size_t)batch * n + ((size_t)batch * n) % 2);
    acc_init<<<(batch + 127) / 128, 128, 0, st>>>(acc, batch);
    ctx->launches += 3 + 2 * (unsigned long long)n;
    int tiles = (n + TILE - 1) / TILE;
    for (int k = 0; k < n; ++k) {
        gj_pivot<T><<<batch, 256, 0, st>>>(A, n, k, col, piv, acc);
        gj_update<T><<<dim3(tiles * tiles, batch), dim3(32, 8), 0, st>>>(A, n, k, col, acc, tiles);
    }
    gj_unpivot<T><<<dim3((n + 127) / 128, batch), 128, 0, st>>>(A, n, piv, acc);
    gj_finish<T><<<(batch + 127) / 128, 128, 0, st>>>(acc, logdet, batch);
    GGF_CK(cudaGetLastError());
    return GGF_OK;
}

}  // namespace

size_t ggf_factor_tmp_bytes(int n, int batch) {
    // max of Pfaffian (2 vectors) and GJ (vector + pivots) scratch, complex slots
    return (size_t)batch * n * 2 * sizeof(cxd) + (size_t)batch * sizeof(PfAcc) + 64;
}

ggf_status ggf_assemble(ggf_ctx* ctx, bool real_family, int n_items, const int* d_item_cfg,
                        const int* d_item_pair, const void* d_links, void* dst, cudaStream_t st) {
    if (n_items == 0) return GGF_OK;
    size_t NN = (size_t)ctx->g.N * ctx->g.N;
    dim3 grid((unsigned)((NN + 255) / 256), n_items);
    ctx->launches += 1;
    if (real_family)
        assemble_kernel<double><<<grid, 256, 0, st>>>(ctx->dc(), d_item_cfg, d_item_pair, d_links, (double*)dst);
    else
        assemble_kernel<cxd><<<grid, 256, 0, st>>>(ctx->dc(), d_item_cfg, d_item_pair, d_links, (cxd*)dst);
    GGF_CK(cudaGetLastError());
    return GGF_OK;
}

ggf_status ggf_pfaffian_batched(ggf_ctx* ctx, bool cplx, int n, int batch, void* A, cxd* d_logpf,
                                cxd* d_phase, void* d_tmp, cudaStream_t st) {
    if (batch == 0) return GGF_OK;
    if (cplx) return run_pfaffian<cxd>(ctx, n, batch, (cxd*)A, d_logpf, d_phase, d_tmp, st);
    return run_pfaffian<double>(ctx, n, batch, (double*)A, d_logpf, d_phase, d_tmp, st);
}

ggf_status ggf_invert_batched(ggf_ctx* ctx, bool cplx, int n, int batch, void* A, cxd* d_logdet,
                              void* d_tmp, cudaStream_t st) {
    if (batch == 0) return GGF_OK;
    if (cplx) return run_invert<cxd>(ctx, n, batch, (cxd*)A, d_logdet, d_tmp, st);
    return run_invert<double>(ctx, n, batch, (double*)A, d_logdet, d_tmp, st);
}

ggf_status ggf_combine(ggf_ctx* ctx, int n_cfg, const cxd* d_ell, double* d_logN, cudaStream_t st) {
    if (n_cfg == 0) return GGF_OK;
    combine_kernel<<<(n_cfg + 127) / 128, 128, 0, st>>>(ctx->dc(), n_cfg, d_ell, d_logN);
    GGF_CK(cudaGetLastError());
    return GGF_OK;
}

ggf_status ggf_loops(ggf_ctx* ctx, int n_cfg, int R, int T, int mode, const void* d_links, double* d_out,
                     cudaStream_t st) {
    loop_kernel<<<n_cfg, 256, 0, st>>>(ctx->g, n_cfg, R, T, mode, d_links, d_out);
    GGF_CK(cudaGetLastError());
    return GGF_OK;
}

ggf_status ggf_plaquette(ggf_ctx* ctx, int n_cfg, const void* d_links, double* d_out, cudaStream_t st) {
    if (n_cfg == 0) return GGF_OK;
    plaquette_kernel<<<n_cfg, 256, 0, st>>>(ctx->g, n_cfg, d_links, d_out);
    GGF_CK(cudaGetLastError());
    return GGF_OK;
}
