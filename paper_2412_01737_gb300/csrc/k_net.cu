// Learned block proposal: the convolutional network, its training and the
// proposal/density of block moves (BF16 activations and weights, FP32
// accumulation; FP32 master weights with Adam).
//
// Network (same convention as the FP64 reference): per site of the L x L
// torus 8 input channels (cos, sin of the x-link and y-link angles; cos, sin
// of the plaquette angle theta1 + theta2 - theta3 - theta4; block flags for the
// two links), with the block's link angles and the plaquettes that contain a
// block link zeroed, so the proposal depends only on the boundary.  Block:
// the 4 x 4 sites from origin (bx, by), its 32 links are the x- and y-links
// whose source site lies in it, ordered site row-major, x then y.  Layers:
// 3 x 3 circular convolutions 8 -> 64 -> 64 -> 64 -> 6, ReLU after the first
// three.  Head per site (a_x, b_x, z_x, a_y, b_y, z_y): mu = atan2(b, a),
// rho = 0.95 sigmoid(z); proposal density the wrapped Cauchy
// f(t) = (1 - rho^2) / (2 pi (1 + rho^2 - 2 rho cos(t - mu))), sampled as
// t = mu - log(rho) tan(pi (u - 1/2)) wrapped into [0, 2 pi).
#include <cuda_bf16.h>
#include <cstring>
#include <vector>
#include "ggf_ctx.h"
#include "ggf_net.h"

ggf_status ggf_conv_fwd_tc(int n, int L, int ci, int co, bool relu, const void* X, const void* W, const float* bias,
                           void* Y, bool out_f32, int* err, int sms, cudaStream_t st);
ggf_status ggf_conv_bwd_data_tc(int n, int L, int ci, int co, const void* W, const float* dY, const void* act,
                                float* dX, int* err, int sms, cudaStream_t st);
ggf_status ggf_conv_bwd_weight_tc(int n, int L, int ci, int co, const void* X, const float* dY, float* dW,
                                  float* db, int* err, int sms, cudaStream_t st);

namespace {

constexpr int C_IN = 8, CH = 64, C_OUT = 6, BLK = 4;
constexpr float RHO_MAX = 0.95f;
constexpr int NLAYER = 4;
__host__ __device__ constexpr int layer_ci(int l) { return l == 0 ? C_IN : CH; }
__host__ __device__ constexpr int layer_co(int l) { return l == NLAYER - 1 ? C_OUT : CH; }
__host__ __device__ constexpr int layer_off(int l) {
    return l == 0 ? 0 : layer_off(l - 1) + layer_co(l - 1) * layer_ci(l - 1) * 9 + layer_co(l - 1);
}
constexpr int NPARAM = layer_off(NLAYER);
static_assert(NPARAM == GGF_NET_PARAMS, "parameter count");

typedef __nv_bfloat16 bf16;

__device__ __forceinline__ int block_link(int L, int bx, int by, int k, int* site) {
    // k = 2 * (j * 4 + i) + d
    int d = k & 1, q = k >> 1, i = q & 3, j = q >> 2;
    int s = ((by + j) % L) * L + (bx + i) % L;
    if (site) *site = s;
    return 2 * s + d;
}

__device__ __forceinline__ bool in_block(int L, int bx, int by, int s) {
    int x = s % L, y = s / L;
    int dx = (x - bx + L) % L, dy = (y - by + L) % L;
    return dx < BLK && dy < BLK;
}

// X[b][c][s] (bf16) for n samples: angles theta[cfg[b]] (or b), block origin blocks[b]
__global__ void features_kernel(int n, int L, const double* theta, const int* cfg, const int* blocks, bf16* X) {
    const int b = blockIdx.x;
    if (b >= n) return;
    const int V = L * L, nl = 2 * V;
    const double* th = theta + (size_t)(cfg ? cfg[b] : b) * nl;
    const int bx = blocks[2 * b], by = blocks[2 * b + 1];
    bf16* Xb = X + (size_t)b * C_IN * V;
    for (int s = threadIdx.x; s < V; s += blockDim.x) {
        int x = s % L, y = s / L;
        int sx = y * L + (x + 1) % L, sy = ((y + 1) % L) * L + x;
        bool bs = in_block(L, bx, by, s);
        bool bsx = in_block(L, bx, by, sx), bsy = in_block(L, bx, by, sy);
        float v[C_IN] = {0, 0, 0, 0, 0, 0, 0, 0};
        if (!bs) {
            v[0] = (float)cos(th[2 * s]); v[1] = (float)sin(th[2 * s]);
            v[2] = (float)cos(th[2 * s + 1]); v[3] = (float)sin(th[2 * s + 1]);
        }
        // plaquette links: (s, x), (sx, y), (sy, x), (s, y); a link is in the block iff its source site is
        if (!bs && !bsx && !bsy) {
            double a = th[2 * s] + th[2 * sx + 1] - th[2 * sy] - th[2 * s + 1];
            v[4] = (float)cos(a); v[5] = (float)sin(a);
        }
        v[6] = bs ? 1.f : 0.f;
        v[7] = bs ? 1.f : 0.f;
#pragma unroll
        for (int c = 0; c < C_IN; ++c) Xb[(size_t)c * V + s] = __float2bfloat16(v[c]);
    }
}

// Head: per sample the 32 block links.  mode 0: log q of theta's block links
// into logq[b]; mode 1: loss (sum -log f / n into loss[0] atomically) and dOut;
// mode 2 (proposal): draw new angles into prop[b][32], log q(new) - log q(old)
// into logq[b].
__global__ void head_kernel(int n, int L, int mode, const float* out, const double* theta, const int* cfg,
                            const int* blocks, double* logq, float* dOut, double* loss, double* prop,
                            uint64_t seed, uint64_t counter, uint64_t koff) {
    const int b = blockIdx.x;
    if (b >= n) return;
    const int V = L * L, nl = 2 * V;
    const double* th = theta + (size_t)(cfg ? cfg[b] : b) * nl;
    const int bx = blocks[2 * b], by = blocks[2 * b + 1];
    const float* ob = out + (size_t)b * C_OUT * V;
    __shared__ double red[32];
    double lsum = 0.0;
    const int k = threadIdx.x;            // 32 threads, one block link each
    if (k < 32) {
        int s;
        int l = block_link(L, bx, by, k, &s);
        int d = k & 1;
        double a = ob[(3 * d) * V + s], bb = ob[(3 * d + 1) * V + s], z = ob[(3 * d + 2) * V + s];
        double sig = 1.0 / (1.0 + exp(-z));
        double rho = RHO_MAX * sig;
        double mu = atan2(bb, a);
        double t_old = th[l];
        auto logf = [&](double t) {
            return log1p(-rho * rho) - log(GGF_TWO_PI) - log(1.0 + rho * rho - 2.0 * rho * cos(t - mu));
        };
        if (mode == 0) {
            lsum = logf(t_old);
        } else if (mode == 1) {
            double D = 1.0 + rho * rho - 2.0 * rho * cos(t_old - mu);
            lsum = -logf(t_old);
            double dmu = 2.0 * rho * sin(t_old - mu) / D;
            double drho = -2.0 * rho / (1.0 - rho * rho) - (2.0 * rho - 2.0 * cos(t_old - mu)) / D;
            double r2 = a * a + bb * bb;
            float* db_ = dOut + (size_t)b * C_OUT * V;
            db_[(3 * d) * V + s] = (float)(-(dmu * (-bb / r2)) / n);
            db_[(3 * d + 1) * V + s] = (float)(-(dmu * (a / r2)) / n);
            db_[(3 * d + 2) * V + s] = (float)(-(drho * RHO_MAX * sig * (1.0 - sig)) / n);
        } else {
            uint64_t c4[4] = {counter, (uint64_t)k, 7, 0}, o4[4];
            philox4x64_10(c4, seed, koff + (uint64_t)b, o4);
            double u = u53(o4[0]);
            double t = mu - log(rho) * tan(M_PI * (u - 0.5));
            t = fmod(t, GGF_TWO_PI);
            if (t < 0.0) t += GGF_TWO_PI;
            if (t >= GGF_TWO_PI) t -= GGF_TWO_PI;
            prop[(size_t)b * 32 + k] = t;
            lsum = logf(t) - logf(t_old);
        }
    }
    red[k] = lsum;
    __syncwarp();
    if (k == 0) {
        double sm_ = 0.0;
        for (int q = 0; q < 32; ++q) sm_ += red[q];
        if (mode == 0 || mode == 2) logq[b] = sm_;
        else atomicAdd(loss, sm_ / n);
    }
}

__global__ void to_bf16(int n, const float* a, bf16* b) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = __float2bfloat16(a[i]);
}

__global__ void adam_kernel(int n, float* p, const float* g, float* m, float* v, float lr, float b1, float b2,
                            float eps, float c1, float c2, bf16* pb) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float gi = g[i];
    float mi = b1 * m[i] + (1.f - b1) * gi;
    float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = pi;
    pb[i] = __float2bfloat16(pi);
}

__global__ void init_params(float* p, uint64_t seed) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NPARAM) return;
    int l = 0;
    while (l + 1 < NLAYER && i >= layer_off(l + 1)) ++l;
    int rel = i - layer_off(l);
    int nw = layer_co(l) * layer_ci(l) * 9;
    if (rel >= nw) { p[i] = 0.f; return; }           // biases
    uint64_t c4[4] = {(uint64_t)i, 11, 0, 0}, o4[4];
    philox4x64_10(c4, seed, 0x6e6574, o4);
    float bound = sqrtf(6.f / (layer_ci(l) * 9));      // He-uniform for ReLU layers
    if (l == NLAYER - 1) bound *= 0.1f;                // near-flat initial proposal
    p[i] = (float)((u53(o4[0]) * 2.0 - 1.0) * bound);
}

// minibatch: configuration index and block origin per sample from Philox
__global__ void draw_batch(int n, int n_cfg, int L, uint64_t seed, uint64_t step, int* cfg, int* blocks) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n) return;
    uint64_t c4[4] = {step, (uint64_t)b, 13, 0}, o4[4];
    philox4x64_10(c4, seed, 0x747261696e, o4);
    cfg[b] = min(n_cfg - 1, (int)(u53(o4[0]) * n_cfg));
    blocks[2 * b] = min(L - 1, (int)(u53(o4[1]) * L));
    blocks[2 * b + 1] = min(L - 1, (int)(u53(o4[2]) * L));
}

}  // namespace

struct ggf_net {
    int device = 0, L = 0;
    uint64_t seed = 0;
    std::string err;
    float* p = nullptr;        // FP32 master parameters
    bf16* pb = nullptr;        // BF16 copy used by the kernels
    float* g = nullptr;        // gradient
    float* m = nullptr;
    float* v = nullptr;
    long long t = 0;           // Adam steps
    int cap = 0;               // batch capacity of the workspace
    bf16* X[NLAYER] = {nullptr, nullptr, nullptr, nullptr};   // layer inputs (post-ReLU)
    float* out = nullptr;      // head outputs
    float* dA = nullptr;       // gradient buffers (ping-pong)
    float* dB = nullptr;
    int* cfg = nullptr;
    int* blocks = nullptr;
    double* scal = nullptr;    // loss accumulator
    int* d_err = nullptr;      // raised by a tensor-core convolution whose bounded wait ran out
    int sms = 0;               // streaming multiprocessors of the device
};

static ggf_status net_fail(ggf_net* n, ggf_status st, const std::string& m) {
    if (n) n->err = m;
    return st;
}
#define NET_CK(call)                                                                   \
    do {                                                                               \
        cudaError_t _e = (call);                                                       \
        if (_e != cudaSuccess) return net_fail(net, _e == cudaErrorMemoryAllocation ? GGF_ENOMEM : GGF_ECUDA, \
                                               std::string(#call) + ": " + cudaGetErrorString(_e)); \
    } while (0)

static void net_free_ws(ggf_net* net) {
    for (auto& x : net->X) { if (x) cudaFree(x); x = nullptr; }
    void* ps[] = {net->out, net->dA, net->dB, net->cfg, net->blocks, net->scal};
    for (void* q : ps) if (q) cudaFree(q);
    net->out = nullptr; net->dA = net->dB = nullptr; net->cfg = nullptr; net->blocks = nullptr; net->scal = nullptr;
    net->cap = 0;
}

static ggf_status net_ws(ggf_net* net, int n) {
    if (n <= net->cap) return GGF_OK;
    net_free_ws(net);
    const size_t V = (size_t)net->L * net->L;
    for (int l = 0; l < NLAYER; ++l) NET_CK(cudaMalloc(&net->X[l], (size_t)n * layer_ci(l) * V * sizeof(bf16)));
    NET_CK(cudaMalloc(&net->out, (size_t)n * C_OUT * V * sizeof(float)));
    NET_CK(cudaMalloc(&net->dA, (size_t)n * CH * V * sizeof(float)));
    NET_CK(cudaMalloc(&net->dB, (size_t)n * CH * V * sizeof(float)));
    NET_CK(cudaMalloc(&net->cfg, (size_t)n * sizeof(int)));
    NET_CK(cudaMalloc(&net->blocks, (size_t)n * 2 * sizeof(int)));
    NET_CK(cudaMalloc(&net->scal, 4 * sizeof(double)));
    net->cap = n;
    return GGF_OK;
}

static int px_threads(int L) { return L * L >= 256 ? 256 : ((L * L + 31) / 32) * 32; }

// forward pass for n samples whose inputs are already in X[0]; head to net->out
ggf_status ggf_net_forward(ggf_net* net, int n, cudaStream_t st) {
    const int L = net->L;
    for (int l = 0; l < NLAYER; ++l) {
        const int ci = layer_ci(l), co = layer_co(l);
        const bf16* W = net->pb + layer_off(l);
        const float* b = net->p + layer_off(l) + co * ci * 9;
        const bool last = l == NLAYER - 1;
        ggf_status rc = ggf_conv_fwd_tc(n, L, ci, co, !last, net->X[l], W, b, last ? (void*)net->out : (void*)net->X[l + 1],
                                        last, net->d_err, net->sms, st);
        if (rc != GGF_OK) return net_fail(net, rc, "tensor-core convolution (forward) failed to launch");
    }
    return GGF_OK;
}

static ggf_status net_backward(ggf_net* net, int n, cudaStream_t st) {
    const int L = net->L;
    float* dcur = net->dA;      // gradient w.r.t. the current layer's output
    float* dnext = net->dB;
    for (int l = NLAYER - 1; l >= 0; --l) {
        const int ci = layer_ci(l), co = layer_co(l);
        float* dW = net->g + layer_off(l);
        float* db = dW + co * ci * 9;
        ggf_status rc = ggf_conv_bwd_weight_tc(n, L, ci, co, net->X[l], dcur, dW, db, net->d_err, net->sms, st);
        if (rc != GGF_OK) return net_fail(net, rc, "tensor-core convolution (weight gradient) failed to launch");
        if (l > 0) {
            rc = ggf_conv_bwd_data_tc(n, L, ci, co, net->pb + layer_off(l), dcur, net->X[l], dnext, net->d_err,
                                      net->sms, st);
            if (rc != GGF_OK) return net_fail(net, rc, "tensor-core convolution (input gradient) failed to launch");
            std::swap(dcur, dnext);
        }
    }
    return GGF_OK;
}

// log q / loss+grad / proposal for n samples (theta on the device)
ggf_status ggf_net_head(ggf_net* net, int n, int mode, const double* theta, const int* cfg, const int* blocks,
                        double* logq, double* prop, uint64_t seed, uint64_t counter, cudaStream_t st,
                        uint64_t koff) {
    GGF_TRY(net_ws(net, n));
    const int L = net->L, V = L * L;
    features_kernel<<<n, px_threads(L), 0, st>>>(n, L, theta, cfg, blocks, net->X[0]);
    NET_CK(cudaGetLastError());
    GGF_TRY(ggf_net_forward(net, n, st));
    if (mode == 1) {
        NET_CK(cudaMemsetAsync(net->dA, 0, (size_t)n * C_OUT * V * sizeof(float), st));
        NET_CK(cudaMemsetAsync(net->scal, 0, sizeof(double), st));
    }
    head_kernel<<<n, 32, 0, st>>>(n, L, mode, net->out, theta, cfg, blocks, logq, net->dA, net->scal, prop, seed,
                                  counter, koff);
    NET_CK(cudaGetLastError());
    if (mode == 1) GGF_TRY(net_backward(net, n, st));
    return GGF_OK;
}

int ggf_net_L(const ggf_net* net) { return net ? net->L : 0; }

// GGF_ETIMEOUT once a tensor-core convolution's bounded wait ran out
// (synchronises the device).
ggf_status ggf_net_check(ggf_net* net) {
    int h = 0;
    if (cudaDeviceSynchronize() != cudaSuccess || cudaMemcpy(&h, net->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return net_fail(net, GGF_ECUDA, "network error word unreadable");
    if (h) return net_fail(net, GGF_ETIMEOUT, "a tensor-core convolution's bounded wait ran out");
    return GGF_OK;
}

extern "C" {

ggf_status ggf_net_create(ggf_net** out, int device, int L, uint64_t seed) {
    if (!out) return GGF_EINVAL;
    *out = nullptr;
    if (L < BLK || L > 64) return GGF_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) return GGF_ECUDA;
    ggf_net* net = new ggf_net();
    net->device = device;
    net->L = L;
    net->seed = seed;
    ggf_status s = GGF_OK;
    auto ck = [&](cudaError_t e) { if (e != cudaSuccess && s == GGF_OK) s = GGF_ENOMEM; };
    ck(cudaMalloc(&net->p, NPARAM * sizeof(float)));
    ck(cudaMalloc(&net->pb, NPARAM * sizeof(bf16)));
    ck(cudaMalloc(&net->g, NPARAM * sizeof(float)));
    ck(cudaMalloc(&net->m, NPARAM * sizeof(float)));
    ck(cudaMalloc(&net->v, NPARAM * sizeof(float)));
    ck(cudaMalloc(&net->d_err, sizeof(int)));
    if (s != GGF_OK) { ggf_net_destroy(net); return s; }
    cudaMemset(net->d_err, 0, sizeof(int));
    cudaDeviceGetAttribute(&net->sms, cudaDevAttrMultiProcessorCount, device);
    init_params<<<(NPARAM + 255) / 256, 256>>>(net->p, seed);
    to_bf16<<<(NPARAM + 255) / 256, 256>>>(NPARAM, net->p, net->pb);
    cudaMemset(net->m, 0, NPARAM * sizeof(float));
    cudaMemset(net->v, 0, NPARAM * sizeof(float));
    if (cudaDeviceSynchronize() != cudaSuccess) { ggf_net_destroy(net); return GGF_ECUDA; }
    *out = net;
    return GGF_OK;
}

void ggf_net_destroy(ggf_net* net) {
    if (!net) return;
    cudaSetDevice(net->device);
    net_free_ws(net);
    void* ps[] = {net->p, net->pb, net->g, net->m, net->v, net->d_err};
    for (void* q : ps) if (q) cudaFree(q);
    delete net;
}

const char* ggf_net_last_error(const ggf_net* net) { return net ? net->err.c_str() : "null network"; }

ggf_status ggf_net_get_params(ggf_net* net, float* out) {
    if (!net || !out) return GGF_EINVAL;
    cudaSetDevice(net->device);
    NET_CK(cudaMemcpy(out, net->p, NPARAM * sizeof(float), cudaMemcpyDeviceToHost));
    return GGF_OK;
}

ggf_status ggf_net_set_params(ggf_net* net, const float* in) {
    if (!net || !in) return GGF_EINVAL;
    cudaSetDevice(net->device);
    NET_CK(cudaMemcpy(net->p, in, NPARAM * sizeof(float), cudaMemcpyHostToDevice));
    to_bf16<<<(NPARAM + 255) / 256, 256>>>(NPARAM, net->p, net->pb);
    NET_CK(cudaMemset(net->m, 0, NPARAM * sizeof(float)));
    NET_CK(cudaMemset(net->v, 0, NPARAM * sizeof(float)));
    net->t = 0;
    NET_CK(cudaDeviceSynchronize());
    return GGF_OK;
}

ggf_status ggf_net_logq(ggf_net* net, int n, const double* theta, const int* blocks, double* logq, int mem,
                        void* stream) {
    if (!net || n < 1 || !theta || !blocks || !logq) return GGF_EINVAL;
    cudaSetDevice(net->device);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t nl = 2 * (size_t)net->L * net->L;
    const double* dth = theta;
    const int* dbl = blocks;
    double* dlq = logq;
    void *t1 = nullptr, *t2 = nullptr, *t3 = nullptr;
    if (mem == GGF_MEM_HOST) {
        NET_CK(cudaMalloc(&t1, n * nl * sizeof(double)));
        NET_CK(cudaMalloc(&t2, n * 2 * sizeof(int)));
        NET_CK(cudaMalloc(&t3, n * sizeof(double)));
        NET_CK(cudaMemcpy(t1, theta, n * nl * sizeof(double), cudaMemcpyHostToDevice));
        NET_CK(cudaMemcpy(t2, blocks, n * 2 * sizeof(int), cudaMemcpyHostToDevice));
        dth = (const double*)t1; dbl = (const int*)t2; dlq = (double*)t3;
    }
    ggf_status s = ggf_net_head(net, n, 0, dth, nullptr, dbl, dlq, nullptr, 0, 0, st);
    if (s == GGF_OK && mem == GGF_MEM_HOST) {
        if (cudaMemcpy(logq, dlq, n * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) s = GGF_ECUDA;
    } else if (s == GGF_OK) {
        if (cudaStreamSynchronize(st) != cudaSuccess) s = GGF_ECUDA;
    }
    if (t1) cudaFree(t1);
    if (t2) cudaFree(t2);
    if (t3) cudaFree(t3);
    if (s == GGF_OK) s = ggf_net_check(net);
    return s;
}

ggf_status ggf_net_loss_grad(ggf_net* net, int n, const double* theta, const int* blocks, double* loss,
                             float* grad) {
    if (!net || n < 1 || !theta || !blocks || !loss || !grad) return GGF_EINVAL;
    cudaSetDevice(net->device);
    const size_t nl = 2 * (size_t)net->L * net->L;
    void *t1 = nullptr, *t2 = nullptr;
    NET_CK(cudaMalloc(&t1, n * nl * sizeof(double)));
    NET_CK(cudaMalloc(&t2, n * 2 * sizeof(int)));
    NET_CK(cudaMemcpy(t1, theta, n * nl * sizeof(double), cudaMemcpyHostToDevice));
    NET_CK(cudaMemcpy(t2, blocks, n * 2 * sizeof(int), cudaMemcpyHostToDevice));
    ggf_status s = ggf_net_head(net, n, 1, (const double*)t1, nullptr, (const int*)t2, nullptr, nullptr, 0, 0, 0);
    if (s == GGF_OK) {
        if (cudaMemcpy(loss, net->scal, sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(grad, net->g, NPARAM * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
            s = GGF_ECUDA;
    }
    cudaFree(t1);
    cudaFree(t2);
    if (s == GGF_OK) s = ggf_net_check(net);
    return s;
}

ggf_status ggf_net_train(ggf_net* net, int n_cfg, const double* theta, int batch, int n_steps, float lr,
                         float* losses, void* stream) {
    if (!net || n_cfg < 1 || !theta || batch < 1 || n_steps < 0) return GGF_EINVAL;
    cudaSetDevice(net->device);
    cudaStream_t st = (cudaStream_t)stream;
    GGF_TRY(net_ws(net, batch));
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (int k = 0; k < n_steps; ++k) {
        draw_batch<<<(batch + 127) / 128, 128, 0, st>>>(batch, n_cfg, net->L, net->seed, (uint64_t)net->t, net->cfg,
                                                       net->blocks);
        NET_CK(cudaGetLastError());
        GGF_TRY(ggf_net_head(net, batch, 1, theta, net->cfg, net->blocks, nullptr, nullptr, 0, 0, st));
        net->t += 1;
        float c1 = 1.f - powf(b1, (float)net->t), c2 = 1.f - powf(b2, (float)net->t);
        adam_kernel<<<(NPARAM + 255) / 256, 256, 0, st>>>(NPARAM, net->p, net->g, net->m, net->v, lr, b1, b2, eps, c1,
                                                          c2, net->pb);
        NET_CK(cudaGetLastError());
        if (losses) {
            double l = 0;
            NET_CK(cudaMemcpyAsync(&l, net->scal, sizeof(double), cudaMemcpyDeviceToHost, st));
            NET_CK(cudaStreamSynchronize(st));
            losses[k] = (float)l;
        }
    }
    NET_CK(cudaStreamSynchronize(st));
    return ggf_net_check(net);
}

}  // extern "C"
