// Internal interface between the proposal network (k_net.cu) and the block
// sampler (k_block.cu).
#pragma once
#include "ggf_ctx.h"

int ggf_net_L(const ggf_net* net);
// mode 2: features of `theta` (n configurations, block origins `blocks`),
// forward pass, new block angles into prop[n][32] and log q(new) - log q(old)
// into logq[n]; Philox counter (counter, link k, 7, 0), key (seed, koff + sample).
ggf_status ggf_net_head(ggf_net* net, int n, int mode, const double* theta, const int* cfg, const int* blocks,
                        double* logq, double* prop, uint64_t seed, uint64_t counter, cudaStream_t st,
                        uint64_t koff = 0);
// GGF_ETIMEOUT once a tensor-core convolution's bounded wait ran out
// (synchronises the device), else GGF_OK.
ggf_status ggf_net_check(ggf_net* net);
