/* ggf.h - C ABI of libggf, a GB300 (sm_103a) sampler for gauged
 * superpositions of Gaussian fermionic PEPS (arXiv 2412.01737).
 *
 * The library samples gauge-link configurations G of an L x L periodic
 * lattice with probability p(G) = N(G) / N (Sec. 5.1), where
 *     N(G) = sum_nm lambda_n^* lambda_m N_nm(G)            (Sec. 5)
 * and N_nm(G) = <psi_n(G)|psi_m(G)>, psi_n(G) = <B_n| U(G) |A> (Sec. 4).
 * Each N_nm(G) is a constant times the Pfaffian of the virtual-mode matrix
 *     M_nm(G) = D + O(G) Gamma_{X_nm} O(G)^T,
 * D the direct sum of the sites' virtual covariance blocks, Gamma_{X_nm}
 * the link-local covariance of |B_n><B_m| / <B_m|B_n>, O(G) the gauge twist
 * on the source-end virtual Majoranas (Sec. 3.1, Sec. 5).
 *
 * Input conventions (all arrays row-major, all indices 0-based):
 *   site s = y*L + x; link l = 2*s + d joins the +d end of s (source end,
 *   carries the twist) to the -d end of s + e_d (d = 0: x, 1: y).
 *   Site Majorana layout [phys(2) | end -x | end +x | end -y | end +y], each
 *   end 2*n_v Majoranas, m_s = 2 + 8 n_v.  Bond layout per link
 *   [source end (2 n_v) | target end (2 n_v)], r = 4 n_v.
 *   Majoranas c_{2i} = psi_i + psi_i^dag, c_{2i+1} = -i (psi_i - psi_i^dag);
 *   covariance Gamma_ab = (i/2) <[c_a, c_b]> (Sec. 3.2).
 *   Z2 links: int8 values +1 / -1.  U(1) links: double angles in [0, 2 pi);
 *   a source-end mode of charge q is twisted by exp(i q theta n).
 *   SU(2) links (n_v = 2: one doublet per link end): four doubles per link,
 *   a unit quaternion (a0, a1, a2, a3) for u = a0 1 + i (a1 sigma_x +
 *   a2 sigma_y + a3 sigma_z); the source-end doublet is twisted by
 *   psi^dag_j -> sum_k psi^dag_k u_kj (the right-regular action, App. A).
 *   The weight is then invariant under u_l -> h_t^dag u_l h_s, and the
 *   plaquette observable is (1/2) tr(u1^dag u2^dag u3 u4).  The SU(2)
 *   proposal is u -> r u with
 *   r = cos d + i sin d (n . sigma), d = width (u_prop - 1/2) and n uniform
 *   on the sphere from Philox words 2 and 3 (z = 2 u - 1, phi = 2 pi u).
 *
 * Memory: every entry point that takes array arguments also takes `mem`:
 * GGF_MEM_DEVICE (device pointers, borrowed until the stream work ends) or
 * GGF_MEM_HOST (host pointers; the call copies in and out and returns after
 * synchronising the stream).  The caller owns every buffer it passes; the
 * library owns its internal state (inverses, workspaces).  No exception
 * crosses the ABI; every call returns a ggf_status and leaves a message for
 * ggf_last_error.  Calls on one context are not thread safe.
 * `stream` is a cudaStream_t (NULL = legacy default stream).
 */
#ifndef GGF_H
#define GGF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GGF_Z2 0
#define GGF_U1 1
#define GGF_SU2 2
#define GGF_FP64 0
#define GGF_FP32 1
#define GGF_MEM_DEVICE 0
#define GGF_MEM_HOST 1
#define GGF_N_OBS 3 /* per sweep and chain: plaquette mean, log N(G), acceptance */
#define GGF_OBS_PLAQUETTE 0

typedef enum {
    GGF_OK = 0,
    GGF_EINVAL = 1,     /* bad argument or size */
    GGF_ENOMEM = 2,     /* device allocation failed */
    GGF_ECUDA = 3,      /* a CUDA call failed */
    GGF_ESINGULAR = 4,  /* a matrix M(G) was singular (N(G) = 0) */
    GGF_ETIMEOUT = 5,   /* a bounded device wait ran out */
    GGF_EDRIFT = 6,     /* tracked log-weights drifted past tolerance */
    GGF_ESTATE = 7,     /* call out of order (e.g. sample before init) */
    GGF_EIO = 8         /* checkpoint file error */
} ggf_status;

typedef struct ggf_ctx ggf_ctx;

/* Create a context on CUDA device `device`.  *out is NULL on failure. */
ggf_status ggf_create(ggf_ctx** out, int device);
/* Free the context and everything it owns.  NULL is accepted. */
void ggf_destroy(ggf_ctx* ctx);
/* Message for the last failing call on ctx (valid until the next call). */
const char* ggf_last_error(const ggf_ctx* ctx);

/* Periodic L x L lattice, L >= 1 (Sec. 3: PEPS on a square lattice).
 * Resets groups, Gaussians and chains. */
ggf_status ggf_init_lattice(ggf_ctx* ctx, int L);

/* Gauge group (GGF_Z2, GGF_U1 or GGF_SU2, Sec. 2.1-2.2) and n_v in {1, 2}
 * virtual complex modes per link end (SU(2): n_v = 2, one doublet).
 * q_src[n_v]: U(1) charges of the source-end modes (ignored for Z2 and SU(2),
 * may be NULL then). */
ggf_status ggf_init_group(ggf_ctx* ctx, int group, int n_v, const int* q_src);

/* Variational parameters of the Ansatz (Sec. 4-5), host pointers:
 *   gamma_site [V][m_s][m_s]  pure site covariances Gamma_A (one per site),
 *   gamma_bond [K][2V][r][r]  pure bond covariances Gamma_{B_n} per link,
 *   lambda     [K][2]         complex weights lambda_n (re, im).
 * Builds the link-local covariances of |B_n><B_m|/<B_m|B_n>, the constants
 * <B_m|B_n> with the reference-state phase convention <B_n|B_0> > 0, B_0 :=
 * B_1 (Sec. 5), and the virtual blocks D.  1 <= K <= 8.  Host work only. */
ggf_status ggf_init_gaussians(ggf_ctx* ctx, const double* gamma_site, int K,
                              const double* gamma_bond, const double* lambda);

/* Introspection of the per-pair constants, P = K(K+1)/2 pairs ordered
 * (0,0)..(K-1,K-1) then (n,m), n<m, row by row.  log_c[2P]: complex log of the
 * constant c_nm in N_nm(G) = c_nm Pf(M_nm(G)) (diagonal pairs: log|c_nn|);
 * pairs[2P]: (n, m).  Either pointer may be NULL.  Host pointers. */
ggf_status ggf_get_constants(const ggf_ctx* ctx, int* n_pairs, double* log_c, int* pairs);

/* log N(G) for n_cfg configurations (Sec. 5): assemble M_nm(G) for every
 * pair, take log Pf(M_nm(G)) in FP64 on the GPU (site-by-site elimination
 * along the lattice; the dense Parlett-Reid Pfaffian for an item whose
 * pivot falls below 1e-8) and combine.
 *   links  [n_cfg][2V]  int8 (Z2) or double (U(1))
 *   logN   [n_cfg]      log N(G) (unnormalised; -inf if N(G) <= 0)
 *   ell    [n_cfg][P][2] optional (NULL): log Pf(M_nm(G)) as (log|Pf|, arg);
 *                       diagonal pairs report (log|Pf|, 0). */
ggf_status ggf_logweight(ggf_ctx* ctx, int n_cfg, const void* links, double* logN,
                         double* ell, int mem, void* stream);

/* Allocation-free log N(G): the same result as ggf_logweight.  The paper has
 * no counterpart for this call; it exists for callers that cannot allocate
 * device memory when they need the weights: hosts whose GPU memory is
 * budgeted once at start-up, processes that share the GPU under an
 * allocator that refuses further cudaMalloc calls, and loops that cannot
 * pay the implicit device synchronisation of cudaFree.  It calls no
 * cudaMalloc/cudaFree or
 * allocating library routine: all scratch lives in one fixed 32 MiB device
 * array inside the library (held by every GPU that loads the library until
 * the process exits).  The (configuration, pair) factorisations are done in
 * groups that fit the array, one at a time at the largest size, so any K is
 * accepted while M_nm is at most 1024 x 1024 (N = 8 n_v L^2 <= 1024); larger
 * lattices return GGF_EINVAL.  links [n_cfg][2V] and logN [n_cfg] are DEVICE
 * pointers.  The first call on a device looks up the array's device address
 * (a runtime query that allocates nothing).  Every call on a device
 * shares the array and it keeps the last call's contents: calls whose GPU
 * work overlaps race and must be serialised by the caller.  Work is enqueued
 * on `stream`; the call does not synchronise. */
ggf_status ggf_logweight_noalloc(ggf_ctx* ctx, int n_cfg, const void* links, double* logN, void* stream);

/* Wilson-loop observables from links alone (Sec. 2.3, Sec. 5.1).
 * which = GGF_OBS_PLAQUETTE: out[n_cfg] = mean over the V plaquettes of the
 * trace of the oriented plaquette product (Z2: product of signs; U(1): cos of
 * theta1 + theta2 - theta3 - theta4; SU(2): (1/2) tr(u1^dag u2^dag u3 u4)). */
ggf_status ggf_observable(ggf_ctx* ctx, int which, int n_cfg, const void* links,
                          double* out, int mem, void* stream);

/* Wilson loops from links alone (Sec. 5.1: oriented products of link
 * operators along closed paths, diagonal in G): out[n_cfg] = mean over the V
 * lower-left corners of the trace of the oriented product around the R x T
 * rectangle (R steps +x, T steps +y, back along -x and -y; 1 <= R, T <= L;
 * R = T = 1 is the plaquette).  A forward step contributes the covariant
 * link matrix (Z2 g; U(1) e^{i theta}, real part of the product; SU(2)
 * u^dag), a backward step its inverse; SU(2) takes (1/2) tr.  GGF_EINVAL for
 * R or T outside [1, L]. */
ggf_status ggf_wilson_loop(ggf_ctx* ctx, int R, int T, int n_cfg, const void* links, double* out, int mem,
                           void* stream);

/* Loops winding once around the torus along y (Polyakov loops of the
 * periodic lattice, closed through the boundary): out[n_cfg] = mean over the
 * L columns x of the trace of the product of the y links at x, with the
 * orientation rule of ggf_wilson_loop. */
ggf_status ggf_polyakov_loop(ggf_ctx* ctx, int n_cfg, const void* links, double* out, int mem, void* stream);

typedef struct {
    int precision;      /* GGF_FP64, or GGF_FP32 (inverse and updates in FP32,
                           ratios, log-weights and refresh in FP64) */
    int refresh_every;  /* full FP64 refresh of a chain after this many accepts */
    double width;       /* U(1) proposal: theta += width * (u - 1/2) */
    uint64_t seed;      /* Philox4x64-10 key word 0 (word 1 = chain_offset + chain index) */
    int delay;          /* <= 1: apply every accepted rank-r update to the
                           whole W at once (true columns);
                           k > 1 (at most 64): sweep in batches of k
                           consecutive links.  Their Majorana sets are
                           disjoint, so a batch needs only the k r x k r
                           block of the inverse on their union T: the
                           batch's proposals and accepted updates run on that
                           block and the composed update W - W[:, T] X W[T, :]
                           is folded into W with one rank-(k r) product
                           (delayed Sherman-Morrison-Woodbury updates, with
                           the true columns W[:, T]); learned-proposal block
                           moves need k >= 32. */
    int graph;          /* != 0: capture one sweep (all link steps, flushes,
                           observables) into a CUDA graph on first use and
                           replay it; 0: launch every kernel eagerly */
    uint64_t chain_offset;  /* Philox key word 1 = chain_offset + chain: a
                               replica holding chains i0 .. i0 + n - 1 of a
                               larger ensemble passes i0 and draws exactly
                               the numbers those chains draw in one run */
} ggf_chain_opts;

/* Create n_chains Markov chains starting at links [n_chains][2V] and build
 * their inverses W_nm = M_nm^{-1} and log-weights (full FP64 factorisation;
 * identical starting configurations are factored once).  Resets the sweep
 * counter to 0. */
ggf_status ggf_chains_init(ggf_ctx* ctx, int n_chains, const void* links,
                           const ggf_chain_opts* opts, int mem, void* stream);

/* Run n_sweeps Metropolis sweeps on every chain (Sec. 5.1).  A sweep
 * proposes links l = 0 .. 2V-1 in order (Z2 flip; U(1) theta += width (u -
 * 1/2) wrapped into [0, 2 pi); SU(2) the quaternion move described above),
 * scores each proposal by the low-rank Pfaffian
 * ratio on the cached inverse, accepts iff u < N(G')/N(G) and applies the
 * rank-r Sherman-Morrison-Woodbury update.  Random numbers: Philox4x64-10 with
 * counter (sweep, link, 0, 0), key (seed, chain); word 0 -> u_accept, word 1
 * -> u_propose (SU(2): words 2 and 3 give the axis), u = (word >> 11) 2^-53.
 *   obs [n_sweeps][n_chains][GGF_N_OBS] (may be NULL) */
ggf_status ggf_sample(ggf_ctx* ctx, int n_sweeps, double* obs, int mem, void* stream);

/* Sweep several independent problems together (uneven lattices, groups,
 * K, precisions): every context's captured sweep becomes a child of one
 * parent CUDA graph, so each sweep of the whole batch is a single graph
 * launch on the device.  All contexts must be on the same device, have chains
 * initialised with opts.graph != 0, and appear once.  obs[k] (may be NULL)
 * receives context k's observables as in ggf_sample.  Refreshes run per
 * context between launches.  Per-kernel timing (ggf_profile) is not recorded
 * in this mode. */
ggf_status ggf_sample_group(ggf_ctx* const* ctxs, int n_ctx, int n_sweeps, double* const* obs, int mem,
                            void* stream);

/* Current links of all chains, [n_chains][2V]. */
ggf_status ggf_chains_links(ggf_ctx* ctx, void* links, int mem, void* stream);

/* Tracked log Pf(M_nm) of all chains, [n_chains][P][2] as (log|Pf|, arg). */
ggf_status ggf_chains_ell(ggf_ctx* ctx, double* ell, int mem, void* stream);

/* Electric-field observables (Sec. 5.3) at the current configuration G of
 * every chain: the per-configuration factor f_E(G)_l of the single-link
 * integral, whose mean over samples of p(G) estimates the link's electric
 * term:
 *   Z2:   f_E(G)_l = sum_nm lambda_n^* lambda_m <psi_n(G)|psi_m(G^(l))> / N(G),
 *         G^(l) = G with link l flipped: the flip X_l, of which the Z2
 *         electric term is a linear function;
 *   U(1): f_E(G)_l = -d^2/dtheta'^2 of sum_nm lambda_n^* lambda_m
 *         <psi_n(G)|psi_m(theta'; G)> / N(G) at theta' = theta_l: the Casimir
 *         J_l^2 (J = -i d/dtheta), i.e. the twist charge Q_l = sum_j q_j n_j
 *         of the link's source-end modes squared, inserted on the ket;
 *   SU(2): the Casimir sum_a J_a J_a of right translations of the ket's link,
 *         i.e. sum_a (Q^a)^2 = (3/4)(n_0 + n_1 - 2 n_0 n_1) on the source
 *         doublet, inserted on the ket.
 * Computed from the cached inverses by Wick's theorem on the covariance
 * Gamma_O = i 1 - (1 + i D) W_nm (1 + i O Gamma_X O^T) restricted to the
 * source-end Majoranas S (Z2: (-1)^{n_v} Pf(Gamma_O[S, S]); U(1), SU(2):
 * occupations from Gamma_O[S, S]); only the 8 n_v x 4 n_v block of W between the source
 * site and the link is read.  Pending delayed updates are folded into W first.
 *   out [n_chains][2V][2] FP64 (re, im), caller-owned.  A single
 *   configuration's value is complex; its average over p(G) is real.
 * GGF_ESTATE before ggf_chains_init. */
ggf_status ggf_chains_electric(ggf_ctx* ctx, double* out, int mem, void* stream);

/* Gauge-invariant link terms (Sec. 5.2 with the link operator of the
 * observable): for link l = (s -> t),
 *   out[c][l] = u_l(G) sum_nm lambda_n^* lambda_m <psi_n(G)| F_s F_t |psi_m(G)> / N(G),
 * u_l = g_l (Z2) or e^{i theta_l} (U(1)), F_s = psi_s if charges[s] > 0 else
 * psi_s^dag, F_t = psi_t^dag if charges[t] > 0 else psi_t, psi_s =
 * (c_2s + i c_2s+1) / 2.  With the Gauss generator sum_out J - sum_in J +
 * q_s n_s this operator is gauge invariant; for staggered charges it is the
 * pair term, and T_l + T_l^dag the link's hopping term (its expectation is
 * 2 Re of the mean of out).  For Z2 every bilinear times g_l is invariant
 * and the same F are used.
 *   charges   [V] host int32, the sites' physical charges (+1 or -1, as the
 *             site states were built); 0 gives GGF_EINVAL.
 *   out       [n_chains][2V][2] FP64 (re, im), or null.
 *   pair_out  [n_chains][2V][K][K][2] FP64: the per-pair parts N_nm <F F>_nm
 *             u_l / N(G) (lambda^dag X lambda gives out), or null.
 * Both caller-owned, in the memory `mem` says; at least one non-null.
 * Blocking: returns after the results are written (it allocates and frees
 * scratch).  GGF_EINVAL for SU(2) chains, GGF_ESTATE before
 * ggf_chains_init. */
ggf_status ggf_chains_link_terms(ggf_ctx* ctx, const int* charges, double* out, double* pair_out, int mem,
                                 void* stream);

/* U(1) electric field (Sec. 5.3): out[c][l] = -i d/dtheta' of
 * sum_nm lambda_n^* lambda_m <psi_n(G)|psi_m(theta'; G)> / N(G) at
 * theta' = theta_l, i.e. the twist charge Q_l = sum_j q_j n_j of the link's
 * source-end modes inserted on the ket, from the same Gamma_O[S, S] as
 * ggf_chains_electric.  Site tensors conserve the total charge and bond
 * pairs are neutral, so in every configuration
 *   sum_{l out of s} out[c][l] - sum_{l into s} out[c][l] + q_s <n_s> = 0
 * with <n_s> = (1 + i site[s]) / 2 from ggf_chains_fermion (Gauss's law).
 *   out [n_chains][2V][2] FP64 (re, im), caller-owned.  GGF_EINVAL for
 *   non-U(1) chains or a null `out`, GGF_ESTATE before ggf_chains_init. */
ggf_status ggf_chains_electric_field(ggf_ctx* ctx, double* out, int mem, void* stream);

/* Fermionic observables (Sec. 5.2): Majorana bilinears on the physical
 * modes (site s carries c_2s, c_2s+1) at the current configuration G of every
 * chain,
 *     site[s]              = sum_nm lambda_n^* lambda_m <psi_n|c_2s c_2s+1|psi_m> / N(G),
 *     link[l][alpha][beta] = the same for c_{2s+alpha} c_{2t+beta}, l = (s -> t).
 * Densities are n_s = (1 + i site[s]) / 2; hoppings psi_s^dag psi_t and
 * pairings are linear in the link block; a gauge-invariant observable
 * multiplies them by its string of link variables, which is diagonal in G
 * (the per-sample product is the caller's).  Computed by Wick's theorem from
 * the physical covariance A + B W_nm B^T of each pair (A, B the sites'
 * physical and physical-virtual blocks; only the 8 n_v x 8 n_v block of W
 * between the two sites is read).  Pending delayed updates are folded into W
 * first.
 *   site [n_chains][V][2], link [n_chains][2V][2][2][2], FP64 (re, im),
 *   caller-owned; either may be NULL (not both: GGF_EINVAL).  GGF_ESTATE
 *   before ggf_chains_init. */
ggf_status ggf_chains_fermion(ggf_ctx* ctx, double* site, double* link, int mem, void* stream);

/* Score of the link blocks, per pair: out[c][p][l] = (w_p N_p / N(G))
 * (1/2) (O_l^T W_p[l, l] O_l)^T (r x r complex), w_p the pair weight
 * (|lambda_n|^2, or 2 lambda_n^* lambda_m for n < m), W_p[l, l] the block of
 * the pair's inverse on link l's r Majoranas and O_l the link's twist.  Since
 * N_p = c_p Pf(D + O Gamma_X^p O^T),
 *   d log N(G) = Re sum_p sum_l tr(U_p[l]^T dGamma_X^p[l]) + Re sum_p (w_p N_p / N(G)) d log c_p;
 * for K = 1 (Gamma_X = Gamma_B, c constant) this is the gradient with respect
 * to the bond covariances; for K > 1 the caller chains through the
 * transition covariances Gamma_X^nm and the pair constants.  Pending delayed
 * updates are folded into W first.
 *   out [n_chains][P][2V][r][r][2] FP64 (re, im), caller-owned.  GGF_EINVAL
 *   for a null `out`, GGF_ESTATE before ggf_chains_init. */
ggf_status ggf_chains_link_score(ggf_ctx* ctx, double* out, int mem, void* stream);

/* Nearest-neighbour four-point function (Sec. 5.2, a weight-four Majorana
 * monomial): out[c][l] = sum_nm lambda_n^* lambda_m
 * <psi_n|c_2s c_2s+1 c_2t c_2t+1|psi_m> / N(G) for link l = (s -> t), by
 * Wick's theorem -Pf of the physical covariance A + B W_nm B^T on those four
 * Majoranas (three 8 n_v x 8 n_v blocks of W per pair).  With the site
 * bilinears it gives density-density correlations,
 * <n_s n_t> = (1 + i site[s] + i site[t] - out) / 4.  A self-link gives -1.
 *   out [n_chains][2V][2] FP64 (re, im), caller-owned.  GGF_EINVAL for a
 *   null `out`, GGF_ESTATE before ggf_chains_init. */
ggf_status ggf_chains_fermion4(ggf_ctx* ctx, double* out, int mem, void* stream);

/* Per-pair parts of the per-configuration quantities, for optimising the
 * superposition weights: every quantity of Secs. 5.1-5.3 is a Hermitian form
 * in lambda, O(G) = sum_nm lambda_n^* lambda_m N_nm(G) o_nm(G), so
 *   <O>_lambda = lambda^dag Obar lambda / lambda^dag Nbar lambda
 * with Obar, Nbar the expectations over p(G) (the context's lambda) of the
 * matrices below; the lambda minimising an energy built from them is the
 * lowest generalised eigenvector.  out [n_chains][items][K][K][2] FP64 (re,
 * im) of N_nm(G) o_nm(G) / N(G), every ordered pair (n, m):
 *   GGF_PAIRS_NORM      items = 1: o_nm = 1 (Wilson loops: multiply by W(G));
 *   GGF_PAIRS_ELECTRIC  items = 2V: the electric insertion per link
 *                       (ggf_chains_electric's terms);
 *   GGF_PAIRS_SITE      items = V: -i Gamma_eff^nm[2s, 2s+1];
 *   GGF_PAIRS_LINK      items = 2V x 2 x 2: the link blocks of
 *                       ggf_chains_fermion, per pair;
 *   GGF_PAIRS_FIELD     items = 2V (U(1) chains only): the electric field
 *                       of ggf_chains_electric_field, per pair;
 *   GGF_PAIRS_FOUR      items = 2V: the four-point function of
 *                       ggf_chains_fermion4, per pair.
 * Contracting with lambda_n^* lambda_m gives the combined quantity (the
 * gauge-invariant link terms' parts come from ggf_chains_link_terms).  Pending
 * delayed updates are folded into W first.  GGF_EINVAL for an unknown `what`
 * or a null `out`, GGF_ESTATE before ggf_chains_init. */
#define GGF_PAIRS_NORM 0
#define GGF_PAIRS_ELECTRIC 1
#define GGF_PAIRS_SITE 2
#define GGF_PAIRS_LINK 3
#define GGF_PAIRS_FIELD 4
#define GGF_PAIRS_FOUR 5
ggf_status ggf_chains_pairs(ggf_ctx* ctx, int what, double* out, int mem, void* stream);

/* Score of the site blocks: out[c][s][i][j] = d log N(G_c) / d D_s[i][j]
 * for every chain c and site s, D_s the site's virtual covariance block
 * (B x B, B = 8 n_v, entries treated as independent), FP64.  For pure site
 * states N_nm(G) is a constant times Pf(D + O Gamma_X O^T), so the score is
 * Re sum_nm lambda_n^* lambda_m (N_nm(G) / N(G)) (1/2) W_nm[s, s]^T from the
 * cached inverses.  A change of the site parameters changes log N(G) by
 * sum_ij S_ij dD_ij; the gradient of a Wilson-loop energy is then the
 * covariance E_p[(W(G) - E) sum_s tr(S_s^T dD_s)].  Pending delayed updates
 * are folded into W first.  out [n_chains][V][B][B], caller-owned.
 * GGF_EINVAL for a null `out`, GGF_ESTATE before ggf_chains_init. */
ggf_status ggf_chains_score(ggf_ctx* ctx, double* out, int mem, void* stream);

/* Fault injection for tests: write NaN into element (i, j) (real part for a
 * complex pair) of one chain's cached inverse W_pair.  The sampler rejects a
 * proposal whose W_SS block is not finite (ratio 0), so the chain stalls
 * without error until a refresh rebuilds W from its links.  Synchronises the
 * device.  GGF_EINVAL for an index out of range, GGF_ESTATE before
 * ggf_chains_init. */
ggf_status ggf_debug_poison_inverse(ggf_ctx* ctx, int chain, int pair, int i, int j);
/* Test hook (no counterpart in the paper): multiply the cached FP32 inverse
 * of one chain and pair by `factor`, an error of known size for the refresh
 * to repair.  Synchronous. */
ggf_status ggf_debug_scale_inverse(ggf_ctx* ctx, int chain, int pair, double factor);

/* Copy the cached inverse W_nm = M_nm(G)^{-1} of one chain and pair (pair
 * index as in ggf_get_constants) into out [N][N][2] as FP64 (re, im), N = 8 n_v
 * L^2.  For tests and diagnostics. */
ggf_status ggf_chains_inverse(ggf_ctx* ctx, int chain, int pair, double* out, int mem, void* stream);

/* Residual of the cached inverse of one FP32 chain and pair (pair index as in
 * ggf_get_constants): *rmax = max |I - M_nm(G) W| over the entries (M
 * assembled in FP64 from the chain's links, the product in FP32).  apply != 0
 * then refines W by one Newton step W <- W + W (I - M W) on the tensor cores
 * (one TF32 product when *rmax <= 1e-4, else the FP32-accurate three-product
 * split; skipped when *rmax > 5e-2).  The periodic refresh skips the step at
 * the FP32 floor (*rmax <= 4e-6) and repeats it, at most three times, while
 * the residual shrinks.  The
 * paper has no counterpart; for tests and diagnostics.  Synchronous. */
ggf_status ggf_chains_refine(ggf_ctx* ctx, int chain, int pair, int apply, double* rmax);

typedef struct {
    uint64_t proposals, accepts, refreshes, sweeps;
    double max_drift;   /* max |l_tracked - l_refresh| over refreshes so far */
    uint64_t launches;  /* CUDA kernels launched by ggf_sample since ggf_chains_init */
    uint64_t block_proposals, block_accepts;   /* learned-proposal block moves */
    int n_chains, n_pairs;
    double max_resid;          /* FP32 chains: largest |I - M W| entry met by a
                                  refresh before its Newton step */
    uint64_t dense_refreshes;  /* FP32 chains refreshed by FP64 Gauss-Jordan
                                  because the Newton steps could not bring
                                  the residual to the FP32 floor */
    uint64_t refine_steps;     /* Newton steps taken by refreshes */
    uint64_t dense_pfaffians;  /* log-Pfaffians that fell back from the
                                  site-by-site to the dense elimination */
    uint64_t flush_wave;       /* FP32 delayed modes: chains per wave of the
                                  tensor-core flush (0 otherwise) */
} ggf_chain_stats;

ggf_status ggf_chains_stats(ggf_ctx* ctx, ggf_chain_stats* out);

/* Per-chain failure report (the aggregate counters above say that something
 * failed, this says which chain): status[n_chains] (int32, host or device per
 * mem) gets GGF_ESINGULAR for a chain whose factorisation met a singular
 * M_nm(G) or whose tracked log-weights are not finite, GGF_EDRIFT for one
 * whose largest |l_tracked - l_refresh| so far exceeds drift_tol (tol <= 0:
 * not checked), else GGF_OK.  Synchronises `stream`. */
ggf_status ggf_chains_status(ggf_ctx* ctx, double drift_tol, int32_t* status, int mem, void* stream);

/* Write / read the chain state (links, sweep counter, options, log-weights,
 * counters).  Inverses are rebuilt on resume by a full refresh, so resumed
 * chains make the same decisions as uninterrupted ones. */
/* Chain state in memory, for residency waves (more chains than fit in HBM,
 * paged to host memory, e.g. the Grace CPU's over NVLink-C2C): the links,
 * cached inverses, tracked log-weights, refresh counters, drift, options and
 * sweep counter of the context's chains, after folding pending updates.
 * Loading a state into a context whose chains have the same problem, count,
 * precision and delay continues those chains bit for bit (no refactorisation);
 * the loaded options (seed, width, refresh cadence) replace the context's and
 * the captured sweep graph is rebuilt on the next ggf_sample.
 *   state_size: bytes of the state; save_state/load_state: dst/src of that
 *   size, host (GGF_MEM_HOST; pinned memory copies fastest) or device memory,
 *   caller-owned.  GGF_EINVAL for a state of another problem or shape,
 *   GGF_ESTATE before ggf_chains_init. */
ggf_status ggf_chains_state_size(ggf_ctx* ctx, uint64_t* bytes);
ggf_status ggf_chains_save_state(ggf_ctx* ctx, void* dst, int mem, void* stream);
ggf_status ggf_chains_load_state(ggf_ctx* ctx, const void* src, int mem, void* stream);

ggf_status ggf_checkpoint(ggf_ctx* ctx, const char* path);
ggf_status ggf_resume(ggf_ctx* ctx, const char* path, void* stream);

/* Kernel timing with CUDA events recorded on the launching stream, for
 * benchmarks.  ggf_profile(ctx, 1) starts recording events around the launch
 * groups issued by ggf_sample and ggf_sample_blocks and resets the totals;
 * ggf_profile(ctx, 0) stops.  Categories:
 *   GGF_KT_RATIO    link-step ratio launches (one link per launch), and the
 *                   batched link steps on the small matrices (batch_steps)
 *   GGF_KT_UPDATE   immediate rank-r updates; row/column gathers of the
 *                   pending-panel path (block moves)
 *   GGF_KT_REFRESH  full refreshes
 *   GGF_KT_FLUSH    delayed-update flushes W <- W - U V
 *   GGF_KT_GATHER   batched mode: W[:, T], W[T, :] and W[T, T] gathers
 *   GGF_KT_APPLY    batched mode: V <- X V
 * ggf_kernel_time returns the accumulated device milliseconds and the number
 * of timed launch groups since the last reset.  Events are read at the end of
 * each sweep.  In graph mode the sweep replayed while timing is on is the same
 * captured sweep with event-record nodes around its launch groups (captured
 * once, kept beside the plain graph). */
#define GGF_KT_RATIO 0
#define GGF_KT_UPDATE 1
#define GGF_KT_REFRESH 2
#define GGF_KT_FLUSH 3
#define GGF_KT_GATHER 4
#define GGF_KT_APPLY 5
#define GGF_KT_N 6
ggf_status ggf_profile(ggf_ctx* ctx, int enable);
ggf_status ggf_kernel_time(ggf_ctx* ctx, int which, double* ms, uint64_t* launches);

/* Self-test of the tensor-core delayed-update flush (W <- W - U V^T with
 * FP32 data on tcgen05 TF32 tensor cores, three-product split): runs it on
 * one N x N (cplx = 0) or complex N x N (cplx = 1) matrix with seeded data
 * and a rank-`rank` panel (rank a multiple of 4, <= 512) and reports the
 * largest error relative to the largest entry of an FP64 reference, over both
 * flush kernels: the per-tile split (Newton step of the refresh) and the
 * pre-split one the sweeps use.  Needs only a context (allocates its own
 * buffers).  Not part of the method. */
ggf_status ggf_selftest_flush(ggf_ctx* ctx, int cplx, int N, int rank, double* max_rel_err);

/* The same seeded case with its data, for a reference computed outside the
 * library: which = 0 runs the per-tile-split flush, 1 the pre-split one.
 * Host outputs (caller-owned):
 *   w0, w1  [N][N] floats (cplx = 0) or [N][N][2] (re, im), the input and
 *           output W;
 *   pan     the panels: planes U, V^T (cplx = 0) or U re, U im, V^T re,
 *           V^T im, each NP x KP floats with NP = N rounded up to 256 and
 *           KP = rank rounded up to 8, element (row, q) of a plane at
 *           ((q / 8) NP + row) 8 + q % 8.  Only rows < N and q < rank enter:
 *           w1 = w0 - U (V^T)^T over them.
 * Not part of the method. */
ggf_status ggf_selftest_flush_data(ggf_ctx* ctx, int cplx, int N, int rank, int which, float* w0, float* pan,
                                   float* w1);

/* ---- Learned block proposal ------------------------------------------------
 * A small convolutional network proposes new angles for the 32 links of a
 * 4 x 4 block of sites (U(1) only) from the links outside the block; block
 * moves are accepted by exact Metropolis-Hastings against p(G) (Sec. 5.1),
 * so the sampled distribution does not depend on how well it is trained.
 * Architecture: per-site input channels (cos, sin of the site's x- and
 * y-link angles; cos, sin of the plaquette angle; block flags of the two
 * links) with the block's links and the plaquettes containing them zeroed;
 * 3x3 circular convolutions 8 -> 64 -> 64 -> 64 -> 6 with ReLU between; per
 * block link a wrapped Cauchy density with mu = atan2(b, a), rho = 0.95
 * sigmoid(z) from the head.  BF16 weights and activations, FP32 accumulation,
 * FP32 master weights trained with Adam on configurations the sampler made.
 * Parameters: one FP32 array of GGF_NET_PARAMS, per layer W[co][ci][3][3]
 * then bias[co]. */
#define GGF_NET_PARAMS 81990
typedef struct ggf_net ggf_net;
ggf_status ggf_net_create(ggf_net** out, int device, int L, uint64_t seed);
void ggf_net_destroy(ggf_net* net);
const char* ggf_net_last_error(const ggf_net* net);
ggf_status ggf_net_get_params(ggf_net* net, float* out /* host, GGF_NET_PARAMS */);
ggf_status ggf_net_set_params(ggf_net* net, const float* in /* host; resets Adam */);
/* log q of the block links of n configurations: theta [n][2L^2], blocks
 * [n][2] origins (bx, by), logq [n]. */
ggf_status ggf_net_logq(ggf_net* net, int n, const double* theta, const int* blocks, double* logq, int mem,
                        void* stream);
/* Training loss (mean over the n samples of -sum log f) and its gradient
 * [GGF_NET_PARAMS]; host arrays. */
ggf_status ggf_net_loss_grad(ggf_net* net, int n, const double* theta, const int* blocks, double* loss,
                             float* grad);
/* n_steps Adam steps (lr; betas 0.9, 0.999) on minibatches of `batch`
 * samples: a configuration drawn from theta [n_cfg][2L^2] (DEVICE) and a block
 * origin, both from Philox.  losses [n_steps] host, optional. */
ggf_status ggf_net_train(ggf_net* net, int n_cfg, const double* theta, int batch, int n_steps, float lr,
                         float* losses, void* stream);

/* n_moves block moves of every chain of a U(1) context whose chains were
 * initialised with delay >= 32 (see the steps in the section comment): block
 * origin per chain from Philox (counter (move, 0, 21, 0), key (seed, chain)),
 * proposal from `net` (same lattice size), the 32 link changes applied as
 * tentative rank-r updates whose Pfaffian ratios multiply to the block ratio,
 * and Metropolis-Hastings acceptance u < [N(G')/N(G)] q(old)/q(new)
 * (u from counter (move, 0, 23, 0)).  obs [n_moves][n_chains][GGF_N_OBS] as in
 * ggf_sample (acceptance column: 1 or 0 for the move).  No refresh runs inside
 * this call. */
ggf_status ggf_sample_blocks(ggf_ctx* ctx, ggf_net* net, int n_moves, double* obs, int mem, void* stream);

/* Wait for the context's work on `stream` and report device-side errors. */
ggf_status ggf_sync(ggf_ctx* ctx, void* stream);

#ifdef __cplusplus
}
#endif
#endif
