/*
 * tnmc.h - C ABI of the batched Tensor Network Monte Carlo hot path
 * (arXiv 2509.19006, "BatchTNMC") for one NVIDIA B300 (sm_103a).
 *
 * The library runs, for a batch of 2D Edwards-Anderson disorder
 * realizations of possibly different sizes L_n (open boundaries):
 *   (a) the bottom-up boundary-MPS environments (Sec. 2.2, Sec. 3.2, Fig. 2):
 *       each row's transfer MPO applied to the bond-chi MPS and truncated
 *       back to chi by QR / SVD;
 *   (b) row-by-row, spin-by-spin ancestral proposals with their log q
 *       (Sec. 2.3 Eq. 9, Sec. 3.3);
 *   (c) the exact energy (Eq. 1) and the independence Metropolis-Hastings
 *       accept of Eq. 10;
 * and log Z from the top-row environment (Eq. 6).
 *
 * Conventions shared by every call
 * --------------------------------
 * - Memory: the caller owns every buffer. The library allocates no device
 *   memory: everything it needs lives in one caller-provided workspace
 *   (size from tnmc_workspace_size). The handle itself is a small host
 *   struct created by tnmc_create and released by tnmc_destroy.
 * - Streams: every call enqueues its kernels on the stream given to
 *   tnmc_create and returns without waiting (except tnmc_create and
 *   tnmc_get_device_status, which synchronise that stream).
 * - Pointers named d_* are device pointers, h_* host pointers.
 * - Errors: argument, state and launch errors are returned synchronously.
 *   Errors found by the kernels (bad couplings, a numerical breakdown, a
 *   bounded wait that ran out) are recorded per realization in device
 *   flags read by tnmc_get_device_status. No call aborts, traps or prints.
 * - Spin bits: 1 means s = +1, 0 means s = -1 (Sec. 3.3 uses 2*cfg-1).
 *   Sites of a realization are stored in raster order i = r*L + c, r = 0
 *   the top row (Eq. 3, Fig. 1a).
 * - Batched arrays: realization n's block starts after the blocks of
 *   realizations 0..n-1 (L_m^2 sites each, times S samples where the array
 *   holds S configurations per realization).
 * - Random numbers: Philox4x64-10 (Salmon et al., SC'11), key (seed, 0);
 *   spin draw of site i of proposal id t in realization n uses counter
 *   (i >> 2, t, g, 0) word i & 3; the accept test of proposal t uses
 *   (0, t, g, 1) word 0; the random initial state uses (i >> 2, 0, g, 2)
 *   word i & 3, where g is the realization's stream id (its index n unless
 *   set by tnmc_set_realization_ids). A word w becomes u = (2 (w >> 12) + 1) 2^-53.
 */
#ifndef TNMC_H
#define TNMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TNMC_OK = 0,
  TNMC_ERR_ARG = 1,          /* a bad argument (null pointer, size out of range) */
  TNMC_ERR_WORKSPACE = 2,    /* workspace too small or misaligned */
  TNMC_ERR_CUDA = 3,         /* a CUDA runtime call or a kernel launch failed */
  TNMC_ERR_NUMERIC = 4,      /* device flag: NaN/Inf or a vanishing norm */
  TNMC_ERR_TIMEOUT = 5,      /* device flag: a bounded wait ran out */
  TNMC_ERR_STATE = 6,        /* calls out of order (e.g. propose before build) */
  TNMC_ERR_UNSUPPORTED = 7   /* a valid request this build does not implement */
} tnmc_status;

/* Arithmetic of the environment build and of the sampling contractions.
 * Log scales, log q, log p and energies are float64 in every mode. */
typedef enum {
  TNMC_FP64 = 0,   /* all tensor arithmetic and the cache in float64 */
  TNMC_FP32 = 1,   /* all tensor arithmetic and the cache in float32 */
  TNMC_TF32 = 2,   /* float32 build, cache and sampling as TNMC_FP32, with the build's two
                      dense products per site (the previous row's site times the carried
                      triangular factor, Sec. 3.2's MPO x MPS contraction in parity form, and
                      the SVD input Q x blockdiag(U S)) on the tensor cores: operands rounded
                      to TF32 (10 mantissa bits), float32 accumulation; every row normalised
                      into the float64 log scale. Default cutoff 1e-6, as TNMC_FP32: the two
                      modes differ only in the rounding of the products. Accurate at small
                      beta only; the errors against the float64 oracle are tabulated by
                      tests/test_gpu_precision_table.py */
  TNMC_BF16 = 3,   /* as TNMC_TF32 with BF16 operands (7 mantissa bits) */
  TNMC_MIXED = 4,  /* float64 environment build (QR / SVD truncation, carried between
                      rows in float64), float32 cache and float32 sampling contractions */
  TNMC_DFLOAT = 5  /* double-float arithmetic (a float32 pair hi + lo, 48 significant bits,
                      float32's exponent range) for the environment build, the cache and the
                      sampling contractions, run on the FP32 pipes; the per-draw scalars,
                      log scales, log q, log p and energies in float64. The beta = 3 regime
                      needs float64-class accuracy in both the truncation and the sampling
                      contractions; this mode gives it without the float64 pipe */
} tnmc_prec;

/* Device flags (bit mask per realization) reported by tnmc_get_device_status. */
#define TNMC_FLAG_BAD_COUPLINGS 1  /* layout inconsistent, border not zero, or not finite */
#define TNMC_FLAG_NUMERIC 2        /* NaN/Inf, or both conditionals of a draw vanished */
#define TNMC_FLAG_TIMEOUT 4        /* a bounded device wait gave up */

typedef struct {
  int32_t n_real;        /* number of disorder realizations, >= 1 */
  const int32_t *L;      /* host array [n_real]: side L_n of each realization, 1 <= L_n <= 4096 */
  int32_t chi;           /* maximum bond dimension of the boundary MPS, 1 <= chi <= 64 */
  double beta;           /* inverse temperature, finite, >= 0 */
  int32_t prec;          /* tnmc_prec */
  int32_t max_samples;   /* largest S passed to propose / score / mh_step, >= 1 */
  double cutoff;         /* relative singular-value cutoff of the truncation (Sec. 1's
                            truncation threshold): at each bond keep the chi largest
                            singular values that exceed cutoff * (largest). <= 0 selects
                            the default of the precision: 1e-12 (FP64, MIXED, DFLOAT),
                            1e-6 (FP32, TF32, BF16).
                            Numerically-zero singular values must be dropped: their
                            noise directions grow under the next rows' transfer MPOs. */
  int32_t ckpt_every;    /* 0: cache the environment of every row. K >= 2: cache only rows
                            0, K, 2K, ... (checkpoints) plus one K-row segment, so the cache
                            holds ceil(L/K) + K rows per realization instead of L; propose,
                            score and mh_init then rebuild each K-row segment from the
                            checkpoint below it before sampling it (top segment first),
                            about one more environment build per call. Results are the same
                            bits as with 0. With TNMC_MIXED the checkpoint rows are also kept
                            in float64 (the precision the build carries between rows). */
  int32_t q_states;      /* 0 or 2: the Ising model of Eq. 1 (every mode above). 3 or 4: the
                            q-state Potts extension (Sec. 5), E = -sum J_ij delta(s_i, s_j) with
                            states 0 .. q-1 stored one byte per site; prec = TNMC_FP64 or
                            TNMC_FP32 (build, cache and sampling contractions in that type; the
                            per-draw probabilities, log q and energies in float64), chi <= 16
                            with q^2 chi <= 144, no checkpoints, no
                            learned correction. Proposals draw the first state k with
                            u < p_0 + ... + p_k (float64 partial sums, the site's Philox uniform).
                            Entry points other than build_envs, log_z, propose, score,
                            mh_init_empty and mh_step return TNMC_ERR_UNSUPPORTED for Potts
                            handles. Other values: TNMC_ERR_ARG (q = 1, q < 0) or
                            TNMC_ERR_UNSUPPORTED (q > 4, or a limit above). */
} tnmc_config;

typedef struct tnmc_handle tnmc_handle;

/* Human-readable name of a status code (static string, never NULL; unknown codes
 * get a generic name). The paper has no counterpart. Cannot fail. */
const char *tnmc_status_string(tnmc_status s);

/* Bytes of device workspace a configuration needs (written to *bytes); host only.
 * The size covers the coupling copy, the environment cache (Sec. 3.2 keeps one
 * environment per row; here L_n^2 sites of chi x chi values per realization, held in
 * device memory rather than on disk), the per-row log scales and bond sector sizes, and
 * the scratch of the environment build and of the sampler (right environments of
 * max_samples chains). Errors: TNMC_ERR_ARG (a field out of range or a NULL argument),
 * TNMC_ERR_UNSUPPORTED (a Potts request beyond the kernels, see q_states). */
tnmc_status tnmc_workspace_size(const tnmc_config *cfg, size_t *bytes);

/* Bind a configuration to a workspace and a CUDA stream (the paper has no counterpart).
 * d_ws: device pointer, 256-byte aligned, at least tnmc_workspace_size bytes;
 *       owned by the caller and used by the handle until tnmc_destroy.
 * cuda_stream: a cudaStream_t (NULL = legacy default stream).
 * Copies the per-realization table to the workspace and synchronises the
 * stream once. Errors: TNMC_ERR_ARG, TNMC_ERR_WORKSPACE, TNMC_ERR_CUDA. */
tnmc_status tnmc_create(const tnmc_config *cfg, void *d_ws, size_t ws_bytes,
                        void *cuda_stream, tnmc_handle **out);

/* Release the host handle (the workspace stays the caller's). NULL is a no-op. The
 * paper has no counterpart. Cannot fail. */
void tnmc_destroy(tnmc_handle *h);

/* Build the boundary-MPS environments of every realization (Sec. 3.2 and
 * Sec. 3.4: the bottom-row MPS, then for rows L-2..0 the row MPO applied to
 * the MPS below and compressed to chi by a left-to-right QR sweep and a
 * right-to-left truncating SVD sweep).
 * d_J: couplings in the paper's layout (Sec. 3.1): for each realization an
 *      (L_n, L_n, 4) float32 block, (left, up, right, down) per site, 0 on
 *      the open boundary; blocks concatenated over n ((sum L_n^2) x 4 floats).
 *      Read during this call's kernels only; the library keeps its own copy.
 * Realizations whose couplings fail the checks get TNMC_FLAG_BAD_COUPLINGS.
 * Errors: TNMC_ERR_ARG, TNMC_ERR_CUDA. */
tnmc_status tnmc_build_envs(tnmc_handle *h, const float *d_J);

/* log Z of every realization from the top-row environment (Eq. 6):
 * lambda_0 + log of the row-0 MPS with every physical leg summed.
 * d_logz: float64 [n_real]. Errors: TNMC_ERR_ARG, TNMC_ERR_STATE, TNMC_ERR_CUDA. */
tnmc_status tnmc_log_z(tnmc_handle *h, double *d_logz);

/* Draw S proposals per realization (Sec. 3.3, Eq. 5 and Eq. 9), proposal ids
 * prop_base .. prop_base + S - 1 (the Philox counters; distinct ids give
 * independent proposals, equal ids reproduce them bit for bit).
 * d_spins: uint8 [sum_n S L_n^2], raster order per configuration;
 * d_logq : float64 [n_real * S], log q(s) of each proposal (the log of the
 *          probabilities the draws were taken from);
 * d_E    : float64 [n_real * S], the energy of Eq. 1 (exact for +-J).
 * Errors: TNMC_ERR_ARG (S > max_samples), TNMC_ERR_STATE, TNMC_ERR_CUDA. */
tnmc_status tnmc_propose(tnmc_handle *h, int32_t S, uint64_t seed, uint64_t prop_base,
                         uint8_t *d_spins, double *d_logq, double *d_E);

/* Teacher-forced scoring (Sec. 3.3 with every spin forced; Eq. 9 and Eq. 1): log q and E
 * of S given configurations per realization (same layouts as tnmc_propose; d_spins is
 * read-only here). A configuration with a vanished conditional scores log q = -inf.
 * Errors: TNMC_ERR_ARG (S < 1 or S > max_samples, a NULL pointer), TNMC_ERR_STATE
 * (before tnmc_build_envs), TNMC_ERR_CUDA. */
tnmc_status tnmc_score(tnmc_handle *h, int32_t S, const uint8_t *d_spins,
                       double *d_logq, double *d_E);

/* Random initial chain state of every realization (uniform spins, Philox
 * stream 2, proposal id 0) scored by the proposal q: the start of the independence chain
 * of Eq. 10 (the paper does not state its chains' start).
 * d_state_spins: uint8 [sum L_n^2]; d_state_logq, d_state_E: float64 [n_real].
 * Errors: TNMC_ERR_ARG, TNMC_ERR_STATE (before tnmc_build_envs), TNMC_ERR_CUDA,
 * TNMC_ERR_UNSUPPORTED (Potts handles: use tnmc_mh_init_empty). */
tnmc_status tnmc_mh_init(tnmc_handle *h, uint64_t seed, uint8_t *d_state_spins,
                         double *d_state_logq, double *d_state_E);

/* Importance-sampling observables of S proposals per realization (the layouts of
 * tnmc_propose). With weights w_k = exp(-beta E_k - log q_k) (Eq. 1, Eq. 9; the
 * ratio of Eq. 10), d_out: float64 [n_real][6] receives per realization
 *   log mean_k w_k (an estimate of log Z), the effective sample size
 *   (sum w)^2 / sum w^2, the energy per spin sum w E / (N sum w), and, over the
 *   proposal pairs (0,1), (2,3), ... weighted by w_a w_b, the overlap moments
 *   <q^2>, <q^4> of q_ab = (1/N) sum_i s_i^a s_i^b and the Binder ratio
 *   (3 - <q^4>/<q^2>^2) / 2 (NaN when S < 2); N = L_n^2.
 * Weights are formed in the log domain, shifted by their maximum; every sum runs
 * in a fixed order. Errors: TNMC_ERR_ARG, TNMC_ERR_CUDA. */
tnmc_status tnmc_observables(tnmc_handle *h, int32_t S, const uint8_t *d_spins,
                             const double *d_logq, const double *d_E, double *d_out);

/* A chain state with no configuration yet: spins 0, E = 0 and log q = +inf,
 * so that the first proposal of the next tnmc_mh_step has log r = +inf and is
 * accepted: the chain then starts at a draw of q (no counterpart in the
 * paper). Use it where the random state of tnmc_mh_init can have
 * q = 0 in the arithmetic: in float32, the conditional of an unlikely forced
 * spin cancels to exactly 0 and such a chain would reject forever.
 * The forced first acceptance is counted in d_n_accept.
 * Errors: TNMC_ERR_ARG (a NULL pointer), TNMC_ERR_CUDA. */
tnmc_status tnmc_mh_init_empty(tnmc_handle *h, uint8_t *d_state_spins, double *d_state_logq,
                               double *d_state_E);

/* Independence Metropolis-Hastings (Eq. 10) over S proposals per
 * realization, consumed in id order prop_base .. prop_base + S - 1: proposal
 * t is accepted iff log u_t < (-beta E' - log q') - (-beta E - log q).
 * d_prop_*  : the outputs of tnmc_propose for the same S and prop_base;
 * d_state_* : the chain state, read and updated in place;
 * d_accept  : uint8 [n_real * S], 1 where the proposal was accepted;
 * d_n_accept: int64 [n_real], accepted proposals of this call added in.
 * Errors: TNMC_ERR_ARG, TNMC_ERR_CUDA. */
tnmc_status tnmc_mh_step(tnmc_handle *h, int32_t S, uint64_t seed, uint64_t prop_base,
                         const uint8_t *d_prop_spins, const double *d_prop_logq,
                         const double *d_prop_E, uint8_t *d_state_spins,
                         double *d_state_logq, double *d_state_E, uint8_t *d_accept,
                         int64_t *d_n_accept);

/* Optional diagnostic outputs (the paper has no counterpart), written by later calls until
 * reset with NULL. Errors: TNMC_ERR_ARG (NULL handle), TNMC_ERR_UNSUPPORTED (see Potts below).
 * d_logits : float32 [n_real * S * L^2] of propose / score: the logit of Eq. 5
 *            each draw was taken from (requires equal L for all realizations
 *            or is indexed like d_spins);
 * d_spectra: float64 [sum_n L_n (L_n + 1) chi] of build_envs: at row r,
 *            bond b (between sites b-1 and b), the kept singular values
 *            divided by the largest, in decreasing order, zero padded;
 * d_rowinfo: float64 [sum_n L_n * 14] of build_envs: per row (log of the
 *            2-norm of F_r, smallest relative gap s_kept/s_dropped - 1 at a
 *            cut, largest discarded weight, bonds where values were dropped,
 *            largest bond dimension, mean bond dimension, Jacobi SVDs run,
 *            mean Jacobi sweeps per SVD, then SM cycles spent in: MPO
 *            application + R handling, QR + Q formation, Theta product +
 *            setup (in float64 including the QR that preconditions the
 *            Jacobi), Jacobi, selection + stores, and the row's algorithmic
 *            flops: textbook counts of its QRs (2mn^2 - 2n^3/3, twice for Q),
 *            SVDs (4a^2b + 8ab^2 + 9b^3, Golub-Reinsch) and products).
 *            Potts handles (q_states >= 3) accept d_rowinfo only and fill its
 *            mean bond, SVD, sweep and flop fields and, in the four cycle fields,
 *            phase A, the Theta products, the Jacobi sweeps and selection + stores
 *            (the others 0); d_logits and d_spectra return TNMC_ERR_UNSUPPORTED. */
tnmc_status tnmc_set_diagnostics(tnmc_handle *h, float *d_logits, double *d_spectra,
                                 double *d_rowinfo);

/* ------------------------------------------------------------------------
 * Learned proposal correction (an extension; the paper has no counterpart).
 * A small network Delta_i = f(x_i) of seven local features shifts each
 * conditional logit of Eq. 5 before its draw, l_i <- l_i + Delta_i, and
 * log q (Eq. 9) is taken from the shifted logit, so q stays a normalised
 * distribution and the accept test of Eq. 10 keeps sampling exactly.
 * Features of site i = (r, c), 0 where the neighbour is absent:
 *   x0 = l_i (uncorrected logit of Eq. 5) clamped to [-32, 32]
 *   x1 = 2 beta Jv[r-1][c] s(r-1, c)
 *   x2 = beta Jh[r][c-1] s(r, c-1)          x3 = Jh[r][c]     x4 = Jv[r][c]
 *   x5 = s(r-1, c+1)                        x6 = beta
 * (Jh[r][c] joins (r,c)-(r,c+1), Jv[r][c] joins (r,c)-(r+1,c); s = +-1.)
 * The clamp keeps the input finite where a conditional vanishes (l_i = +-inf);
 * the corrected logit is the unclamped l_i + Delta_i.
 * Network: x rounded to bfloat16; h1 = g(W1 x + b1) rounded to bfloat16;
 * h2 = g(W2 h1 + b2); Delta = w3 . h2 + b3, with the smooth ReLU
 * g(z) = 0 (z <= -1), (z + 1)^2 / 4 (|z| < 1), z (z >= 1); float32
 * accumulation. Parameters: bfloat16 for inference, a float32 master copy for
 * training, both in this element layout: */
#define TNMC_MLP_FEATURES 7
#define TNMC_MLP_IN 16          /* W1 input columns; columns 7..15 are zero */
#define TNMC_MLP_HIDDEN 64
#define TNMC_MLP_OFF_W1 0       /* W1 [64][16], output-major */
#define TNMC_MLP_OFF_B1 1024    /* b1 [64] */
#define TNMC_MLP_OFF_W2 1088    /* W2 [64][64], output-major */
#define TNMC_MLP_OFF_B2 5184    /* b2 [64] */
#define TNMC_MLP_OFF_W3 5248    /* w3 [64] */
#define TNMC_MLP_OFF_B3 5312    /* b3, then 7 zeros */
#define TNMC_MLP_PARAMS 5320
#define TNMC_MLP_FEAT_STRIDE 8  /* floats per example row: x0 .. x6, then 0 */

/* Learned correction (no counterpart in the paper; its output enters q, Eq. 9, so
 * Eq. 10 stays exact). Use (enabled != 0) or stop using (enabled == 0, d_params_bf16
 * ignored) the correction in later tnmc_propose, tnmc_propose_static, tnmc_score,
 * tnmc_mh_init calls of this handle. d_params_bf16: device, 16-byte aligned,
 * TNMC_MLP_PARAMS bfloat16 values; the caller keeps it alive and unchanged
 * while those calls' kernels run. Errors: TNMC_ERR_ARG, TNMC_ERR_UNSUPPORTED (enabling it
 * on a Potts handle). */
tnmc_status tnmc_set_correction(tnmc_handle *h, const void *d_params_bf16, int32_t enabled);

/* Learned correction (no counterpart in the paper). Training examples from S
 * configurations per realization of this handle:
 * the features of every site. d_spins: as in tnmc_score; d_logits: float32,
 * the uncorrected logits of those configurations (tnmc_score with the
 * diagnostic logits set and no correction); d_feat: float32
 * [sum_n S L_n^2][TNMC_MLP_FEAT_STRIDE], in the order of d_spins.
 * Errors: TNMC_ERR_ARG, TNMC_ERR_STATE, TNMC_ERR_CUDA. */
tnmc_status tnmc_mlp_features(tnmc_handle *h, int32_t S, const uint8_t *d_spins,
                              const float *d_logits, float *d_feat);

/* Floats of scratch tnmc_mlp_grad needs (the learned correction: no counterpart in the
 * paper). Cannot fail. */
size_t tnmc_mlp_scratch_floats(void);

/* Learned correction (no counterpart in the paper). Mean binary cross entropy of
 * sigmoid(x0 + Delta) against the target
 * probability sigmoid(t) and its gradient in the parameters (backpropagation,
 * the two bfloat16 roundings passed straight through), over a minibatch.
 * d_feat: float32 [n_ex][8]; d_target_logit: float32 [n_ex];
 * B > 0: B examples drawn uniformly with replacement; example k is row
 *        floor(u n_ex), u the Philox uniform of counter (k >> 2, step, 0, 3)
 *        word k & 3 under key (seed, 0);  B == 0: all n_ex rows in order;
 * d_params_bf16: the network; d_grad: float32 [TNMC_MLP_PARAMS] (written);
 * d_loss: float64 [1] (written); d_scratch: float32 [tnmc_mlp_scratch_floats()];
 * stream: a cudaStream_t. The reduction order is fixed: equal inputs give
 * equal bits. Errors: TNMC_ERR_ARG, TNMC_ERR_CUDA. */
tnmc_status tnmc_mlp_grad(const float *d_feat, const float *d_target_logit, int64_t n_ex,
                          int32_t B, uint64_t seed, int32_t step, const void *d_params_bf16,
                          float *d_grad, double *d_loss, float *d_scratch, void *stream);

/* Learned correction (no counterpart in the paper). One Adam step (Kingma & Ba, 2015,
 * bias-corrected; step counts from 1) on the
 * float32 master copy d_master with moments d_m, d_v (all [TNMC_MLP_PARAMS],
 * updated in place), then the bfloat16 copy d_params_bf16 (round to nearest
 * even). Errors: TNMC_ERR_ARG, TNMC_ERR_CUDA. */
tnmc_status tnmc_mlp_adam(float *d_master, float *d_m, float *d_v, const float *d_grad,
                          int32_t step, float lr, float beta1, float beta2, float eps,
                          void *d_params_bf16, void *stream);

/* bfloat16 copy (round to nearest even) of a float32 parameter vector (the learned
 * correction: no counterpart in the paper). Errors: TNMC_ERR_ARG, TNMC_ERR_CUDA. */
tnmc_status tnmc_mlp_pack(const float *d_master, void *d_params_bf16, void *stream);

/* Learned correction (no counterpart in the paper). Delta of n_ex example rows (d_feat
 * as above) by the tensor-core network of
 * the sampler; d_delta: float32 [n_ex]. Errors: TNMC_ERR_ARG, TNMC_ERR_CUDA. */
tnmc_status tnmc_mlp_forward(const float *d_feat, int64_t n_ex, const void *d_params_bf16,
                             float *d_delta, void *stream);

/* Proposals without caller-provided scratch (the paper has no counterpart).
 * Same results and layouts as tnmc_propose, bit for bit, but the right
 * environments of the chains (S x sum_n L_n x chi values, 8 bytes each in
 * TNMC_FP64 mode, 4 otherwise, chi rounded up to 8/16/32/64) live in a
 * fixed 32 MiB device array owned by the library instead of the workspace.
 * It is for callers that cannot allocate device memory at the point of the
 * call: code running under a memory pool that is already fully reserved,
 * inside a region where the allocator must not be entered, or in a runtime
 * that owns all allocations and hands this library only the buffers it asked
 * for at setup. S may exceed the handle's max_samples as long as the scratch
 * fits in the array; larger requests return TNMC_ERR_ARG (see
 * tnmc_propose_static_limit). Nothing is allocated: no cudaMalloc, no
 * cudaFree, no allocating library routine.
 * Every call shares the one array, and nothing in it needs to start at zero
 * (each value read is written earlier in the same launch). Calls that overlap
 * on the GPU -- two streams, or two handles at the same time -- race on the
 * array and must be ordered by the caller. The first call on a device looks
 * up the array's device address once (cudaGetSymbolAddress, with that device
 * current) and keeps it for the life of the process; make that first call before
 * any stream capture. A device reset (or a release of the primary context) after
 * that first call is not supported: later calls would use the old address.
 * Errors: TNMC_ERR_ARG, TNMC_ERR_STATE, TNMC_ERR_CUDA. */
tnmc_status tnmc_propose_static(tnmc_handle *h, int32_t S, uint64_t seed, uint64_t prop_base,
                                uint8_t *d_spins, double *d_logq, double *d_E);

/* Bytes of the fixed device array used by tnmc_propose_static (no counterpart in the
 * paper). Cannot fail. */
size_t tnmc_propose_static_limit(void);

/* Budget, in SM clock cycles, of every bounded device wait of this handle's
 * later calls (0 = the default, about 20 s). The float64 build of at most 74
 * realizations runs as pairs of CTAs that hand parity sector 1's Jacobi SVDs
 * to each other through distributed shared memory; each hand-off waits on a
 * flag for at most this budget. A wait that runs out sets TNMC_FLAG_TIMEOUT
 * (read by tnmc_get_device_status as TNMC_ERR_TIMEOUT), the owning CTA then
 * does the work itself, and the launch ends normally. Failure-detection tests
 * set a tiny budget to make the waits run out (the paper has no counterpart).
 * Errors: TNMC_ERR_ARG. */
tnmc_status tnmc_set_wait_budget(tnmc_handle *h, int64_t cycles);

/* Stream ids of the realizations (the paper has no counterpart; it runs one
 * process): h_ids is a host array [n_real] of distinct non-negative ids, or NULL
 * for 0 .. n_real-1 (the default). A realization's random numbers depend on its
 * stream id, not on its position in this handle, so a batch split over several
 * processes (each handle holding a shard, ids = the realizations' indices in the
 * whole set) draws exactly what one handle over the whole set draws. Takes effect
 * for later calls; synchronises the handle's stream.
 * Errors: TNMC_ERR_ARG (negative id), TNMC_ERR_CUDA. */
tnmc_status tnmc_set_realization_ids(tnmc_handle *h, const int64_t *h_ids);

/* Kernel layout of the environment build (the paper has no counterpart; every layout
 * computes the same method and differs from the others in summation order only):
 *   bits 0-1, the Jacobi SVD of a parity sector where a realization runs on a pair of
 *     CTAs (float64, double-float): 0 = the precision's default (float64: 8 lanes per
 *     row pair on half the CTA; double-float: 16 lanes on the whole CTA), 1 = 8 lanes
 *     on the whole CTA, 2 = 8 lanes on half the CTA (3 is invalid);
 *   bit 2 (4): one CTA per realization even where pairs of CTAs fit;
 *   bit 3 (8): in the one-CTA build, 8 lanes per row pair instead of 4;
 *   bit 4 (16): the float32 build (TNMC_FP32, TF32, BF16) on pairs of CTAs where they
 *     fit, its Jacobi chosen by bits 0-1 (0 = 16 lanes on the whole CTA); without it the
 *     float32 build runs one CTA per realization;
 *   bit 5 (32): the float32 build's Jacobi preconditioned by a pivoted Householder QR, as
 *     the float64 and double-float builds always are: fewer sweeps, but the float32 Q is
 *     orthogonal only to float32 rounding, so the truncation is a little less accurate
 *     (float64 and double-float ignore the bit).
 * Applies to later tnmc_build_envs calls (and the segment rebuilds of checkpointed
 * handles). Errors: TNMC_ERR_ARG. */
tnmc_status tnmc_set_build_variant(tnmc_handle *h, int32_t variant);

/* The handle's current build layout (-1 for a NULL handle; no counterpart in the paper). */
int32_t tnmc_get_build_variant(const tnmc_handle *h);

/* Autotuner of the build layout (the paper has no counterpart): ingests d_J (as
 * tnmc_build_envs), then for each candidate layout of the handle's precision builds
 * `rows` rows of every realization, timed with CUDA events on the handle's stream, and
 * keeps the fastest for later builds. The timed rows are the `rows` rows below the
 * middle of the smallest lattice, rebuilt from the cached row under them (their bond
 * dimensions are those of the whole build); the rows from the middle down are built once
 * first, untimed, unless the handle holds a full build. With checkpoints, for TNMC_MIXED,
 * or for lattices below 2 rows + 2, the bottom `rows` rows are timed instead (their bonds
 * are smaller). h_variants / h_ms (host, optional, capacity *h_count on entry) receive the
 * candidates and their times in ms; *h_count receives the number of candidates.
 * Synchronises the stream. The timing launches overwrite rows of the cache, so the
 * handle must be built again (tnmc_build_envs) before proposals.
 * Errors: TNMC_ERR_ARG, TNMC_ERR_CUDA, TNMC_ERR_UNSUPPORTED (Potts handles). */
tnmc_status tnmc_autotune_build(tnmc_handle *h, const float *d_J, int32_t rows, int32_t *h_variants,
                                float *h_ms, int32_t *h_count);

/* Copy the per-realization device flags (TNMC_FLAG_*) to h_flags [n_real],
 * after synchronising the stream; clears them when clear != 0 (failure detection; the
 * paper has no counterpart).
 * Returns TNMC_OK, or TNMC_ERR_NUMERIC / TNMC_ERR_TIMEOUT if any flag of
 * that kind is set (bad couplings map to TNMC_ERR_ARG); TNMC_ERR_ARG for a NULL
 * argument, TNMC_ERR_CUDA if the copy fails. */
tnmc_status tnmc_get_device_status(tnmc_handle *h, int32_t *h_flags, int32_t clear);

/* Sizes of the internal layout, for tests (no counterpart in the paper): bytes of the
 * cache, of the environment-build scratch and of the sampler scratch; host only. A NULL
 * output is skipped. Errors: as tnmc_workspace_size. */
tnmc_status tnmc_layout_info(const tnmc_config *cfg, size_t *cache_bytes,
                             size_t *env_scratch_bytes, size_t *sample_scratch_bytes);

#ifdef __cplusplus
}
#endif

#endif /* TNMC_H */
