// C ABI of the TNMC library (include/tnmc.h): workspace planning, argument
// checks and kernel launches. No device memory is allocated here.
#include "../../include/tnmc.h"
#include "common.cuh"

#include <algorithm>
#include <cmath>
#include <new>
#include <numeric>
#include <vector>

namespace tnmc {
cudaError_t launch_ingest(const Layout &lay, const float *J, cudaStream_t st);
cudaError_t launch_env_build(const Layout &lay, int mode, int CH, cudaStream_t st);
cudaError_t launch_log_z(const Layout &lay, int prec, double *logz, cudaStream_t st);
cudaError_t launch_init_state(const Layout &lay, uint64_t seed, uint8_t *spins, cudaStream_t st);
cudaError_t launch_empty_state(const Layout &lay, double *logq, double *E, cudaStream_t st);
cudaError_t launch_observables(const Layout &lay, int S, const uint8_t *spins, const double *logq,
                               const double *E, double *out, cudaStream_t st);
cudaError_t launch_mh(const Layout &lay, int S, uint64_t seed, uint64_t base, const uint8_t *ps,
                      const double *pl, const double *pe, uint8_t *ss, double *sl, double *se,
                      uint8_t *acc, int64_t *nacc, cudaStream_t st);
cudaError_t launch_propose(const Layout &lay, int prec, int CH, int S, uint64_t seed,
                           uint64_t base, uint8_t *spins, double *lq, double *E, cudaStream_t st);
cudaError_t launch_score(const Layout &lay, int prec, int CH, int S, const uint8_t *spins,
                         double *lq, double *E, cudaStream_t st);
int64_t env_slot_bytes(int mode, int CH, int L_max, int chi);
cudaError_t launch_propose_static(const Layout &lay, int prec, int CH, int S, uint64_t seed,
                                  uint64_t base, uint8_t *spins, double *lq, double *E,
                                  int64_t sum_L, cudaStream_t st, bool *too_big);
int64_t static_scratch_bytes();
int64_t sampler_smem_bytes(int prec, int CH, int L_max);
cudaError_t launch_mlp_features(const Layout &lay, int S, int L_max, const uint8_t *spins,
                                const float *logits, float *feat, cudaStream_t st);
int64_t potts_slot_bytes(int L_max, int esz);
bool potts_supported(int q, int chi);
int potts_scratch_ch();
cudaError_t launch_potts_build(const Layout &lay, int q, int prec, cudaStream_t st);
cudaError_t launch_potts_log_z(const Layout &lay, int q, int prec, double *logz, cudaStream_t st);
cudaError_t launch_potts_sample(const Layout &lay, int q, int prec, int S, uint64_t seed, uint64_t base,
                                const uint8_t *in, uint8_t *out, double *lq, double *E, cudaStream_t st);
}  // namespace tnmc

using namespace tnmc;

namespace {

constexpr int kMaxL = 4096;
constexpr int kEnvSlots = 148;   // workspace slots of the environment build: at most one per SM of a B300

struct Plan {
  int CH = 0;
  int64_t sum_L2 = 0, sum_L = 0, sum_bonds = 0, sum_cache = 0;   // sum_cache: chi x chi matrices
  int L_max = 0;
  int64_t off_reals, off_order, off_flags, off_counter, off_jr, off_jd, off_cache, off_bonds,
      off_lam, off_env, off_samp, off_ckpt64, total;
  int64_t sum_ckpt = 0;   // chi x chi matrices of float64 checkpoint rows (MIXED + checkpoints)
  int64_t cache_bytes, env_bytes, samp_bytes, env_slot;
  int env_slots;
};

int pick_ch(int chi) {
  for (int ch : {8, 16, 32, 64})
    if (chi <= ch) return ch;
  return -1;
}

tnmc_status check_cfg(const tnmc_config *cfg) {
  if (!cfg || !cfg->L || cfg->n_real < 1) return TNMC_ERR_ARG;
  if (cfg->chi < 1 || cfg->chi > 64) return TNMC_ERR_ARG;
  if (!std::isfinite(cfg->beta) || cfg->beta < 0) return TNMC_ERR_ARG;
  if (cfg->max_samples < 1 || cfg->max_samples > (1 << 24)) return TNMC_ERR_ARG;
  if (!std::isfinite(cfg->cutoff) || cfg->cutoff >= 1.0) return TNMC_ERR_ARG;
  if (cfg->ckpt_every < 0 || cfg->ckpt_every == 1) return TNMC_ERR_ARG;
  if (cfg->prec < TNMC_FP64 || cfg->prec > TNMC_DFLOAT) return TNMC_ERR_ARG;
  if (cfg->q_states < 0 || cfg->q_states == 1) return TNMC_ERR_ARG;
  if (cfg->q_states > 2) {   // the q-state Potts extension: float64 kernels with fixed panel bounds
    if ((cfg->prec != TNMC_FP64 && cfg->prec != TNMC_FP32) || cfg->ckpt_every != 0 ||
        !potts_supported(cfg->q_states, cfg->chi))
      return TNMC_ERR_UNSUPPORTED;
  }
  for (int n = 0; n < cfg->n_real; ++n)
    if (cfg->L[n] < 1 || cfg->L[n] > kMaxL) return TNMC_ERR_ARG;
  return TNMC_OK;
}

// 0: float64 build + float64 cache; 1: float32 build + cache (FP32, and TF32 / BF16 with the
// dense products on the tensor cores); 2: float64 build, float32 cache; 3: double-float build + cache
int env_mode(int prec) {
  if (prec == TNMC_FP64) return 0;
  if (prec == TNMC_FP32 || prec == TNMC_TF32 || prec == TNMC_BF16) return 1;
  return prec == TNMC_DFLOAT ? 3 : 2;
}
// operand rounding of the build's dense products (env_build.cu, TCMODE_*)
int tc_mode_of(int prec) { return prec == TNMC_TF32 ? 1 : (prec == TNMC_BF16 ? 2 : 0); }
// type of the cache and of the sampler: 0 = float64, 1 = float32, 2 = double-float
int cache_code(int prec) { return prec == TNMC_FP64 ? 0 : (prec == TNMC_DFLOAT ? 2 : 1); }
// bytes of a cache / sampler value
int64_t value_bytes(int prec) { return cache_code(prec) == 1 ? 4 : 8; }
// the float32 modes (FP32, TF32, BF16) share float32's cutoff: their truncations differ only
// in the rounding of the products
double default_cutoff(int prec) {
  return (prec == TNMC_FP32 || prec == TNMC_TF32 || prec == TNMC_BF16) ? 1e-6 : 1e-12;
}

// q-state Potts handles (q_states >= 3)
bool is_potts(const tnmc_config *cfg) { return cfg->q_states > 2; }

Plan make_plan(const tnmc_config *cfg) {
  Plan p;
  const bool potts = is_potts(cfg);
  p.CH = potts ? potts_scratch_ch() : pick_ch(cfg->chi);
  const int64_t esz = value_bytes(cfg->prec);
  // a Potts site is q dense chi x chi matrices; an Ising site one parity-form matrix
  const int64_t site_mats = potts ? cfg->q_states : 1;
  for (int n = 0; n < cfg->n_real; ++n) {
    const int64_t L = cfg->L[n];
    p.sum_L2 += L * L;
    p.sum_L += L;
    p.sum_bonds += L * (L + 1);
    p.sum_cache += cache_rows(int(L), cfg->ckpt_every) * L;
    if (cfg->ckpt_every > 0 && cfg->prec == TNMC_MIXED)
      p.sum_ckpt += int64_t((L + cfg->ckpt_every - 1) / cfg->ckpt_every) * L;
    p.L_max = std::max<int>(p.L_max, int(L));
  }
  int64_t o = 0;
  auto take = [&](int64_t bytes) { const int64_t at = o; o += align256(bytes); return at; };
  p.off_reals = take(int64_t(cfg->n_real) * sizeof(RealInfo));
  p.off_order = take(int64_t(cfg->n_real) * 4);
  p.off_flags = take(int64_t(cfg->n_real) * 4);
  p.off_counter = take(64 * 4);
  p.off_jr = take(p.sum_L2 * 4);
  p.off_jd = take(p.sum_L2 * 4);
  p.cache_bytes = p.sum_cache * site_mats * int64_t(cfg->chi) * cfg->chi * esz;
  p.off_cache = take(p.cache_bytes);
  p.off_bonds = take(p.sum_bonds * 8);
  p.off_lam = take(p.sum_L * 8);
  p.env_slots = std::min(cfg->n_real, kEnvSlots);
  p.env_slot = potts ? potts_slot_bytes(p.L_max, int(esz))
                     : env_slot_bytes(env_mode(cfg->prec), p.CH, p.L_max, cfg->chi);
  p.env_bytes = p.env_slot * p.env_slots;
  p.off_env = take(p.env_bytes);
  p.samp_bytes = int64_t(cfg->max_samples) * p.sum_L * p.CH * esz;
  p.off_samp = take(p.samp_bytes);
  // MIXED carries the build between rows in float64: its checkpoints keep that row
  p.off_ckpt64 = take(p.sum_ckpt * int64_t(cfg->chi) * cfg->chi * 8);
  p.total = o;
  return p;
}

cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

}  // namespace

struct tnmc_handle {
  std::vector<int32_t> L;
  std::vector<RealInfo> reals;   // host copy of the per-realization table
  tnmc_config cfg;
  Plan plan;
  Layout lay;
  int env_code;    // env_mode()
  int prec_code;   // cache_code(): sampler / log Z kernels on float64 (0), float32 (1), double-float (2)
  cudaStream_t stream;
  bool built = false;
  int q = 2;       // 2: Ising; 3 or 4: the q-state Potts extension (potts.cu)
};

namespace {

// Run a sampler launch over all rows, or, with checkpointed environments, one
// K-row segment at a time from the top: rebuild the segment's rows from the
// checkpoint below it, then sample them (the chains carry over in the outputs).
template <typename F>
cudaError_t for_segments(tnmc_handle *h, F launch_rows) {
  const int K = h->cfg.ckpt_every;
  if (K <= 0) return launch_rows(h->lay);
  const int nseg = (h->plan.L_max + K - 1) / K;
  for (int s = 0; s < nseg; ++s) {
    Layout l2 = h->lay;
    l2.seg_begin = s * K;
    l2.seg_end = s * K + K;
    cudaError_t e = launch_env_build(l2, h->env_code, h->plan.CH, h->stream);
    if (e == cudaSuccess) e = launch_rows(l2);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace

extern "C" {

const char *tnmc_status_string(tnmc_status s) {
  switch (s) {
    case TNMC_OK: return "ok";
    case TNMC_ERR_ARG: return "invalid argument";
    case TNMC_ERR_WORKSPACE: return "workspace too small or misaligned";
    case TNMC_ERR_CUDA: return "CUDA error";
    case TNMC_ERR_NUMERIC: return "numerical breakdown (device flag)";
    case TNMC_ERR_TIMEOUT: return "bounded device wait ran out (device flag)";
    case TNMC_ERR_STATE: return "call out of order";
    case TNMC_ERR_UNSUPPORTED: return "not supported by this build";
  }
  return "unknown status";
}

tnmc_status tnmc_workspace_size(const tnmc_config *cfg, size_t *bytes) {
  if (!bytes) return TNMC_ERR_ARG;
  const tnmc_status s = check_cfg(cfg);
  if (s != TNMC_OK) return s;
  *bytes = size_t(make_plan(cfg).total);
  return TNMC_OK;
}

tnmc_status tnmc_layout_info(const tnmc_config *cfg, size_t *cache_bytes, size_t *env_bytes,
                             size_t *samp_bytes) {
  const tnmc_status s = check_cfg(cfg);
  if (s != TNMC_OK) return s;
  const Plan p = make_plan(cfg);
  if (cache_bytes) *cache_bytes = size_t(p.cache_bytes);
  if (env_bytes) *env_bytes = size_t(p.env_bytes);
  if (samp_bytes) *samp_bytes = size_t(p.samp_bytes);
  return TNMC_OK;
}

tnmc_status tnmc_create(const tnmc_config *cfg, void *d_ws, size_t ws_bytes, void *cuda_stream,
                        tnmc_handle **out) {
  if (!out) return TNMC_ERR_ARG;
  *out = nullptr;
  tnmc_status s = check_cfg(cfg);
  if (s != TNMC_OK) return s;
  const Plan p = make_plan(cfg);
  if (!d_ws || (reinterpret_cast<uintptr_t>(d_ws) & 255) != 0 || ws_bytes < size_t(p.total))
    return TNMC_ERR_WORKSPACE;
  tnmc_handle *h = new (std::nothrow) tnmc_handle();
  if (!h) return TNMC_ERR_ARG;
  h->L.assign(cfg->L, cfg->L + cfg->n_real);
  h->cfg = *cfg;
  h->cfg.L = h->L.data();
  h->plan = p;
  h->env_code = env_mode(cfg->prec);
  h->prec_code = cache_code(cfg->prec);
  h->q = is_potts(cfg) ? cfg->q_states : 2;
  h->stream = as_stream(cuda_stream);
  unsigned char *ws = static_cast<unsigned char *>(d_ws);

  // per-realization table and the longest-first order
  std::vector<RealInfo> reals(cfg->n_real);
  int64_t so = 0, bo = 0, ro = 0, co = 0, ko = 0;
  for (int n = 0; n < cfg->n_real; ++n) {
    const int64_t L = cfg->L[n];
    reals[n].L = int32_t(L);
    reals[n].pad = 0;
    reals[n].site_off = so;
    reals[n].bond_off = bo;
    reals[n].row_off = ro;
    reals[n].line_off = ro;
    reals[n].cache_off = co;
    reals[n].ckpt_off = ko;
    reals[n].gid = n;
    so += L * L; bo += L * (L + 1); ro += L;
    co += cache_rows(int(L), cfg->ckpt_every) * L;
    if (cfg->ckpt_every > 0 && cfg->prec == TNMC_MIXED) ko += int64_t((L + cfg->ckpt_every - 1) / cfg->ckpt_every) * L;
  }
  std::vector<int32_t> order(cfg->n_real);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return cfg->L[a] > cfg->L[b]; });

  Layout &lay = h->lay;
  lay.reals = reinterpret_cast<const RealInfo *>(ws + p.off_reals);
  lay.order = reinterpret_cast<const int32_t *>(ws + p.off_order);
  lay.n_real = cfg->n_real;
  lay.chi = cfg->chi;
  lay.L_max = p.L_max;
  lay.max_samples = cfg->max_samples;
  lay.beta = cfg->beta;
  lay.cutoff = cfg->cutoff > 0 ? cfg->cutoff : default_cutoff(cfg->prec);
  lay.jr = reinterpret_cast<float *>(ws + p.off_jr);
  lay.jd = reinterpret_cast<float *>(ws + p.off_jd);
  lay.cache = ws + p.off_cache;
  lay.ckpt_every = cfg->ckpt_every;
  lay.seg_begin = -1;
  lay.seg_end = 0;
  lay.wait_cycles = 0;
  lay.variant = 0;
  lay.tune_rows = 0;
  lay.tc_mode = tc_mode_of(cfg->prec);
  lay.ckpt64 = p.sum_ckpt > 0 ? reinterpret_cast<double *>(ws + p.off_ckpt64) : nullptr;
  lay.bonds = reinterpret_cast<int2 *>(ws + p.off_bonds);
  lay.lam = reinterpret_cast<double *>(ws + p.off_lam);
  lay.flags = reinterpret_cast<int32_t *>(ws + p.off_flags);
  lay.counter = reinterpret_cast<int32_t *>(ws + p.off_counter);
  lay.env_scratch = ws + p.off_env;
  lay.env_slot_bytes = p.env_slot;
  lay.env_slots = p.env_slots;
  lay.samp_scratch = ws + p.off_samp;
  lay.mlp = nullptr;
  lay.dbg_logits = nullptr;
  lay.dbg_spectra = nullptr;
  lay.dbg_rowinfo = nullptr;

  cudaError_t e = cudaMemcpyAsync(ws + p.off_reals, reals.data(), reals.size() * sizeof(RealInfo),
                                  cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ws + p.off_order, order.data(), order.size() * 4, cudaMemcpyHostToDevice,
                        h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(ws + p.off_flags, 0, size_t(cfg->n_real) * 4, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    delete h;
    return TNMC_ERR_CUDA;
  }
  h->reals = std::move(reals);
  *out = h;
  return TNMC_OK;
}

void tnmc_destroy(tnmc_handle *h) { delete h; }

tnmc_status tnmc_set_diagnostics(tnmc_handle *h, float *d_logits, double *d_spectra,
                                 double *d_rowinfo) {
  if (!h) return TNMC_ERR_ARG;
  if (h->q > 2 && (d_logits || d_spectra)) return TNMC_ERR_UNSUPPORTED;   // Potts: row records only
  h->lay.dbg_logits = d_logits;
  h->lay.dbg_spectra = d_spectra;
  h->lay.dbg_rowinfo = d_rowinfo;
  return TNMC_OK;
}

tnmc_status tnmc_set_correction(tnmc_handle *h, const void *d_params_bf16, int32_t enabled) {
  if (!h) return TNMC_ERR_ARG;
  if (h->q > 2 && enabled) return TNMC_ERR_UNSUPPORTED;
  if (!enabled) {
    h->lay.mlp = nullptr;
    return TNMC_OK;
  }
  if (!d_params_bf16 || (reinterpret_cast<uintptr_t>(d_params_bf16) & 15) != 0) return TNMC_ERR_ARG;
  h->lay.mlp = static_cast<const uint16_t *>(d_params_bf16);
  return TNMC_OK;
}

tnmc_status tnmc_mlp_features(tnmc_handle *h, int32_t S, const uint8_t *d_spins,
                              const float *d_logits, float *d_feat) {
  if (!h || !d_spins || !d_logits || !d_feat || S < 1) return TNMC_ERR_ARG;
  if ((reinterpret_cast<uintptr_t>(d_feat) & 15) != 0) return TNMC_ERR_ARG;
  if (h->q > 2) return TNMC_ERR_UNSUPPORTED;
  if (!h->built) return TNMC_ERR_STATE;   // the couplings are copied in by tnmc_build_envs
  return launch_mlp_features(h->lay, S, h->plan.L_max, d_spins, d_logits, d_feat, h->stream) ==
                 cudaSuccess
             ? TNMC_OK
             : TNMC_ERR_CUDA;
}

tnmc_status tnmc_set_realization_ids(tnmc_handle *h, const int64_t *h_ids) {
  if (!h) return TNMC_ERR_ARG;
  for (int n = 0; n < h->cfg.n_real; ++n) {
    const int64_t id = h_ids ? h_ids[n] : n;
    if (id < 0) return TNMC_ERR_ARG;
    h->reals[n].gid = id;
  }
  // the table is read by later launches on this stream; the host copy lives in the handle
  const cudaError_t e = cudaMemcpyAsync(const_cast<RealInfo *>(h->lay.reals), h->reals.data(),
                                        h->reals.size() * sizeof(RealInfo), cudaMemcpyHostToDevice,
                                        h->stream);
  if (e == cudaSuccess) return cudaStreamSynchronize(h->stream) == cudaSuccess ? TNMC_OK : TNMC_ERR_CUDA;
  return TNMC_ERR_CUDA;
}

tnmc_status tnmc_set_build_variant(tnmc_handle *h, int32_t variant) {
  if (!h || variant < 0 || variant > 63 || (variant & 3) == 3) return TNMC_ERR_ARG;
  h->lay.variant = variant;
  return TNMC_OK;
}

int32_t tnmc_get_build_variant(const tnmc_handle *h) { return h ? h->lay.variant : -1; }

tnmc_status tnmc_autotune_build(tnmc_handle *h, const float *d_J, int32_t rows, int32_t *h_variants,
                                float *h_ms, int32_t *h_count) {
  if (!h || !d_J || rows < 1 || !h_count) return TNMC_ERR_ARG;
  if (h->q > 2) return TNMC_ERR_UNSUPPORTED;
  // candidate layouts of this precision (env_build.cu, VARIANT_*)
  std::vector<int32_t> cand;
  if (h->env_code == 0 || h->env_code == 3) cand = {0, 1, 2, 4, 4 | 8};
  else if (h->env_code == 1)   // one CTA, or pairs (bit 4); with or without the QR preconditioning (bit 5)
    cand = {0, 8, 16, 16 | 1, 16 | 2, 32, 32 | 8};
  else cand = {0, 8};
  // The candidates are timed on the `rows` rows below the middle of the smallest lattice,
  // rebuilt from the cached row under them: those rows carry the bond dimensions of the
  // whole build, while the bottom rows' bonds are still small. The rows from the middle
  // down are built once first (untimed) unless the handle holds a full build already.
  // (Not with checkpoints, nor for MIXED, whose float64 carry between rows is not cached:
  // there the bottom rows are timed.)
  const int L_min = *std::min_element(h->L.begin(), h->L.end());
  const bool mid = h->cfg.ckpt_every == 0 && h->env_code != 2 && L_min >= 2 * rows + 2;
  cudaError_t e = launch_ingest(h->lay, d_J, h->stream);
  if (e == cudaSuccess && mid && !h->built) {
    Layout l0 = h->lay;
    l0.dbg_logits = nullptr; l0.dbg_spectra = nullptr; l0.dbg_rowinfo = nullptr;
    l0.seg_begin = L_min / 2;
    l0.seg_end = h->plan.L_max;   // every realization from its bottom row up to the middle
    e = launch_env_build(l0, h->env_code, h->plan.CH, h->stream);
  }
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&ev0);
  if (e == cudaSuccess) e = cudaEventCreate(&ev1);
  int best = -1;
  float best_ms = 0.f;
  for (size_t k = 0; k < cand.size() && e == cudaSuccess; ++k) {
    Layout l2 = h->lay;
    l2.variant = cand[k];
    l2.dbg_logits = nullptr; l2.dbg_spectra = nullptr; l2.dbg_rowinfo = nullptr;
    // an untimed one-row launch loads the kernel
    if (mid) { l2.seg_begin = L_min / 2 - 1; l2.seg_end = L_min / 2; }
    else l2.tune_rows = 1;
    e = launch_env_build(l2, h->env_code, h->plan.CH, h->stream);
    if (mid) { l2.seg_begin = L_min / 2 - rows; l2.seg_end = L_min / 2; }
    else l2.tune_rows = rows;
    if (e == cudaSuccess) e = cudaEventRecord(ev0, h->stream);
    if (e == cudaSuccess) e = launch_env_build(l2, h->env_code, h->plan.CH, h->stream);
    if (e == cudaSuccess) e = cudaEventRecord(ev1, h->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev0, ev1);
    if (e != cudaSuccess) break;
    if (h_variants && int(k) < *h_count) h_variants[k] = cand[k];
    if (h_ms && int(k) < *h_count) h_ms[k] = ms;
    if (best < 0 || ms < best_ms) { best = int(k); best_ms = ms; }
  }
  if (ev0) cudaEventDestroy(ev0);
  if (ev1) cudaEventDestroy(ev1);
  *h_count = int32_t(cand.size());
  if (e != cudaSuccess) return TNMC_ERR_CUDA;
  h->lay.variant = cand[best];
  h->built = false;   // the timed launches overwrote bottom rows of the cache
  return TNMC_OK;
}

tnmc_status tnmc_set_wait_budget(tnmc_handle *h, int64_t cycles) {
  if (!h || cycles < 0) return TNMC_ERR_ARG;
  h->lay.wait_cycles = cycles;
  return TNMC_OK;
}

tnmc_status tnmc_build_envs(tnmc_handle *h, const float *d_J) {
  if (!h || !d_J) return TNMC_ERR_ARG;
  cudaError_t e = launch_ingest(h->lay, d_J, h->stream);
  if (h->q > 2) {
    if (e == cudaSuccess) e = launch_potts_build(h->lay, h->q, h->prec_code, h->stream);
    if (e != cudaSuccess) return TNMC_ERR_CUDA;
    h->built = true;
    return TNMC_OK;
  }
  if (e == cudaSuccess && h->lay.dbg_spectra)
    e = cudaMemsetAsync(h->lay.dbg_spectra, 0,
                        size_t(h->plan.sum_bonds) * h->cfg.chi * sizeof(double), h->stream);
  if (e == cudaSuccess) e = launch_env_build(h->lay, h->env_code, h->plan.CH, h->stream);
  if (e != cudaSuccess) return TNMC_ERR_CUDA;
  h->built = true;
  return TNMC_OK;
}

tnmc_status tnmc_log_z(tnmc_handle *h, double *d_logz) {
  if (!h || !d_logz) return TNMC_ERR_ARG;
  if (!h->built) return TNMC_ERR_STATE;
  if (h->q > 2)
    return launch_potts_log_z(h->lay, h->q, h->prec_code, d_logz, h->stream) == cudaSuccess ? TNMC_OK
                                                                                           : TNMC_ERR_CUDA;
  return launch_log_z(h->lay, h->prec_code, d_logz, h->stream) == cudaSuccess ? TNMC_OK
                                                                               : TNMC_ERR_CUDA;
}

tnmc_status tnmc_propose(tnmc_handle *h, int32_t S, uint64_t seed, uint64_t prop_base,
                         uint8_t *d_spins, double *d_logq, double *d_E) {
  if (!h || !d_spins || !d_logq || !d_E) return TNMC_ERR_ARG;
  if (S < 1 || S > h->cfg.max_samples) return TNMC_ERR_ARG;
  if (!h->built) return TNMC_ERR_STATE;
  if (h->q > 2)
    return launch_potts_sample(h->lay, h->q, h->prec_code, S, seed, prop_base, nullptr, d_spins, d_logq,
                               d_E, h->stream) == cudaSuccess ? TNMC_OK : TNMC_ERR_CUDA;
  return for_segments(h, [&](const Layout &l) {
           return launch_propose(l, h->prec_code, h->plan.CH, S, seed, prop_base, d_spins, d_logq,
                                 d_E, h->stream);
         }) == cudaSuccess
             ? TNMC_OK
             : TNMC_ERR_CUDA;
}

tnmc_status tnmc_propose_static(tnmc_handle *h, int32_t S, uint64_t seed, uint64_t prop_base,
                                uint8_t *d_spins, double *d_logq, double *d_E) {
  if (!h || !d_spins || !d_logq || !d_E) return TNMC_ERR_ARG;
  if (S < 1) return TNMC_ERR_ARG;
  if (h->q > 2) return TNMC_ERR_UNSUPPORTED;
  if (!h->built) return TNMC_ERR_STATE;
  bool too_big = false;
  const int64_t esz = value_bytes(h->cfg.prec);
  if (int64_t(S) * h->plan.sum_L * h->plan.CH * esz > static_scratch_bytes()) return TNMC_ERR_ARG;
  const cudaError_t e = for_segments(h, [&](const Layout &l) {
    return launch_propose_static(l, h->prec_code, h->plan.CH, S, seed, prop_base, d_spins, d_logq,
                                 d_E, h->plan.sum_L, h->stream, &too_big);
  });
  if (too_big) return TNMC_ERR_ARG;
  return e == cudaSuccess ? TNMC_OK : TNMC_ERR_CUDA;
}

size_t tnmc_propose_static_limit(void) { return size_t(static_scratch_bytes()); }

tnmc_status tnmc_score(tnmc_handle *h, int32_t S, const uint8_t *d_spins, double *d_logq,
                       double *d_E) {
  if (!h || !d_spins || !d_logq || !d_E) return TNMC_ERR_ARG;
  if (S < 1 || S > h->cfg.max_samples) return TNMC_ERR_ARG;
  if (!h->built) return TNMC_ERR_STATE;
  if (h->q > 2)
    return launch_potts_sample(h->lay, h->q, h->prec_code, S, 0, 0, d_spins, nullptr, d_logq, d_E,
                               h->stream) == cudaSuccess ? TNMC_OK : TNMC_ERR_CUDA;
  return for_segments(h, [&](const Layout &l) {
           return launch_score(l, h->prec_code, h->plan.CH, S, d_spins, d_logq, d_E, h->stream);
         }) == cudaSuccess
             ? TNMC_OK
             : TNMC_ERR_CUDA;
}

tnmc_status tnmc_mh_init(tnmc_handle *h, uint64_t seed, uint8_t *d_state_spins,
                         double *d_state_logq, double *d_state_E) {
  if (!h || !d_state_spins || !d_state_logq || !d_state_E) return TNMC_ERR_ARG;
  if (h->q > 2) return TNMC_ERR_UNSUPPORTED;
  if (!h->built) return TNMC_ERR_STATE;
  cudaError_t e = launch_init_state(h->lay, seed, d_state_spins, h->stream);
  if (e == cudaSuccess)
    e = for_segments(h, [&](const Layout &l) {
      return launch_score(l, h->prec_code, h->plan.CH, 1, d_state_spins, d_state_logq, d_state_E,
                          h->stream);
    });
  return e == cudaSuccess ? TNMC_OK : TNMC_ERR_CUDA;
}

tnmc_status tnmc_observables(tnmc_handle *h, int32_t S, const uint8_t *d_spins,
                             const double *d_logq, const double *d_E, double *d_out) {
  if (!h || !d_spins || !d_logq || !d_E || !d_out || S < 1) return TNMC_ERR_ARG;
  if (h->q > 2) return TNMC_ERR_UNSUPPORTED;
  return launch_observables(h->lay, S, d_spins, d_logq, d_E, d_out, h->stream) == cudaSuccess
             ? TNMC_OK
             : TNMC_ERR_CUDA;
}

tnmc_status tnmc_mh_init_empty(tnmc_handle *h, uint8_t *d_state_spins, double *d_state_logq,
                               double *d_state_E) {
  if (!h || !d_state_spins || !d_state_logq || !d_state_E) return TNMC_ERR_ARG;
  cudaError_t e = cudaMemsetAsync(d_state_spins, 0, size_t(h->plan.sum_L2), h->stream);
  if (e == cudaSuccess) e = launch_empty_state(h->lay, d_state_logq, d_state_E, h->stream);
  return e == cudaSuccess ? TNMC_OK : TNMC_ERR_CUDA;
}

tnmc_status tnmc_mh_step(tnmc_handle *h, int32_t S, uint64_t seed, uint64_t prop_base,
                         const uint8_t *d_prop_spins, const double *d_prop_logq,
                         const double *d_prop_E, uint8_t *d_state_spins, double *d_state_logq,
                         double *d_state_E, uint8_t *d_accept, int64_t *d_n_accept) {
  if (!h || !d_prop_spins || !d_prop_logq || !d_prop_E || !d_state_spins || !d_state_logq ||
      !d_state_E || !d_accept || !d_n_accept)
    return TNMC_ERR_ARG;
  if (S < 1 || S > h->cfg.max_samples) return TNMC_ERR_ARG;
  return launch_mh(h->lay, S, seed, prop_base, d_prop_spins, d_prop_logq, d_prop_E, d_state_spins,
                   d_state_logq, d_state_E, d_accept, d_n_accept, h->stream) == cudaSuccess
             ? TNMC_OK
             : TNMC_ERR_CUDA;
}

tnmc_status tnmc_get_device_status(tnmc_handle *h, int32_t *h_flags, int32_t clear) {
  if (!h || !h_flags) return TNMC_ERR_ARG;
  cudaError_t e = cudaMemcpyAsync(h_flags, h->lay.flags, size_t(h->cfg.n_real) * 4,
                                  cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e == cudaSuccess && clear) {
    e = cudaMemsetAsync(h->lay.flags, 0, size_t(h->cfg.n_real) * 4, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  }
  if (e != cudaSuccess) return TNMC_ERR_CUDA;
  int32_t any = 0;
  for (int n = 0; n < h->cfg.n_real; ++n) any |= h_flags[n];
  if (any & FLAG_NUMERIC) return TNMC_ERR_NUMERIC;
  if (any & FLAG_TIMEOUT) return TNMC_ERR_TIMEOUT;
  if (any & FLAG_BAD_J) return TNMC_ERR_ARG;
  return TNMC_OK;
}

}  // extern "C"
