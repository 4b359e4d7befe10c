// Coupling ingest (Sec. 3.1 layout), log Z from the top-row environment
// (Eq. 6), the random initial state and the independence Metropolis-Hastings
// scan of Eq. 10.
#include "common.cuh"

namespace tnmc {

namespace {

// One CTA per realization: check the (L, L, 4) paper layout (left, up, right,
// down per site; zero on open boundaries; shared bonds equal on both sides;
// finite) and keep the right and down couplings of every site.
__global__ void ingest_kernel(Layout lay, const float *J) {
  const int n = blockIdx.x;
  const RealInfo ri = lay.reals[n];
  const int L = ri.L;
  const float *Jn = J + 4 * ri.site_off;
  __shared__ int bad;
  if (threadIdx.x == 0) {
    bad = 0;
    atomicAnd(lay.flags + n, ~FLAG_BAD_J);
  }
  __syncthreads();
  int my_bad = 0;
  for (int s = threadIdx.x; s < L * L; s += blockDim.x) {
    const int r = s / L, c = s % L;
    const float lf = Jn[4 * s + 0], up = Jn[4 * s + 1], rt = Jn[4 * s + 2], dn = Jn[4 * s + 3];
    if (!isfinite(lf) || !isfinite(up) || !isfinite(rt) || !isfinite(dn)) my_bad = 1;
    if (c == 0 && lf != 0.f) my_bad = 1;
    if (r == 0 && up != 0.f) my_bad = 1;
    if (c == L - 1 && rt != 0.f) my_bad = 1;
    if (r == L - 1 && dn != 0.f) my_bad = 1;
    if (c < L - 1 && rt != Jn[4 * (s + 1) + 0]) my_bad = 1;
    if (r < L - 1 && dn != Jn[4 * (s + L) + 1]) my_bad = 1;
    lay.jr[ri.site_off + s] = rt;
    lay.jd[ri.site_off + s] = dn;
  }
  if (my_bad) bad = 1;
  __syncthreads();
  if (threadIdx.x == 0 && bad) set_flag(lay.flags, n, FLAG_BAD_J);
}

// One warp per realization, float64: Z = exp(lambda_0) sum_s F_0(s). Summing
// the physical leg of a parity-form site gives 2 A(+); starting from the even
// trivial bond only the even-even blocks contribute.
template <typename T>
__global__ void log_z_kernel(Layout lay, double *logz) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  if (warp >= lay.n_real) return;
  const int n = warp;
  extern __shared__ double vsh[];          // per warp: 2 x 64
  double *v = vsh + wib * 128, *vn = v + 64;
  const RealInfo ri = lay.reals[n];
  const int L = ri.L, chi = lay.chi;
  const T *C0 = (const T *)lay.cache + ri.cache_off * int64_t(chi) * chi;   // row 0 (slot 0)
  const int2 *bd = lay.bonds + ri.bond_off;                                // row 0 bonds
  for (int a = lane; a < 64; a += 32) v[a] = (a == 0) ? 1.0 : 0.0;
  __syncwarp();
  double lacc = 0.0;
  for (int c = 0; c < L; ++c) {
    const int el = bd[c].x, er = bd[c + 1].x;
    const T *C = C0 + int64_t(c) * chi * chi;
    double s2 = 0.0;
    for (int b = lane; b < 64; b += 32) {
      double acc = 0.0;
      if (b < er)
        for (int a = 0; a < el; ++a) acc += v[a] * 2.0 * (double)C[a * chi + b];
      vn[b] = acc;
      s2 += acc * acc;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    const double nrm = sqrt(s2);
    __syncwarp();
    for (int b = lane; b < 64; b += 32) v[b] = nrm > 0.0 ? vn[b] / nrm : 0.0;
    lacc += log(nrm);
    __syncwarp();
  }
  if (lane == 0) {
    const double val = lay.lam[ri.row_off + 0] + lacc + log(fabs(v[0]) > 0 ? fabs(v[0]) : 0.0);
    logz[n] = val;
    if (!isfinite(val)) set_flag(lay.flags, n, FLAG_NUMERIC);
  }
}

// Random initial configuration: spin bit = top bit of the Philox word of
// counter (i >> 2, 0, gid, 2), word i & 3 (gid: the realization's stream id).
__global__ void init_state_kernel(Layout lay, uint64_t seed, uint8_t *spins) {
  const int n = blockIdx.x;
  const RealInfo ri = lay.reals[n];
  const int64_t L2 = int64_t(ri.L) * ri.L;
  for (int64_t g = threadIdx.x; g < (L2 + 3) / 4; g += blockDim.x) {
    const U64x4 w = philox4x64_10((uint64_t)g, 0ull, (uint64_t)ri.gid, TAG_INIT, seed, 0ull);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t i = 4 * g + q;
      if (i < L2) spins[ri.site_off + i] = (uint8_t)(w.x[q] >> 63);
    }
  }
}

// One CTA per realization: the chain consumes the S proposals in id order.
__global__ void mh_kernel(Layout lay, int S, uint64_t seed, uint64_t base, const uint8_t *p_spins,
                          const double *p_logq, const double *p_E, uint8_t *st_spins,
                          double *st_logq, double *st_E, uint8_t *accept, int64_t *n_accept) {
  const int n = blockIdx.x;
  const RealInfo ri = lay.reals[n];
  const int64_t L2 = int64_t(ri.L) * ri.L;
  __shared__ int last;
  if (threadIdx.x == 0) {
    const double nb = -lay.beta;
    double lq = st_logq[n], E = st_E[n];
    int lst = -1;
    int64_t cnt = 0;
    for (int t = 0; t < S; ++t) {
      const double Ep = p_E[int64_t(n) * S + t], lqp = p_logq[int64_t(n) * S + t];
      const double a = __dsub_rn(__dmul_rn(nb, Ep), lqp);
      const double b = __dsub_rn(__dmul_rn(nb, E), lq);
      const double lr = __dsub_rn(a, b);
      const U64x4 w = philox4x64_10(0ull, base + (uint64_t)t, (uint64_t)ri.gid, TAG_MH, seed, 0ull);
      const double u = word_to_uniform(w.x[0]);
      const int acc = log(u) < lr ? 1 : 0;
      accept[int64_t(n) * S + t] = (uint8_t)acc;
      if (acc) { lst = t; lq = lqp; E = Ep; ++cnt; }
    }
    st_logq[n] = lq;
    st_E[n] = E;
    n_accept[n] += cnt;
    last = lst;
  }
  __syncthreads();
  if (last >= 0) {
    const uint8_t *src = p_spins + int64_t(S) * ri.site_off + int64_t(last) * L2;
    uint8_t *dst = st_spins + ri.site_off;
    for (int64_t i = threadIdx.x; i < L2; i += blockDim.x) dst[i] = src[i];
  }
}

}  // namespace

cudaError_t launch_ingest(const Layout &lay, const float *J, cudaStream_t st) {
  ingest_kernel<<<lay.n_real, 256, 0, st>>>(lay, J);
  return cudaGetLastError();
}

cudaError_t launch_log_z(const Layout &lay, int prec, double *logz, cudaStream_t st) {
  const int wpb = 4;
  const int blocks = (lay.n_real + wpb - 1) / wpb;
  const size_t smem = wpb * 128 * sizeof(double);
  if (prec == 0) log_z_kernel<double><<<blocks, 32 * wpb, smem, st>>>(lay, logz);
  else if (prec == 2) log_z_kernel<dfloat><<<blocks, 32 * wpb, smem, st>>>(lay, logz);
  else log_z_kernel<float><<<blocks, 32 * wpb, smem, st>>>(lay, logz);
  return cudaGetLastError();
}

// Importance-sampling observables of each realization's S proposals, with weights
// w_k = exp(-beta E_k - log q_k) (Eq. 1, Eq. 9; the ratio of Eq. 10): log mean w,
// the effective sample size (sum w)^2 / sum w^2, <E>/N, and over the proposal
// pairs (2k, 2k+1) with pair weights w_a w_b the overlap moments <q^2>, <q^4> of
// q_ab = (1/N) sum_i s_i^a s_i^b and the Binder ratio (3 - <q^4>/<q^2>^2) / 2.
// One CTA per realization; every sum in a fixed order.
constexpr int OBS_THREADS = 256;

__device__ __forceinline__ double block_sum(double v, double *red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < OBS_THREADS / 32; ++w) t += red[w];
  return t;
}

__global__ void observables_kernel(Layout lay, int S, const uint8_t *spins, const double *logq,
                                   const double *E, double *out) {
  __shared__ double red[OBS_THREADS / 32];
  __shared__ double sh_m;
  const int n = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const RealInfo ri = lay.reals[n];
  const int64_t N = int64_t(ri.L) * ri.L;
  const double beta = lay.beta;
  const double *lq = logq + int64_t(n) * S, *en = E + int64_t(n) * S;
  // the largest log weight (log-domain shift)
  double m = -INFINITY;
  for (int k = tid; k < S; k += OBS_THREADS) m = fmax(m, -beta * en[k] - lq[k]);
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) red[warp] = m;
  __syncthreads();
  if (tid == 0) {
    double t = red[0];
    for (int w = 1; w < OBS_THREADS / 32; ++w) t = fmax(t, red[w]);
    sh_m = t;
  }
  __syncthreads();
  m = sh_m;
  double sw = 0.0, sw2 = 0.0, swe = 0.0;
  for (int k = tid; k < S; k += OBS_THREADS) {
    const double w = exp(-beta * en[k] - lq[k] - m);
    sw += w; sw2 += w * w; swe += w * en[k];
  }
  sw = block_sum(sw, red);
  sw2 = block_sum(sw2, red);
  swe = block_sum(swe, red);
  // replica pairs: one warp per pair counts the differing spins
  double sp = 0.0, sq2 = 0.0, sq4 = 0.0;
  const uint8_t *base = spins + int64_t(S) * ri.site_off;
  for (int p = warp; p < S / 2; p += OBS_THREADS / 32) {
    const uint8_t *a = base + int64_t(2 * p) * N, *b = a + N;
    int64_t diff = 0;
    for (int64_t i = lane; i < N; i += 32) diff += (a[i] != b[i]);
    for (int o = 16; o > 0; o >>= 1) diff += __shfl_xor_sync(0xffffffffu, diff, o);
    if (lane == 0) {
      const double q = double(N - 2 * diff) / double(N);
      const double wp = exp(-beta * en[2 * p] - lq[2 * p] - m) * exp(-beta * en[2 * p + 1] - lq[2 * p + 1] - m);
      sp += wp; sq2 += wp * q * q; sq4 += wp * q * q * q * q;
    }
  }
  sp = block_sum(sp, red);
  sq2 = block_sum(sq2, red);
  sq4 = block_sum(sq4, red);
  if (tid == 0) {
    double *o = out + int64_t(n) * 6;
    o[0] = m + log(sw / double(S));
    o[1] = sw * sw / sw2;
    o[2] = swe / sw / double(N);
    const double q2 = sq2 / sp, q4 = sq4 / sp;
    o[3] = S >= 2 ? q2 : NAN;
    o[4] = S >= 2 ? q4 : NAN;
    o[5] = S >= 2 ? 0.5 * (3.0 - q4 / (q2 * q2)) : NAN;
  }
}

cudaError_t launch_observables(const Layout &lay, int S, const uint8_t *spins, const double *logq,
                               const double *E, double *out, cudaStream_t st) {
  observables_kernel<<<lay.n_real, OBS_THREADS, 0, st>>>(lay, S, spins, logq, E, out);
  return cudaGetLastError();
}

// A chain with no state yet: log q = +inf makes log r = +inf for the first
// proposal, which is therefore accepted, so the chain starts at a draw of q.
__global__ void empty_state_kernel(int n_real, double *logq, double *E) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n < n_real) {
    logq[n] = __longlong_as_double(0x7ff0000000000000ll);   // +inf
    E[n] = 0.0;
  }
}

cudaError_t launch_empty_state(const Layout &lay, double *logq, double *E, cudaStream_t st) {
  empty_state_kernel<<<(lay.n_real + 255) / 256, 256, 0, st>>>(lay.n_real, logq, E);
  return cudaGetLastError();
}

cudaError_t launch_init_state(const Layout &lay, uint64_t seed, uint8_t *spins, cudaStream_t st) {
  init_state_kernel<<<lay.n_real, 256, 0, st>>>(lay, seed, spins);
  return cudaGetLastError();
}

cudaError_t launch_mh(const Layout &lay, int S, uint64_t seed, uint64_t base, const uint8_t *ps,
                      const double *pl, const double *pe, uint8_t *ss, double *sl, double *se,
                      uint8_t *acc, int64_t *nacc, cudaStream_t st) {
  mh_kernel<<<lay.n_real, 256, 0, st>>>(lay, S, seed, base, ps, pl, pe, ss, sl, se, acc, nacc);
  return cudaGetLastError();
}

}  // namespace tnmc
