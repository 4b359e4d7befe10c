// Row-by-row ancestral proposals and teacher-forced scoring (Sec. 3.3,
// Eq. 4-5, Eq. 9), batched over realizations x samples (Sec. 3.4).
//
// A CTA owns 64 chains (samples) of one realization and walks the rows top to
// bottom. For each row it runs
//   right pass  c = L-2 .. 0 : R_c = T_{c+1}[s_up(c+1)] R_{c+1}, normalised,
//                spilled to the sampler scratch;
//   left pass   c = 0 .. L-1 : rho_s = | l M_c[s] R_c |, logit of Eq. 5, the
//                Philox draw, log q (Eq. 9) and the energy (Eq. 1).
// In parity form (common.cuh) M_c[s] = Pi^s C_c Pi^s, so with u = l_even C
// and w = l_odd C (one chi x chi pass over C for both spin values):
//   rho_0 = |(u + w) . R|,  rho_1 = |(u - w) . Pi R|,
//   new l = u + w (s = -1) or Pi (u - w) (s = +1);
// and the fold of the vertical bond into the column on the right is
//   T_c[s] = Pi^s D_c Pi^s,  D_c = C_c with odd blocks scaled by tanh(beta Jv),
// (all-ones bond, t = 0, on the top row). The per-site work is a small GEMM
// over the CTA's chains: each thread holds a 4 chains x 4 columns register
// tile and streams C (staged in shared memory, double-buffered) against the
// chains' vectors (shared memory, chain-minor).
//
// With the learned correction on (CORR, Layout::mlp) a 7 -> 64 -> 64 -> 1
// network adds its output to each logit before the draw (mlp.cuh); the shifted
// logit defines q, so log q stays exact. With checkpointed environments a launch
// walks one segment of rows (Layout::seg_begin, seg_end) and resumes from the
// spins, log q and energies that the segment above left.
#include "common.cuh"
#include "mlp.cuh"

#include <mutex>
#include <type_traits>

namespace tnmc {

namespace {

constexpr int SB = 64;   // chains per CTA
constexpr int TS = 4;    // chains per thread tile
constexpr int TC = 4;    // columns per thread tile

template <typename T> struct Vec4;
template <> struct Vec4<float> {
  static __device__ __forceinline__ void load(const float *p, float v[4]) {
    const float4 x = *reinterpret_cast<const float4 *>(p);
    v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
  }
  static __device__ __forceinline__ void store(float *p, const float v[4]) {
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
  }
};
template <> struct Vec4<dfloat> {
  static __device__ __forceinline__ void load(const dfloat *p, dfloat v[4]) {
    const float4 x = reinterpret_cast<const float4 *>(p)[0];
    const float4 y = reinterpret_cast<const float4 *>(p)[1];
    v[0] = dfloat(x.x, x.y); v[1] = dfloat(x.z, x.w); v[2] = dfloat(y.x, y.y); v[3] = dfloat(y.z, y.w);
  }
  static __device__ __forceinline__ void store(dfloat *p, const dfloat v[4]) {
    reinterpret_cast<float4 *>(p)[0] = make_float4(v[0].hi, v[0].lo, v[1].hi, v[1].lo);
    reinterpret_cast<float4 *>(p)[1] = make_float4(v[2].hi, v[2].lo, v[3].hi, v[3].lo);
  }
};
template <> struct Vec4<double> {
  static __device__ __forceinline__ void load(const double *p, double v[4]) {
    const double2 x = reinterpret_cast<const double2 *>(p)[0];
    const double2 y = reinterpret_cast<const double2 *>(p)[1];
    v[0] = x.x; v[1] = x.y; v[2] = y.x; v[3] = y.y;
  }
  static __device__ __forceinline__ void store(double *p, const double v[4]) {
    reinterpret_cast<double2 *>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2 *>(p)[1] = make_double2(v[2], v[3]);
  }
};

template <int CH>
struct SampPlan {
  static constexpr int NCG = CH / TC;           // column groups
  static constexpr int NT = (SB / TS) * NCG;    // threads
  static constexpr int LDC = CH + 4;            // padded row of the staged site matrix
  static constexpr int OWN = (TS + NCG - 1) / NCG;  // chains whose scalars a lane owns
};

template <typename T, int CH>
__host__ __device__ constexpr int64_t samp_smem_fixed() {
  return int64_t(2 * CH * SampPlan<CH>::LDC + 2 * CH * SB) * sizeof(T);
}

template <typename T, int W>
__device__ __forceinline__ T gsum(T v) {
#pragma unroll
  for (int o = W / 2; o > 0; o >>= 1) v += shfl_xor(v, o);
  return v;
}

// acc += x * y: a fused multiply-add in float32 and float64, the double-float one in
// double-float arithmetic
__device__ __forceinline__ void fma_acc(float &acc, float x, float y) { acc += x * y; }
__device__ __forceinline__ void fma_acc(double &acc, double x, double y) { acc += x * y; }
__device__ __forceinline__ void fma_acc(dfloat &acc, dfloat x, dfloat y) { df::dot_step(acc, x, y); }
// a finished accumulator (double-float sums are kept unnormalised while they run)
__device__ __forceinline__ float fin(float a) { return a; }
__device__ __forceinline__ double fin(double a) { return a; }
__device__ __forceinline__ dfloat fin(dfloat a) { return df::finish(a); }

// Arithmetic of the per-draw scalars (logit, log sigmoid, the draw): the tensor type,
// except for double-float tensors, whose scalars are float64
template <typename T> struct LogitType { using type = T; };
template <> struct LogitType<dfloat> { using type = double; };

template <typename T, int CH, bool FORCED, bool CORR>
__global__ void __launch_bounds__(SampPlan<CH>::NT)
sample_kernel(Layout lay, int S, uint64_t seed, uint64_t prop_base, const uint8_t *in_spins,
              uint8_t *out_spins, double *out_logq, double *out_E) {
  using P = SampPlan<CH>;
  constexpr int NCG = P::NCG, LDC = P::LDC, OWN = P::OWN;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *Cs = (T *)smem_raw;                       // 2 x CH x LDC
  T *Vb = Cs + 2 * CH * LDC;                   // 2 x CH x SB
  const int bpr = (S + SB - 1) / SB;
  const int n = lay.order[blockIdx.x / bpr];
  const int sblk = blockIdx.x % bpr;
  const RealInfo ri = lay.reals[n];
  const int L = ri.L;
  const int WL = (L + 31) / 32;
  uint32_t *bits = (uint32_t *)(Vb + 2 * CH * SB);   // 2 x SB x WL
  // learned correction (optional): staged network, per-chain logits and shifts
  MlpSmem *mp = (MlpSmem *)(bits + 2 * SB * WL);
  float *sh_lg = (float *)(mp + 1);
  float *sh_dl = sh_lg + SB;
  constexpr bool corr = CORR;   // the learned correction is on (lay.mlp != null)
  const int chi = lay.chi;
  const int tid = threadIdx.x, cg = tid % NCG, sg = tid / NCG;
  const int lane = tid & 31;
  const int gbase = lane - cg;                  // first lane of this chain group
  const float *jr = lay.jr + ri.site_off, *jd = lay.jd + ri.site_off;
  const T *cache_n = (const T *)lay.cache + ri.cache_off * int64_t(chi) * chi;
  // rows of this launch: all, or one segment [r_begin, r_end) whose chains
  // continue from the spins, log q and energies written by the segment above
  const int r_begin = lay.seg_begin < 0 ? 0 : lay.seg_begin;
  const int r_end = lay.seg_begin < 0 ? L : min(lay.seg_end, L);
  if (r_begin >= r_end) return;   // uniform over the CTA: no row of this realization
  const int2 *bonds_n = lay.bonds + ri.bond_off;
  T *rs = (T *)lay.samp_scratch + ri.line_off * int64_t(lay.max_samples) * CH;
  const int64_t L2 = int64_t(L) * L;
  const T beta = T(lay.beta);

  int sid[TS];        // global chain index in this realization
  bool act[TS];
#pragma unroll
  for (int j = 0; j < TS; ++j) { sid[j] = sblk * SB + sg * TS + j; act[j] = sid[j] < S; }

  // scalars of the chains this lane owns (chain j owned by lane cg == j % NCG)
  double lq[OWN], en[OWN];
  int sleft[OWN];
  uint64_t pw[OWN][4];
  int64_t pg[OWN];
#pragma unroll
  for (int o = 0; o < OWN; ++o) { lq[o] = 0.0; en[o] = 0.0; sleft[o] = 0; pg[o] = -1; }

  uint32_t *bprev = bits, *bcur = bits + SB * WL;
  for (int e = tid; e < 2 * SB * WL; e += P::NT) bits[e] = 0u;
  if (corr) mlp_stage(mp, lay.mlp, tid, P::NT);
  bool any_bad = false;
  __syncthreads();
  if (r_begin > 0) {
    // resume: the row above from the spins written (or given) so far, and the sums
    const uint8_t *sp = FORCED ? in_spins : out_spins;
#pragma unroll
    for (int o = 0; o < OWN; ++o) {
      const int j = cg + o * NCG;
      if (j < TS && act[j]) {
        const uint8_t *row = sp + int64_t(S) * ri.site_off + int64_t(sid[j]) * L2 + int64_t(r_begin - 1) * L;
        uint32_t *bw = bprev + (sg * TS + j) * WL;
        for (int c = 0; c < L; ++c)
          if (row[c]) bw[c >> 5] |= 1u << (c & 31);
        lq[o] = out_logq[int64_t(n) * S + sid[j]];
        en[o] = out_E[int64_t(n) * S + sid[j]];
      }
    }
    __syncthreads();
  }

  for (int r = r_begin; r < r_end; ++r) {
    const int2 *bd = bonds_n + int64_t(r) * (L + 1);
    const T *crow = cache_n + cache_slot(r, L, lay.ckpt_every, lay.seg_begin) * L * chi * chi;
    // chain-owner lanes clear this row's bits
#pragma unroll
    for (int o = 0; o < OWN; ++o) {
      const int j = cg + o * NCG;
      if (j < TS)
        for (int w = 0; w < WL; ++w) bcur[(sg * TS + j) * WL + w] = 0u;
    }
    // ===================== right pass
    // R_{L-1} = e_0 on the trivial bond L
    for (int e = tid; e < CH * SB; e += P::NT) Vb[e] = (e < SB) ? T(1) : T(0);
    int buf = 0;
    for (int c = L - 2; c >= 0; --c) {
      // stage D_{c+1}^T: Cs[b][a] = C_{c+1}[a][b] * (t_v on odd blocks)
      const int2 bl = bd[c + 1], br = bd[c + 2];
      const T tv = (r > 0) ? Num<T>::tanh_(beta * T(jd[(r - 1) * L + c + 1])) : T(0);
      T *cs = Cs + buf * CH * LDC;
      const T *src = crow + int64_t(c + 1) * chi * chi;
      // only the D_l x D_r block is read: the cache is zero outside the bond dimensions
      const int Dl1 = bl.x + bl.y, Dr1 = br.x + br.y;
      for (int e = tid; e < CH * CH; e += P::NT) {
        const int a = e / CH, b = e % CH;
        T v = (a < Dl1 && b < Dr1) ? src[a * chi + b] : T(0);
        if ((a >= bl.x) != (b >= br.x)) v *= tv;
        cs[b * LDC + a] = v;
      }
      __syncthreads();
      const T *vin = Vb + buf * CH * SB;
      T acc[TS][TC];
#pragma unroll
      for (int j = 0; j < TS; ++j)
#pragma unroll
        for (int t = 0; t < TC; ++t) acc[j][t] = T(0);
      const int Dr = br.x + br.y;
      for (int b = 0; b < Dr; ++b) {
        T x[TS], y[TC];
        Vec4<T>::load(vin + b * SB + sg * TS, x);
        Vec4<T>::load(cs + b * LDC + cg * TC, y);
#pragma unroll
        for (int j = 0; j < TS; ++j)
#pragma unroll
          for (int t = 0; t < TC; ++t) fma_acc(acc[j][t], x[j], y[t]);
      }
#pragma unroll
      for (int j = 0; j < TS; ++j)
#pragma unroll
        for (int t = 0; t < TC; ++t) acc[j][t] = fin(acc[j][t]);
      // output sign Pi^{s_up(c+1)} on bond c+1, then normalise over the bond
      T *vout = Vb + (buf ^ 1) * CH * SB;
#pragma unroll
      for (int j = 0; j < TS; ++j) {
        const int sl = sg * TS + j;
        const int up1 = (r > 0) ? (bprev[sl * WL + ((c + 1) >> 5)] >> ((c + 1) & 31)) & 1 : 0;
        const int up0 = (r > 0) ? (bprev[sl * WL + (c >> 5)] >> (c & 31)) & 1 : 0;
        T nrm = 0;
#pragma unroll
        for (int t = 0; t < TC; ++t) {
          const int a = cg * TC + t;
          if (up1 && a >= bl.x) acc[j][t] = -acc[j][t];
          nrm += acc[j][t] * acc[j][t];
        }
        nrm = gsum<T, NCG>(nrm);
        const T inv = nrm > T(0) ? T(1) / Num<T>::sqrt_(nrm) : T(0);
        if (!(nrm > T(0)) && act[j]) any_bad = true;
        T outv[TC], flp[TC];
#pragma unroll
        for (int t = 0; t < TC; ++t) {
          const int a = cg * TC + t;
          outv[t] = acc[j][t] * inv;
          flp[t] = (up0 && a >= bl.x) ? -outv[t] : outv[t];   // input flip of the next step
        }
        // columns past bond c+1's dimension are zero: not spilled (the left pass reads zeros)
        if (act[j] && cg * TC < Dl1)
          Vec4<T>::store(rs + (int64_t(c) * lay.max_samples + sid[j]) * CH + cg * TC, outv);
#pragma unroll
        for (int t = 0; t < TC; ++t) vout[(cg * TC + t) * SB + sl] = flp[t];
      }
      buf ^= 1;
    }
    __syncthreads();
    // ===================== left pass
    for (int e = tid; e < CH * SB; e += P::NT) Vb[e] = (e < SB) ? T(1) : T(0);   // l = e_0
    buf = 0;
    for (int c = 0; c < L; ++c) {
      const int2 bl = bd[c], br = bd[c + 1];
      T *cs = Cs + buf * CH * LDC;
      const T *src = crow + int64_t(c) * chi * chi;
      const int Dlc = bl.x + bl.y, Drc = br.x + br.y;
      for (int e = tid; e < CH * CH; e += P::NT) {
        const int a = e / CH, b = e % CH;
        cs[a * LDC + b] = (a < Dlc && b < Drc) ? src[a * chi + b] : T(0);
      }
      // right environment tile of this thread
      T R[TS][TC];
#pragma unroll
      for (int j = 0; j < TS; ++j) {
        if (c < L - 1 && act[j] && cg * TC < Drc) {
          Vec4<T>::load(rs + (int64_t(c) * lay.max_samples + sid[j]) * CH + cg * TC, R[j]);
        } else {
#pragma unroll
          for (int t = 0; t < TC; ++t) R[j][t] = (c == L - 1 && cg * TC + t == 0) ? T(1) : T(0);
        }
      }
      __syncthreads();
      const T *vin = Vb + buf * CH * SB;
      T u[TS][TC], w[TS][TC];
#pragma unroll
      for (int j = 0; j < TS; ++j)
#pragma unroll
        for (int t = 0; t < TC; ++t) { u[j][t] = T(0); w[j][t] = T(0); }
      for (int a = 0; a < bl.x; ++a) {
        T x[TS], y[TC];
        Vec4<T>::load(vin + a * SB + sg * TS, x);
        Vec4<T>::load(cs + a * LDC + cg * TC, y);
#pragma unroll
        for (int j = 0; j < TS; ++j)
#pragma unroll
          for (int t = 0; t < TC; ++t) fma_acc(u[j][t], x[j], y[t]);
      }
      const int Dl = bl.x + bl.y;
      for (int a = bl.x; a < Dl; ++a) {
        T x[TS], y[TC];
        Vec4<T>::load(vin + a * SB + sg * TS, x);
        Vec4<T>::load(cs + a * LDC + cg * TC, y);
#pragma unroll
        for (int j = 0; j < TS; ++j)
#pragma unroll
          for (int t = 0; t < TC; ++t) fma_acc(w[j][t], x[j], y[t]);
      }
#pragma unroll
      for (int j = 0; j < TS; ++j)
#pragma unroll
        for (int t = 0; t < TC; ++t) { u[j][t] = fin(u[j][t]); w[j][t] = fin(w[j][t]); }
      // conditional weights, reduced over the column groups
      T x0[TS], x1[TS];
#pragma unroll
      for (int j = 0; j < TS; ++j) {
        T p0 = 0, p1 = 0;
#pragma unroll
        for (int t = 0; t < TC; ++t) {
          const int b = cg * TC + t;
          const T pr = (b >= br.x) ? -R[j][t] : R[j][t];
          p0 += (u[j][t] + w[j][t]) * R[j][t];
          p1 += (u[j][t] - w[j][t]) * pr;
        }
        x0[j] = gsum<T, NCG>(p0);
        x1[j] = gsum<T, NCG>(p1);
      }
      // owners: logit, draw, log q, energy
      const int i = r * L + c;
      const T jup = (r > 0) ? T(jd[(r - 1) * L + c]) : T(0);
      const double jl = (c > 0) ? (double)jr[r * L + c - 1] : 0.0;
      using TL = typename LogitType<T>::type;
      const TL betaL = std::is_same<T, dfloat>::value ? TL(lay.beta) : TL(beta);
      TL lg_own[OWN];
#pragma unroll
      for (int o = 0; o < OWN; ++o) {
        const int j = cg + o * NCG;
        lg_own[o] = TL(0);
        if (j < TS) {
          const int sl = sg * TS + j;
          const int up = (r > 0) ? (bprev[sl * WL + (c >> 5)] >> (c & 31)) & 1 : 0;
          const TL rho0 = TL(fabs(x0[j])), rho1 = TL(fabs(x1[j]));
          TL logit;
          if (rho0 == TL(0) && rho1 == TL(0)) {
            logit = TL(0);
            if (act[j]) any_bad = true;
          } else {
            logit = Num<TL>::log_(rho1) - Num<TL>::log_(rho0);
          }
          if (r > 0) logit += TL(2) * betaL * TL(jup) * TL(up ? 1 : -1);
          lg_own[o] = logit;
          if (corr) sh_lg[sl] = act[j] ? clamp_logit((float)logit) : 0.f;
        }
      }
      if (corr) {
        // the network's shift of every chain's logit: 16 chains per warp pass
        __syncthreads();
        const int g = lane >> 2, t4 = lane & 3;
        for (int m = tid >> 5; m < SB / 16; m += P::NT / 32) {
          uint32_t xw[2];
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int sl = 16 * m + g + 8 * h;
            const uint32_t *bp = bprev + sl * WL, *bc = bcur + sl * WL;
            const double sup = ((bp[c >> 5] >> (c & 31)) & 1) ? 1.0 : -1.0;
            float f0, f1;
            if (t4 == 0) {
              f0 = sh_lg[sl];
              f1 = r > 0 ? (float)(2.0 * lay.beta * (double)jd[(r - 1) * L + c] * sup) : 0.f;
            } else if (t4 == 1) {
              const double sle = c > 0 ? (((bc[(c - 1) >> 5] >> ((c - 1) & 31)) & 1) ? 1.0 : -1.0) : 0.0;
              f0 = c > 0 ? (float)(lay.beta * (double)jr[r * L + c - 1] * sle) : 0.f;
              f1 = jr[r * L + c];
            } else if (t4 == 2) {
              f0 = jd[r * L + c];
              f1 = (r > 0 && c < L - 1) ? (((bp[(c + 1) >> 5] >> ((c + 1) & 31)) & 1) ? 1.f : -1.f) : 0.f;
            } else {
              f0 = (float)lay.beta;
              f1 = 0.f;
            }
            xw[h] = pack_bf16(f0, f1);
          }
          const float2 d = mlp_warp16(mp, xw[0], xw[1], lane);
          if (t4 == 0) {
            sh_dl[16 * m + g] = d.x;
            sh_dl[16 * m + g + 8] = d.y;
          }
        }
        __syncthreads();
#pragma unroll
        for (int o = 0; o < OWN; ++o) {
          const int j = cg + o * NCG;
          if (j < TS) lg_own[o] += TL(sh_dl[sg * TS + j]);
        }
      }
      int sig_own[OWN];
#pragma unroll
      for (int o = 0; o < OWN; ++o) {
        const int j = cg + o * NCG;
        sig_own[o] = 0;
        if (j < TS) {
          const int sl = sg * TS + j;
          const int up = (r > 0) ? (bprev[sl * WL + (c >> 5)] >> (c & 31)) & 1 : 0;
          const TL logit = lg_own[o];
          int sgm;
          if (FORCED) {
            sgm = act[j] ? in_spins[int64_t(S) * ri.site_off + int64_t(sid[j]) * L2 + i] : 0;
          } else {
            const int64_t g = i >> 2;
            if (g != pg[o]) {
              const U64x4 ww = philox4x64_10((uint64_t)g, prop_base + (uint64_t)sid[j],
                                             (uint64_t)ri.gid, TAG_SPIN, seed, 0ull);
#pragma unroll
              for (int q = 0; q < 4; ++q) pw[o][q] = ww.x[q];
              pg[o] = g;
            }
            const double uu = word_to_uniform(pw[o][i & 3]);
            const TL ls = log_sigmoid<TL>(logit);
            sgm = uu < (double)Num<TL>::exp_(ls) ? 1 : 0;
          }
          const TL lpick = sgm ? log_sigmoid<TL>(logit) : log_sigmoid<TL>(-logit);
          lq[o] += (double)lpick;
          const double sv = sgm ? 1.0 : -1.0;
          if (c > 0) en[o] -= jl * sv * (double)(sleft[o] ? 1.0 : -1.0);
          if (r > 0) en[o] -= (double)jup * sv * (up ? 1.0 : -1.0);
          sleft[o] = sgm;
          if (sgm) bcur[sl * WL + (c >> 5)] |= 1u << (c & 31);
          if (act[j]) {
            const int64_t off = int64_t(S) * ri.site_off + int64_t(sid[j]) * L2 + i;
            if (!FORCED) out_spins[off] = (uint8_t)sgm;
            if (lay.dbg_logits) lay.dbg_logits[off] = (float)logit;
          }
          sig_own[o] = sgm;
        }
      }
      // broadcast the decisions to the chain group, update the left environment
      T *vout = Vb + (buf ^ 1) * CH * SB;
#pragma unroll
      for (int j = 0; j < TS; ++j) {
        const int src = gbase + (j % NCG);
        const int sgm = __shfl_sync(0xffffffffu, sig_own[j / NCG], src);
        T nv[TC];
        T nrm = 0;
#pragma unroll
        for (int t = 0; t < TC; ++t) {
          const int b = cg * TC + t;
          nv[t] = sgm ? ((b >= br.x) ? -(u[j][t] - w[j][t]) : (u[j][t] - w[j][t]))
                      : (u[j][t] + w[j][t]);
          nrm += nv[t] * nv[t];
        }
        nrm = gsum<T, NCG>(nrm);
        const T inv = nrm > T(0) ? T(1) / Num<T>::sqrt_(nrm) : T(0);
        if (!(nrm > T(0)) && act[j]) any_bad = true;
#pragma unroll
        for (int t = 0; t < TC; ++t) vout[(cg * TC + t) * SB + sg * TS + j] = nv[t] * inv;
      }
      buf ^= 1;
    }
    __syncthreads();
    uint32_t *tmp = bprev; bprev = bcur; bcur = tmp;
  }
  // results
#pragma unroll
  for (int o = 0; o < OWN; ++o) {
    const int j = cg + o * NCG;
    if (j < TS && act[j]) {
      out_logq[int64_t(n) * S + sid[j]] = lq[o];
      out_E[int64_t(n) * S + sid[j]] = en[o];
    }
  }
  if (any_bad) set_flag(lay.flags, n, FLAG_NUMERIC);
}

}  // namespace

template <typename T, int CH, bool FORCED, bool CORR>
static cudaError_t launch_samp_c(const Layout &lay, int S, uint64_t seed, uint64_t base,
                                 const uint8_t *in, uint8_t *out, double *lq, double *E,
                                 cudaStream_t st) {
  using P = SampPlan<CH>;
  const int WL = (lay.L_max + 31) / 32;
  const int64_t smem = samp_smem_fixed<T, CH>() + int64_t(2) * SB * WL * 4 +
                       (lay.mlp ? int64_t(sizeof(MlpSmem)) + 2 * SB * 4 : 0);
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(sample_kernel<T, CH, FORCED, CORR>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  const int bpr = (S + SB - 1) / SB;
  sample_kernel<T, CH, FORCED, CORR><<<lay.n_real * bpr, P::NT, smem, st>>>(lay, S, seed, base, in,
                                                                            out, lq, E);
  return cudaGetLastError();
}

template <typename T, int CH, bool FORCED>
static cudaError_t launch_samp_t(const Layout &lay, int S, uint64_t seed, uint64_t base,
                                 const uint8_t *in, uint8_t *out, double *lq, double *E,
                                 cudaStream_t st) {
  return lay.mlp ? launch_samp_c<T, CH, FORCED, true>(lay, S, seed, base, in, out, lq, E, st)
                 : launch_samp_c<T, CH, FORCED, false>(lay, S, seed, base, in, out, lq, E, st);
}

template <bool FORCED>
static cudaError_t launch_samp(const Layout &lay, int prec, int CH, int S, uint64_t seed,
                               uint64_t base, const uint8_t *in, uint8_t *out, double *lq,
                               double *E, cudaStream_t st) {
  if (prec == 0) {
    switch (CH) {
      case 8: return launch_samp_t<double, 8, FORCED>(lay, S, seed, base, in, out, lq, E, st);
      case 16: return launch_samp_t<double, 16, FORCED>(lay, S, seed, base, in, out, lq, E, st);
      case 32: return launch_samp_t<double, 32, FORCED>(lay, S, seed, base, in, out, lq, E, st);
      case 64: return launch_samp_t<double, 64, FORCED>(lay, S, seed, base, in, out, lq, E, st);
    }
  } else if (prec == 2) {
    switch (CH) {
      case 8: return launch_samp_t<dfloat, 8, FORCED>(lay, S, seed, base, in, out, lq, E, st);
      case 16: return launch_samp_t<dfloat, 16, FORCED>(lay, S, seed, base, in, out, lq, E, st);
      case 32: return launch_samp_t<dfloat, 32, FORCED>(lay, S, seed, base, in, out, lq, E, st);
      case 64: return launch_samp_t<dfloat, 64, FORCED>(lay, S, seed, base, in, out, lq, E, st);
    }
  } else {
    switch (CH) {
      case 8: return launch_samp_t<float, 8, FORCED>(lay, S, seed, base, in, out, lq, E, st);
      case 16: return launch_samp_t<float, 16, FORCED>(lay, S, seed, base, in, out, lq, E, st);
      case 32: return launch_samp_t<float, 32, FORCED>(lay, S, seed, base, in, out, lq, E, st);
      case 64: return launch_samp_t<float, 64, FORCED>(lay, S, seed, base, in, out, lq, E, st);
    }
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_propose(const Layout &lay, int prec, int CH, int S, uint64_t seed,
                           uint64_t base, uint8_t *spins, double *lq, double *E,
                           cudaStream_t st) {
  return launch_samp<false>(lay, prec, CH, S, seed, base, nullptr, spins, lq, E, st);
}

cudaError_t launch_score(const Layout &lay, int prec, int CH, int S, const uint8_t *spins,
                         double *lq, double *E, cudaStream_t st) {
  return launch_samp<true>(lay, prec, CH, S, 0, 0, spins, nullptr, lq, E, st);
}

// ---------------------------------------------------------------------------
// Proposals without caller-provided scratch. The right environments live in a
// fixed device array owned by this library instead of the workspace. Every
// device that loads the library holds the array until the process exits.
constexpr int64_t kStaticScratchBytes = int64_t(32) << 20;   // 32 MiB
static __device__ __align__(256) unsigned char g_propose_scratch[kStaticScratchBytes];

namespace {
constexpr int kMaxDevices = 64;
void *g_scratch_ptr[kMaxDevices] = {};
std::mutex g_scratch_mu;
}  // namespace

int64_t static_scratch_bytes() { return kStaticScratchBytes; }

// Address of the array on the current device. The array's name in host code is
// only a host-side stand-in, so the device address is looked up once per
// device (with that device current) and cached.
static cudaError_t static_scratch_address(void **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_propose_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

// Same kernel as launch_propose; only the scratch pointer and its per-line
// stride (S chains instead of max_samples) differ. Nothing in the scratch has
// to start at zero: every element the kernel reads was written earlier in the
// same launch.
cudaError_t launch_propose_static(const Layout &lay, int prec, int CH, int S, uint64_t seed,
                                  uint64_t base, uint8_t *spins, double *lq, double *E,
                                  int64_t sum_L, cudaStream_t st, bool *too_big) {
  const int64_t esz = prec == 1 ? 4 : 8;
  *too_big = int64_t(S) * sum_L * CH * esz > kStaticScratchBytes;
  if (*too_big) return cudaSuccess;
  void *scratch = nullptr;
  cudaError_t e = static_scratch_address(&scratch);
  if (e != cudaSuccess) return e;
  Layout l2 = lay;
  l2.samp_scratch = scratch;
  l2.max_samples = S;
  return launch_samp<false>(l2, prec, CH, S, seed, base, nullptr, spins, lq, E, st);
}

int64_t sampler_smem_bytes(int prec, int CH, int L_max) {
  const int WL = (L_max + 31) / 32;
  const int64_t extra = int64_t(2) * SB * WL * 4 + int64_t(sizeof(MlpSmem)) + 2 * SB * 4;
  if (prec != 1) {   // float64 and double-float values are 8 bytes
    switch (CH) {
      case 8: return samp_smem_fixed<double, 8>() + extra;
      case 16: return samp_smem_fixed<double, 16>() + extra;
      case 32: return samp_smem_fixed<double, 32>() + extra;
      case 64: return samp_smem_fixed<double, 64>() + extra;
    }
  } else {
    switch (CH) {
      case 8: return samp_smem_fixed<float, 8>() + extra;
      case 16: return samp_smem_fixed<float, 16>() + extra;
      case 32: return samp_smem_fixed<float, 32>() + extra;
      case 64: return samp_smem_fixed<float, 64>() + extra;
    }
  }
  return -1;
}

}  // namespace tnmc
