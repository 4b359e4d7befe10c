// Shared device definitions of the TNMC library: the workspace layout, the
// Philox4x64-10 generator, numeric helpers and the parity (Z2) conventions of
// the boundary-MPS storage.
//
// Parity storage of the cache (design note, not in the paper). The spin-flip
// symmetry s -> -s of the zero-field models makes every boundary function
// F_r(s) even. Each bond index carries a parity, and a site of the MPS is
// stored as ONE matrix C[a, b] over (left bond, right bond): the physical
// index is implied by parity. In sigma (spin-bit) form the site tensor is
//     M[sigma] = Pi_left^sigma  C  Pi_right^sigma,
// where Pi = diag(+1 on even indices, -1 on odd ones). The even-even and
// odd-odd blocks of C are the symmetric part A(+) = (M[0] + M[1]) / 2 and the
// even-odd / odd-even blocks the antisymmetric part A(-) = (M[0] - M[1]) / 2.
// A bond of dimension D is stored as its even indices first (e of them), then
// its odd ones (o = D - e), then zero padding up to chi.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "dfloat.cuh"

namespace tnmc {

enum : int32_t { FLAG_BAD_J = 1, FLAG_NUMERIC = 2, FLAG_TIMEOUT = 4 };

struct RealInfo {
  int32_t L;
  int32_t pad;
  int64_t site_off;   // sum_{m<n} L_m^2: sites before this realization
  int64_t bond_off;   // sum_{m<n} L_m (L_m + 1): bond-dimension records before it
  int64_t row_off;    // sum_{m<n} L_m: rows before it
  int64_t line_off;   // sum_{m<n} L_m: sampler scratch lines (per sample) before it
  int64_t cache_off;  // first chi x chi matrix of this realization in the cache
  int64_t ckpt_off;   // first chi x chi matrix of its float64 checkpoint rows (MIXED + checkpoints)
  int64_t gid;        // stream id of its random numbers (the counter word that names the
                      // realization): its index n unless the caller set global ids
};

// Device-side view of the workspace; passed by value to every kernel.
struct Layout {
  const RealInfo *reals;
  const int32_t *order;      // realizations by decreasing L (longest first)
  int32_t n_real;
  int32_t chi;               // runtime bond dimension (<= compile-time CH)
  int32_t L_max;
  int32_t max_samples;
  double beta;
  double cutoff;             // relative singular-value cutoff of the truncation
  float *jr;                 // [sum L^2] coupling to the right neighbour (0 on the last column)
  float *jd;                 // [sum L^2] coupling to the lower neighbour (0 on the last row)
  void *cache;               // [sum rows_n L_n][chi][chi] of T: site matrices C, row-major
  int32_t ckpt_every;        // K: 0 = every row cached; else checkpoint rows + one segment
  int32_t seg_begin;         // rows [seg_begin, seg_end) of this launch; seg_begin < 0 = all rows
  int32_t seg_end;
  int64_t wait_cycles;       // budget of a bounded device wait (0: the kernel's default)
  int32_t variant;           // kernel layout of the environment build (env_build.cu, VARIANT_*)
  int32_t tune_rows;         // > 0: build only each realization's bottom tune_rows rows (timing)
  int32_t tc_mode;           // float32 build: the dense products on the tensor cores from TF32
                             // (1) or BF16 (2) operands, float32 accumulation; 0: CUDA cores
  double *ckpt64;            // MIXED with checkpoints: the checkpoint rows in float64, or null
  int2 *bonds;               // [sum L (L+1)]: (even, odd) dimension of bond b of row r
  double *lam;               // [sum L]: log scale lambda_r of row r
  int32_t *flags;            // [n_real]: FLAG_* bits
  int32_t *counter;          // work counters of the persistent kernels
  void *env_scratch;         // [slots][env_slot_bytes]
  int64_t env_slot_bytes;
  int32_t env_slots;
  void *samp_scratch;        // [max_samples * sum L][chi] of T: right environments
  const uint16_t *mlp;       // bfloat16 parameters of the learned correction, or null (off)
  // optional diagnostics (may be null)
  float *dbg_logits;
  double *dbg_spectra;
  double *dbg_rowinfo;
};

// ------------------------------------------------------------------ Philox4x64-10
// Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
// SC'11: ten rounds of two 64x64->128 multiplies, key bumped by the Weyl
// constants between rounds.
struct U64x4 { uint64_t x[4]; };

__device__ __forceinline__ U64x4 philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2,
                                                uint64_t c3, uint64_t k0, uint64_t k1) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
  uint64_t x0 = c0, x1 = c1, x2 = c2, x3 = c3;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += W0; k1 += W1; }
    const uint64_t hi0 = __umul64hi(M0, x0), lo0 = M0 * x0;
    const uint64_t hi1 = __umul64hi(M1, x2), lo1 = M1 * x2;
    const uint64_t y0 = hi1 ^ x1 ^ k0, y2 = hi0 ^ x3 ^ k1;
    x0 = y0; x1 = lo1; x2 = y2; x3 = lo0;
  }
  U64x4 o; o.x[0] = x0; o.x[1] = x1; o.x[2] = x2; o.x[3] = x3;
  return o;
}

enum : uint64_t { TAG_SPIN = 0, TAG_MH = 1, TAG_INIT = 2 };

// u = (2 (w >> 12) + 1) 2^-53, exact in float64, strictly inside (0, 1).
__device__ __forceinline__ double word_to_uniform(uint64_t w) {
  return (double)(2ull * (w >> 12) + 1ull) * 0x1.0p-53;
}

// ------------------------------------------------------------------ numerics
template <typename T> struct Num;
template <> struct Num<float> {
  static __device__ __forceinline__ float log_(float x) { return logf(x); }
  static __device__ __forceinline__ float exp_(float x) { return expf(x); }
  static __device__ __forceinline__ float log1p_(float x) { return log1pf(x); }
  static __device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }
  static __device__ __forceinline__ float tanh_(float x) { return tanhf(x); }
  static __host__ __device__ constexpr float eps() { return 5.9604645e-8f; }
};
template <> struct Num<double> {
  static __device__ __forceinline__ double log_(double x) { return log(x); }
  static __device__ __forceinline__ double exp_(double x) { return exp(x); }
  static __device__ __forceinline__ double log1p_(double x) { return log1p(x); }
  static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
  static __device__ __forceinline__ double tanh_(double x) { return tanh(x); }
  static __host__ __device__ constexpr double eps() { return 1.1102230246251565e-16; }
};
// double-float: tensor arithmetic on the FP32 pipes (dfloat.cuh); the elementary
// functions, needed once per site, through float64
template <> struct Num<dfloat> {
  static __device__ __forceinline__ dfloat log_(dfloat x) { return dfloat(log(double(x))); }
  static __device__ __forceinline__ dfloat exp_(dfloat x) { return dfloat(exp(double(x))); }
  static __device__ __forceinline__ dfloat log1p_(dfloat x) { return dfloat(log1p(double(x))); }
  static __device__ __forceinline__ dfloat sqrt_(dfloat x) { return df::sqrt(x); }
  static __device__ __forceinline__ dfloat tanh_(dfloat x) { return dfloat(tanh(double(x))); }
  static __host__ __device__ constexpr double eps() { return 3.552713678800501e-15; }   // 2^-48
};

// log sigmoid(x) = -softplus(-x), stable for either sign.
template <typename T>
__device__ __forceinline__ T log_sigmoid(T x) {
  const T ax = x < T(0) ? -x : x;
  const T neg = x < T(0) ? x : T(0);
  return neg - Num<T>::log1p_(Num<T>::exp_(-ax));
}

__device__ __forceinline__ void set_flag(int32_t *flags, int n, int32_t bit) {
  atomicOr(flags + n, bit);
}

// Cache rows of a realization of side L. With checkpointing every K rows the
// cache holds the checkpoint rows 0, K, 2K, ... (slot r / K) and one segment of
// K rows (slots ceil(L/K) .. ceil(L/K) + K - 1); without it, row r is slot r.
__host__ __device__ inline int64_t cache_rows(int L, int K) {
  return K > 0 ? int64_t((L + K - 1) / K + K) : int64_t(L);
}
// Slot of row r. Full build (seg_begin < 0): checkpoint rows go to their slot,
// the others alternate between the first two segment slots (each row is read
// only by the row above it). Segment [a, b): its rows go to the segment slots;
// the row below it (b, a multiple of K) is read from its checkpoint.
__host__ __device__ inline int64_t cache_slot(int r, int L, int K, int seg_begin) {
  if (K <= 0) return r;
  const int64_t nck = (L + K - 1) / K;
  if (seg_begin < 0) return (r % K == 0) ? r / K : nck + (r & 1);
  if (r >= seg_begin && r < seg_begin + K) return nck + (r - seg_begin);
  return r / K;
}

// Bytes rounded up to 256 for every workspace region.
__host__ __device__ constexpr int64_t align256(int64_t x) { return (x + 255) & ~int64_t(255); }

}  // namespace tnmc
