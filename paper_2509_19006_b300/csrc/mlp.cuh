// The learned proposal correction's network on the tensor cores (an extension
// of the method; the paper's sampler has no correction).
//
//   x (7 features, rounded to bfloat16) -> h1 = g(W1 x + b1), rounded to
//   bfloat16 -> h2 = g(W2 h1 + b2) -> Delta = w3 . h2 + b3,
//   g(z) = 0 (z <= -1), (z + 1)^2 / 4 (|z| < 1), z (z >= 1).
//
// One warp evaluates 16 rows (chains or examples) with mma.sync m16n8k16
// (bfloat16 operands, float32 accumulators): layer 1 is one k-step per
// 8-wide output tile, layer 2 four k-steps per tile, and the accumulator
// fragments of layer 1 are repacked in registers as the A operand of layer 2
// (in the m16n8k16 layouts an accumulator tile pair covers exactly one A
// k-tile). Layer 3 is a float32 dot product finished across the lane quad.
// Why mma.sync and not tcgen05: inside the sampler the network runs once per
// site on the CTA's 64 chains (a 64 x 64 x 64 product), between two dependent
// steps of the draw; the asynchronous issue / commit / mbarrier round trip of
// tcgen05 and its TMEM traffic cost more than this product itself.
#pragma once
#include <cstdint>
#include <cuda_bf16.h>

#include "common.cuh"
#include "tcmma.cuh"

namespace tnmc {

constexpr int MLP_F = 7;
constexpr int MLP_H = 64;
constexpr int MLP_IN = 16;
constexpr int MLP_OFF_W1 = 0, MLP_OFF_B1 = 1024, MLP_OFF_W2 = 1088, MLP_OFF_B2 = 5184;
constexpr int MLP_OFF_W3 = 5248, MLP_OFF_B3 = 5312, MLP_PARAMS = 5320;
constexpr float MLP_LOGIT_CLAMP = 32.f;   // the logit feature is clamped to +-32 (sigmoid(32) = 1 - 1e-14)
constexpr int MLP_LD1 = 24;   // padded W1 row in shared memory (bank-conflict free fragment loads)
constexpr int MLP_LD2 = 72;   // padded W2 row

// Parameters staged in shared memory (bfloat16 weights, float32 biases).
struct MlpSmem {
  uint16_t W1[MLP_H * MLP_LD1];
  uint16_t W2[MLP_H * MLP_LD2];
  float b1[MLP_H], b2[MLP_H], w3[MLP_H];
  float b3, pad[3];
};

__device__ __forceinline__ float bf16_bits_to_float(uint16_t b) {
  return __uint_as_float(uint32_t(b) << 16);
}

// Stage the parameter vector (bfloat16, global) into shared memory; all
// threads of the block call it, followed by a barrier of the caller's.
__device__ __forceinline__ void mlp_stage(MlpSmem *P, const uint16_t *g, int tid, int nt) {
  for (int e = tid; e < MLP_H * MLP_IN; e += nt) P->W1[(e / MLP_IN) * MLP_LD1 + e % MLP_IN] = g[MLP_OFF_W1 + e];
  for (int e = tid; e < MLP_H * MLP_H; e += nt) P->W2[(e / MLP_H) * MLP_LD2 + e % MLP_H] = g[MLP_OFF_W2 + e];
  for (int e = tid; e < MLP_H; e += nt) {
    P->b1[e] = bf16_bits_to_float(g[MLP_OFF_B1 + e]);
    P->b2[e] = bf16_bits_to_float(g[MLP_OFF_B2 + e]);
    P->w3[e] = bf16_bits_to_float(g[MLP_OFF_W3 + e]);
  }
  if (tid == 0) P->b3 = bf16_bits_to_float(g[MLP_OFF_B3]);
}

__device__ __forceinline__ float clamp_logit(float x) {
  return fminf(fmaxf(x, -MLP_LOGIT_CLAMP), MLP_LOGIT_CLAMP);
}

__device__ __forceinline__ float mlp_act(float z) {
  const float q = 0.25f * (z + 1.f) * (z + 1.f);
  return z >= 1.f ? z : (z <= -1.f ? 0.f : q);
}

// Delta of 16 rows by one warp. Lane (g = lane / 4, t = lane % 4) passes the
// bfloat16 pairs of features (2t, 2t+1) of row g (xa) and of row g + 8 (xb);
// feature 7 is zero. Returns (Delta of row g, Delta of row g + 8) in every
// lane of the quad.
__device__ __forceinline__ float2 mlp_warp16(const MlpSmem *P, uint32_t xa, uint32_t xb, int lane) {
  const int g = lane >> 2, t = lane & 3;
  // layer 1: one k-step (features in columns 0..7, columns 8..15 zero)
  float c1[8][4];
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    const float bl = P->b1[8 * nt + 2 * t], bh = P->b1[8 * nt + 2 * t + 1];
    c1[nt][0] = bl; c1[nt][1] = bh; c1[nt][2] = bl; c1[nt][3] = bh;
    const uint32_t b0 = *reinterpret_cast<const uint32_t *>(&P->W1[(8 * nt + g) * MLP_LD1 + 2 * t]);
    mma_bf16_16816(c1[nt], xa, xb, 0u, 0u, b0, 0u);
  }
  // activation, rounded to bfloat16, repacked as the A operand of layer 2
  uint32_t a[4][4];
#pragma unroll
  for (int kt = 0; kt < 4; ++kt) {
    a[kt][0] = pack_bf16(mlp_act(c1[2 * kt][0]), mlp_act(c1[2 * kt][1]));
    a[kt][1] = pack_bf16(mlp_act(c1[2 * kt][2]), mlp_act(c1[2 * kt][3]));
    a[kt][2] = pack_bf16(mlp_act(c1[2 * kt + 1][0]), mlp_act(c1[2 * kt + 1][1]));
    a[kt][3] = pack_bf16(mlp_act(c1[2 * kt + 1][2]), mlp_act(c1[2 * kt + 1][3]));
  }
  // layer 2 and the partial dot products of layer 3
  float da = 0.f, db = 0.f;
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    const float bl = P->b2[8 * nt + 2 * t], bh = P->b2[8 * nt + 2 * t + 1];
    float c[4] = {bl, bh, bl, bh};
    const uint16_t *wrow = &P->W2[(8 * nt + g) * MLP_LD2 + 2 * t];
#pragma unroll
    for (int kt = 0; kt < 4; ++kt) {
      const uint32_t b0 = *reinterpret_cast<const uint32_t *>(wrow + 16 * kt);
      const uint32_t b1 = *reinterpret_cast<const uint32_t *>(wrow + 16 * kt + 8);
      mma_bf16_16816(c, a[kt][0], a[kt][1], a[kt][2], a[kt][3], b0, b1);
    }
    const float wl = P->w3[8 * nt + 2 * t], wh = P->w3[8 * nt + 2 * t + 1];
    da = fmaf(wl, mlp_act(c[0]), da);
    da = fmaf(wh, mlp_act(c[1]), da);
    db = fmaf(wl, mlp_act(c[2]), db);
    db = fmaf(wh, mlp_act(c[3]), db);
  }
  da += __shfl_xor_sync(0xffffffffu, da, 1);
  da += __shfl_xor_sync(0xffffffffu, da, 2);
  db += __shfl_xor_sync(0xffffffffu, db, 1);
  db += __shfl_xor_sync(0xffffffffu, db, 2);
  return make_float2(da + P->b3, db + P->b3);
}

}  // namespace tnmc
