// Learned proposal correction (an extension of the method; the paper's
// sampler, Sec. 3.3, has no correction): training examples, loss and
// gradient, Adam, and the stand-alone tensor-core forward pass. The sampler
// evaluates the same network inside its per-site loop (sample.cu, mlp.cuh).
//
// Gradient: each CTA of a fixed grid takes tiles of 32 examples, runs the
// forward pass with the same two bfloat16 roundings as the sampler
// (features, first hidden layer) in float32 on the CUDA cores, backpropagates
// the mean binary cross entropy with the roundings passed straight through,
// and keeps its share of the gradient in registers; every CTA writes its
// partial gradient, and a second kernel sums the partials in CTA order, so
// equal inputs give equal bits. The whole network is ~5k parameters and one
// example costs ~14k multiply-adds forward and backward, so a 64k-example
// minibatch is about 1 GFLOP: the training kernels are a small fraction of
// the time of generating their data (two environment builds and scoring).
#include "../../include/tnmc.h"
#include "common.cuh"
#include "mlp.cuh"

#include <cmath>

namespace tnmc {

namespace {

constexpr int GR_THREADS = 256;
constexpr int GR_TILE = 32;
constexpr int GR_BLOCKS = 296;                 // 2 x 148 SMs
constexpr int GR_STRIDE = MLP_PARAMS + 8;      // partial gradient row: parameters, then the loss
constexpr int LDW2 = MLP_H + 1;                // padded float rows of W2 in shared memory

__device__ __forceinline__ float bf16_round(float x) {
  return __bfloat162float(__float2bfloat16_rn(x));
}
__device__ __forceinline__ float act_grad(float z) {
  return z >= 1.f ? 1.f : (z <= -1.f ? 0.f : 0.5f * (z + 1.f));
}
__device__ __forceinline__ float log_sigmoid_f(float z) {
  return fminf(z, 0.f) - log1pf(expf(-fabsf(z)));
}

// Features of every site of S configurations per realization; grid.y = realization.
__global__ void features_kernel(Layout lay, int S, const uint8_t *spins, const float *logits,
                                float *feat) {
  const int n = blockIdx.y;
  const RealInfo ri = lay.reals[n];
  const int L = ri.L;
  const int64_t L2 = int64_t(L) * L;
  const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= int64_t(S) * L2) return;
  const int64_t sid = e / L2;
  const int i = int(e % L2), r = i / L, c = i % L;
  const int64_t base = int64_t(S) * ri.site_off + sid * L2;
  const float *jr = lay.jr + ri.site_off, *jd = lay.jd + ri.site_off;
  auto spin = [&](int rr, int cc) { return spins[base + int64_t(rr) * L + cc] ? 1.0 : -1.0; };
  float x[8];
  x[0] = clamp_logit(logits[base + i]);
  x[1] = r > 0 ? (float)(2.0 * lay.beta * (double)jd[(r - 1) * L + c] * spin(r - 1, c)) : 0.f;
  x[2] = c > 0 ? (float)(lay.beta * (double)jr[r * L + c - 1] * spin(r, c - 1)) : 0.f;
  x[3] = jr[r * L + c];
  x[4] = jd[r * L + c];
  x[5] = (r > 0 && c < L - 1) ? (float)spin(r - 1, c + 1) : 0.f;
  x[6] = (float)lay.beta;
  x[7] = 0.f;
  float4 *o = reinterpret_cast<float4 *>(feat + (base + i) * 8);
  o[0] = make_float4(x[0], x[1], x[2], x[3]);
  o[1] = make_float4(x[4], x[5], x[6], x[7]);
}

struct GradSmem {
  float W1[MLP_H * MLP_F];
  float b1[MLP_H], b2[MLP_H], w3[MLP_H];
  float W2[MLP_H * LDW2];
  float xh[GR_TILE * 8];         // bfloat16-rounded features
  float x0[GR_TILE], p[GR_TILE], dz[GR_TILE], valid[GR_TILE];
  float z1[GR_TILE * MLP_H];     // pre-activations of layer 1, later d loss / d z1
  float h1[GR_TILE * MLP_H];     // bfloat16-rounded g(z1)
  float z2[GR_TILE * MLP_H];     // pre-activations of layer 2, later d loss / d z2
  float red[4 * 3 * MLP_H];      // cross-group sums of b1, b2, w3 gradients
  float b3;
};

__global__ void __launch_bounds__(GR_THREADS)
grad_kernel(const float *feat, const float *tgt, int64_t n_ex, int B, uint64_t seed, int step,
            const uint16_t *prm, float *partial) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  GradSmem &s = *reinterpret_cast<GradSmem *>(smem_raw);
  const int tid = threadIdx.x;
  for (int e = tid; e < MLP_H * MLP_F; e += GR_THREADS)
    s.W1[e] = bf16_bits_to_float(prm[MLP_OFF_W1 + (e / MLP_F) * MLP_IN + e % MLP_F]);
  for (int e = tid; e < MLP_H * MLP_H; e += GR_THREADS)
    s.W2[(e / MLP_H) * LDW2 + e % MLP_H] = bf16_bits_to_float(prm[MLP_OFF_W2 + e]);
  for (int e = tid; e < MLP_H; e += GR_THREADS) {
    s.b1[e] = bf16_bits_to_float(prm[MLP_OFF_B1 + e]);
    s.b2[e] = bf16_bits_to_float(prm[MLP_OFF_B2 + e]);
    s.w3[e] = bf16_bits_to_float(prm[MLP_OFF_W3 + e]);
  }
  if (tid == 0) s.b3 = bf16_bits_to_float(prm[MLP_OFF_B3]);
  const int64_t total = B > 0 ? int64_t(B) : n_ex;
  const float inv_n = 1.f / float(total);
  const int64_t ntiles = (total + GR_TILE - 1) / GR_TILE;

  // register shares of the gradient
  const int hq = tid & 63, eq = tid >> 6;        // (hidden unit, example group) of the tile passes
  const int h2o = tid >> 2, k2o = (tid & 3) * 16;  // W2 block owned: row h2o, columns k2o..k2o+15
  float gW2[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) gW2[j] = 0.f;
  float gW1[2] = {0.f, 0.f};
  float gb1 = 0.f, gb2 = 0.f, gw3 = 0.f, gb3 = 0.f, lsum = 0.f;
  __syncthreads();

  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    // ---- load the tile
    if (tid < GR_TILE) {
      const int64_t k = tile * GR_TILE + tid;
      int64_t row = -1;
      if (k < total) {
        if (B > 0) {
          const U64x4 w = philox4x64_10(uint64_t(k >> 2), uint64_t(step), 0ull, 3ull, seed, 0ull);
          const double u = word_to_uniform(w.x[k & 3]);
          row = min(int64_t(floor(u * double(n_ex))), n_ex - 1);
        } else {
          row = k;
        }
      }
      float f[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      float pt = 0.f;
      if (row >= 0) {
        const float4 a = reinterpret_cast<const float4 *>(feat + row * 8)[0];
        const float4 b = reinterpret_cast<const float4 *>(feat + row * 8)[1];
        f[0] = a.x; f[1] = a.y; f[2] = a.z; f[3] = a.w; f[4] = b.x; f[5] = b.y; f[6] = b.z;
        pt = 1.f / (1.f + expf(-tgt[row]));
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) s.xh[tid * 8 + q] = bf16_round(f[q]);
      s.x0[tid] = f[0];
      s.p[tid] = pt;
      s.valid[tid] = row >= 0 ? 1.f : 0.f;
    }
    __syncthreads();
    // ---- layer 1
    for (int e = eq; e < GR_TILE; e += 4) {
      float z = s.b1[hq];
#pragma unroll
      for (int k = 0; k < MLP_F; ++k) z = fmaf(s.W1[hq * MLP_F + k], s.xh[e * 8 + k], z);
      s.z1[e * MLP_H + hq] = z;
      s.h1[e * MLP_H + hq] = bf16_round(mlp_act(z));
    }
    __syncthreads();
    // ---- layer 2
    for (int e = eq; e < GR_TILE; e += 4) {
      float z = s.b2[hq];
      const float *hr = s.h1 + e * MLP_H;
#pragma unroll 16
      for (int k = 0; k < MLP_H; ++k) z = fmaf(s.W2[hq * LDW2 + k], hr[k], z);
      s.z2[e * MLP_H + hq] = z;
    }
    __syncthreads();
    // ---- output, loss, d loss / d Delta
    if (tid < GR_TILE) {
      float d = s.b3;
      for (int h = 0; h < MLP_H; ++h) d = fmaf(s.w3[h], mlp_act(s.z2[tid * MLP_H + h]), d);
      const float z = s.x0[tid] + d, pt = s.p[tid];
      const float sig = 1.f / (1.f + expf(-z));
      const float v = s.valid[tid];
      s.dz[tid] = v * (sig - pt) * inv_n;
      lsum += v * -(pt * log_sigmoid_f(z) + (1.f - pt) * log_sigmoid_f(-z));
    }
    __syncthreads();
    // ---- layer 3 gradients; d loss / d z2 in place of z2
    for (int e = eq; e < GR_TILE; e += 4) {
      const float z = s.z2[e * MLP_H + hq], dz = s.dz[e];
      gw3 = fmaf(dz, mlp_act(z), gw3);
      const float d2 = dz * s.w3[hq] * act_grad(z);
      gb2 += d2;
      s.z2[e * MLP_H + hq] = d2;
    }
    if (tid == 0)
      for (int e = 0; e < GR_TILE; ++e) gb3 += s.dz[e];
    __syncthreads();
    // ---- W2 gradient (this thread's block) and d loss / d z1 in place of z1
    for (int e = 0; e < GR_TILE; ++e) {
      const float d2 = s.z2[e * MLP_H + h2o];
      const float *hr = s.h1 + e * MLP_H + k2o;
#pragma unroll
      for (int j = 0; j < 16; ++j) gW2[j] = fmaf(d2, hr[j], gW2[j]);
    }
    for (int e = eq; e < GR_TILE; e += 4) {
      float d1 = 0.f;
      const float *dr = s.z2 + e * MLP_H;
#pragma unroll 16
      for (int h = 0; h < MLP_H; ++h) d1 = fmaf(dr[h], s.W2[h * LDW2 + hq], d1);
      s.z1[e * MLP_H + hq] = d1 * act_grad(s.z1[e * MLP_H + hq]);
    }
    __syncthreads();
    // ---- W1, b1 gradients
    for (int q = 0; q < 2; ++q) {
      const int idx = tid + q * GR_THREADS;
      if (idx < MLP_H * MLP_F) {
        const int h = idx / MLP_F, k = idx % MLP_F;
        float a = gW1[q];
        for (int e = 0; e < GR_TILE; ++e) a = fmaf(s.z1[e * MLP_H + h], s.xh[e * 8 + k], a);
        gW1[q] = a;
      }
    }
    for (int e = eq; e < GR_TILE; e += 4) gb1 += s.z1[e * MLP_H + hq];
    __syncthreads();
  }
  // ---- the CTA's partial gradient, in parameter order
  float *out = partial + int64_t(blockIdx.x) * GR_STRIDE;
#pragma unroll
  for (int j = 0; j < 16; ++j) out[MLP_OFF_W2 + h2o * MLP_H + k2o + j] = gW2[j];
  for (int q = 0; q < 2; ++q) {
    const int idx = tid + q * GR_THREADS;
    if (idx < MLP_H * MLP_F) out[MLP_OFF_W1 + (idx / MLP_F) * MLP_IN + idx % MLP_F] = gW1[q];
  }
  for (int e = tid; e < MLP_H * MLP_IN; e += GR_THREADS)
    if (e % MLP_IN >= MLP_F) out[MLP_OFF_W1 + e] = 0.f;
  s.red[(eq * 3 + 0) * MLP_H + hq] = gb1;
  s.red[(eq * 3 + 1) * MLP_H + hq] = gb2;
  s.red[(eq * 3 + 2) * MLP_H + hq] = gw3;
  // the loss sum of the tile rows lives in threads 0..31: reduce within warp 0
  if (tid < 32) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
  }
  __syncthreads();
  if (tid < MLP_H) {
    float a = 0.f, b = 0.f, c = 0.f;
    for (int g = 0; g < 4; ++g) {
      a += s.red[(g * 3 + 0) * MLP_H + tid];
      b += s.red[(g * 3 + 1) * MLP_H + tid];
      c += s.red[(g * 3 + 2) * MLP_H + tid];
    }
    out[MLP_OFF_B1 + tid] = a;
    out[MLP_OFF_B2 + tid] = b;
    out[MLP_OFF_W3 + tid] = c;
  }
  if (tid == 0) {
    out[MLP_OFF_B3] = gb3;
    for (int q = 1; q < 8; ++q) out[MLP_OFF_B3 + q] = 0.f;
    out[MLP_PARAMS] = lsum;
  }
}

// Sum the partial gradients over the CTAs in CTA order; the loss in float64.
__global__ void reduce_kernel(const float *partial, int nblk, float *grad, double *loss,
                              int64_t total) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < MLP_PARAMS) {
    float a = 0.f;
    for (int b = 0; b < nblk; ++b) a += partial[int64_t(b) * GR_STRIDE + p];
    grad[p] = a;
  } else if (p == MLP_PARAMS) {
    double a = 0.0;
    for (int b = 0; b < nblk; ++b) a += (double)partial[int64_t(b) * GR_STRIDE + p];
    *loss = a / double(total);
  }
}

__global__ void adam_kernel(float *th, float *m, float *v, const float *g, float lr, float b1,
                            float b2, float eps, float c1, float c2, uint16_t *out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= MLP_PARAMS) return;
  const float gp = g[p];
  const float mp = b1 * m[p] + (1.f - b1) * gp;
  const float vp = b2 * v[p] + (1.f - b2) * gp * gp;
  m[p] = mp;
  v[p] = vp;
  const float t = th[p] - lr * (mp / c1) / (sqrtf(vp / c2) + eps);
  th[p] = t;
  const __nv_bfloat16 b = __float2bfloat16_rn(t);
  out[p] = *reinterpret_cast<const uint16_t *>(&b);
}

__global__ void pack_kernel(const float *th, uint16_t *out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= MLP_PARAMS) return;
  const __nv_bfloat16 b = __float2bfloat16_rn(th[p]);
  out[p] = *reinterpret_cast<const uint16_t *>(&b);
}

// Delta of example rows by the sampler's warp-level tensor-core network.
__global__ void __launch_bounds__(128) forward_kernel(const float *feat, int64_t n_ex,
                                                      const uint16_t *prm, float *delta) {
  __shared__ MlpSmem P;
  mlp_stage(&P, prm, threadIdx.x, blockDim.x);
  __syncthreads();
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int64_t base = (int64_t(blockIdx.x) * (blockDim.x / 32) + (threadIdx.x >> 5)) * 16;
  uint32_t xw[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int64_t row = base + g + 8 * h;
    float2 f = make_float2(0.f, 0.f);
    if (row < n_ex) f = reinterpret_cast<const float2 *>(feat + row * 8)[t];
    xw[h] = pack_bf16(f.x, f.y);
  }
  const float2 d = mlp_warp16(&P, xw[0], xw[1], lane);
  if (t == 0) {
    if (base + g < n_ex) delta[base + g] = d.x;
    if (base + g + 8 < n_ex) delta[base + g + 8] = d.y;
  }
}

bool aligned(const void *p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

}  // namespace

cudaError_t launch_mlp_features(const Layout &lay, int S, int L_max, const uint8_t *spins,
                                const float *logits, float *feat, cudaStream_t st) {
  const int64_t per = int64_t(S) * L_max * L_max;
  const dim3 grid(unsigned((per + 255) / 256), unsigned(lay.n_real));
  features_kernel<<<grid, 256, 0, st>>>(lay, S, spins, logits, feat);
  return cudaGetLastError();
}

}  // namespace tnmc

using namespace tnmc;

extern "C" {

size_t tnmc_mlp_scratch_floats(void) { return size_t(GR_BLOCKS) * GR_STRIDE; }

tnmc_status tnmc_mlp_grad(const float *d_feat, const float *d_target_logit, int64_t n_ex,
                          int32_t B, uint64_t seed, int32_t step, const void *d_params_bf16,
                          float *d_grad, double *d_loss, float *d_scratch, void *stream) {
  if (!d_feat || !d_target_logit || !d_params_bf16 || !d_grad || !d_loss || !d_scratch)
    return TNMC_ERR_ARG;
  if (n_ex < 1 || B < 0 || !aligned(d_feat, 16) || !aligned(d_params_bf16, 16)) return TNMC_ERR_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int smem = int(sizeof(GradSmem));
  cudaError_t e = cudaFuncSetAttribute(grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return TNMC_ERR_CUDA;
  grad_kernel<<<GR_BLOCKS, GR_THREADS, smem, st>>>(d_feat, d_target_logit, n_ex, B, seed, step,
                                                   static_cast<const uint16_t *>(d_params_bf16),
                                                   d_scratch);
  const int64_t total = B > 0 ? int64_t(B) : n_ex;
  reduce_kernel<<<(MLP_PARAMS + 1 + 255) / 256, 256, 0, st>>>(d_scratch, GR_BLOCKS, d_grad, d_loss,
                                                              total);
  return cudaGetLastError() == cudaSuccess ? TNMC_OK : TNMC_ERR_CUDA;
}

tnmc_status tnmc_mlp_adam(float *d_master, float *d_m, float *d_v, const float *d_grad,
                          int32_t step, float lr, float beta1, float beta2, float eps,
                          void *d_params_bf16, void *stream) {
  if (!d_master || !d_m || !d_v || !d_grad || !d_params_bf16 || step < 1) return TNMC_ERR_ARG;
  if (!(beta1 >= 0.f && beta1 < 1.f && beta2 >= 0.f && beta2 < 1.f && eps > 0.f)) return TNMC_ERR_ARG;
  const float c1 = float(1.0 - std::pow(double(beta1), double(step)));
  const float c2 = float(1.0 - std::pow(double(beta2), double(step)));
  adam_kernel<<<(MLP_PARAMS + 255) / 256, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      d_master, d_m, d_v, d_grad, lr, beta1, beta2, eps, c1, c2,
      static_cast<uint16_t *>(d_params_bf16));
  return cudaGetLastError() == cudaSuccess ? TNMC_OK : TNMC_ERR_CUDA;
}

tnmc_status tnmc_mlp_pack(const float *d_master, void *d_params_bf16, void *stream) {
  if (!d_master || !d_params_bf16) return TNMC_ERR_ARG;
  pack_kernel<<<(MLP_PARAMS + 255) / 256, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      d_master, static_cast<uint16_t *>(d_params_bf16));
  return cudaGetLastError() == cudaSuccess ? TNMC_OK : TNMC_ERR_CUDA;
}

tnmc_status tnmc_mlp_forward(const float *d_feat, int64_t n_ex, const void *d_params_bf16,
                             float *d_delta, void *stream) {
  if (!d_feat || !d_params_bf16 || !d_delta || n_ex < 1) return TNMC_ERR_ARG;
  if (!aligned(d_feat, 16) || !aligned(d_params_bf16, 16)) return TNMC_ERR_ARG;
  const int64_t blocks = (n_ex + 63) / 64;
  if (blocks > 0x7fffffff) return TNMC_ERR_ARG;
  forward_kernel<<<unsigned(blocks), 128, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      d_feat, n_ex, static_cast<const uint16_t *>(d_params_bf16), d_delta);
  return cudaGetLastError() == cudaSuccess ? TNMC_OK : TNMC_ERR_CUDA;
}

}  // extern "C"
