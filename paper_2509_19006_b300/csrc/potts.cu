// q-state Potts extension (Sec. 5: the method carries over to Potts models with the
// physical index of every tensor widened to q states), in float64 or float32 (the element
// type T of the build, the cache and the sampling contractions; per-draw probabilities, log
// scales, log q and energies are float64), batched over realizations x samples like the
// Ising path:
//   E(s) = - sum_<ij> J_ij delta(s_i, s_j),  s_i in {0 .. q-1}.
// There is no parity form here (the Z2 symmetry of the Ising model has no q-state
// analogue that halves the storage), so every site is a dense chi x q x chi tensor,
// stored as A[s][a][b] (q matrices chi x chi, zero padded), and every QR and SVD runs
// on the whole matrix.
//
// potts_build_kernel: one persistent 512-thread CTA per realization. For row r = L-1 .. 0
// the row's transfer MPO (copy tensors W[a, s, b, n] = delta(a, s) Bh[s, b] Bv[s, n], with
// the normalised Boltzmann matrices B(J)[a, b] = exp(beta J delta(a, b) - beta max(J, 0)))
// is applied to the row below and the result compressed back to chi:
//   phase A (sites 0 -> L-1): C[s] = sum_n Bv[s, n] A_c[n] of the row below, the carried
//     triangular factor absorbed, T[(k, s), (b, b')] = Bh[s, b] sum_a' R[k, (s, a')] C[s][a', b'],
//     a Householder QR of T, R normalised (its norm into lambda_r), Q kept for phase B;
//   phase B (sites L-1 -> 0): Theta = Q_c (US) as (left bond) x (q x right bond), a pivoted
//     Householder QR of Theta, a one-sided Jacobi SVD on the rows of [R | Q^T] (the Q^T block
//     ends as U^T), the chi largest singular values above cutoff x largest kept, V^T stored,
//     U S / s_max carried.
// The bottom row is the same sweep over a trivial row below (C = 1).
//
// potts_sample_kernel: one warp per chain, eight chains per CTA sharing the staged site
// tensors; right environments R_c = (sum_s Bv(r-1)[s_up, s] A_{c+1}[s]) R_{c+1} spilled to
// the sampler scratch, then the left sweep: rho_s = | l A_c[s] R_c |, p(s) proportional to
// rho_s Bv(r-1, c)[s_up, s], the state drawn as the first k with u < p_0 + ... + p_k
// (float64 partial sums), log q += log p_k, E += -Jh delta - Jv delta (left bond, then up).
#include "common.cuh"

namespace tnmc {

namespace {

constexpr int PT = 512;          // threads of the build CTA
constexpr int PQ = 4;            // largest q
constexpr int PCH = 16;          // largest chi
constexpr int PD = 48;           // largest q x chi (bond of MPO x MPS)
constexpr int PM = 144;          // largest panel rows (q x PD); q^2 chi <= 144
constexpr int PLDT = 2 * PD + 1; // row stride of [Theta | U^T]
constexpr int P_MAX_SWEEPS = 40;

struct PottsSmem {
  static constexpr int oA = 0;                     // panel, column-major, ld PM
  static constexpr int oR = oA + PM * PD;          // R (row-major, ld PD)
  static constexpr int oC = oR + PD * PD;          // C[s][a'][b'] (ld PCH)
  static constexpr int oT = oC + PQ * PCH * PCH;   // [Theta | U^T] (ld PLDT)
  static constexpr int oU = oT + PD * PLDT;        // U S (row-major, ld PCH)
  static constexpr int oTau = oU + PD * PCH;
  static constexpr int oSn = oTau + PD;
  static constexpr int n = oSn + PD;   // values of the element type
};

template <typename T>
__device__ __forceinline__ T pwarp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// normalised Boltzmann weight of a bond: exp(beta J delta(a, b) - beta max(J, 0))
__device__ __forceinline__ double pweight(double beta, double J, bool same) {
  return exp(beta * J * (same ? 1.0 : 0.0) - beta * fmax(J, 0.0));
}

// Householder QR of the m x n column-major panel A (ld PM) by the whole CTA (LAPACK's
// geqr2 scheme, beta = -sign(x0) |x|; reflectors below the diagonal with v_j = 1 implied).
template <typename T>
__device__ void p_householder(T *A, int m, int n, T *tau) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int kq = min(m, n);
  for (int j = 0; j < kq; ++j) {
    T *col = A + j * PM;
    if (warp == 0) {
      T s2 = T(0);
      for (int i = j + 1 + lane; i < m; i += 32) s2 += col[i] * col[i];
      s2 = pwarp_sum(s2);
      const T x0 = col[j];
      if (s2 == T(0)) {
        if (lane == 0) tau[j] = T(0);
      } else {
        const T mu = sqrt(x0 * x0 + s2);
        const T be = x0 <= T(0) ? mu : -mu;
        const T sc = T(1) / (x0 - be);
        for (int i = j + 1 + lane; i < m; i += 32) col[i] *= sc;
        if (lane == 0) { tau[j] = (be - x0) / be; col[j] = be; }
      }
    }
    __syncthreads();
    const T tj = tau[j];
    if (tj != T(0)) {
      for (int k = j + 1 + warp; k < n; k += PT / 32) {
        T *ck = A + k * PM;
        T w = lane == 0 ? ck[j] : T(0);
        for (int i = j + 1 + lane; i < m; i += 32) w += col[i] * ck[i];
        w = pwarp_sum(w) * tj;
        if (lane == 0) ck[j] -= w;
        for (int i = j + 1 + lane; i < m; i += 32) ck[i] -= w * col[i];
      }
    }
    __syncthreads();
  }
}

// Explicit Q (m x kq) in place of the reflectors (LAPACK's org2r order).
template <typename T>
__device__ void p_form_q(T *A, const T *tau, int m, int kq) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int j = kq - 1; j >= 0; --j) {
    const T tj = tau[j];
    const T *v = A + j * PM;
    if (tj != T(0)) {
      for (int l = j + 1 + warp; l < kq; l += PT / 32) {
        T *ql = A + l * PM;
        T w = lane == 0 ? ql[j] : T(0);
        for (int i = j + 1 + lane; i < m; i += 32) w += v[i] * ql[i];
        w = pwarp_sum(w) * tj;
        if (lane == 0) ql[j] -= w;
        for (int i = j + 1 + lane; i < m; i += 32) ql[i] -= w * v[i];
      }
    }
    __syncthreads();
    if (warp == 0) {
      T *qj = A + j * PM;
      for (int i = lane; i < m; i += 32) {
        if (i < j) qj[i] = T(0);
        else if (i == j) qj[i] = T(1) - tj;
        else qj[i] = -tj * qj[i];
      }
    }
    __syncthreads();
  }
}

// Householder QR with column pivoting (Businger & Golub, 1965) of the row-major m x n
// matrix A (element (i, j) at A[i * PLDT + j]) by the whole CTA: at step j the remaining
// column of largest norm below row j (ties: lower index) is swapped into place; R ends in
// the upper triangle, the reflectors below it, piv[k] = the original index of column k.
// The column norms below the current row are recomputed exactly in every update pass.
template <typename T>
__device__ void p_qr_pivot_rows(T *A, int m, int n, T *tau, T *cn, int *piv) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int kq = min(m, n);
  for (int k = warp; k < n; k += PT / 32) {
    T s2 = T(0);
    for (int i = lane; i < m; i += 32) s2 += A[i * PLDT + k] * A[i * PLDT + k];
    s2 = pwarp_sum(s2);
    if (lane == 0) { cn[k] = s2; piv[k] = k; }
  }
  __syncthreads();
  for (int j = 0; j < kq; ++j) {
    if (warp == 0) {
      T best = T(-1);
      int bk = j;
      for (int k = j + lane; k < n; k += 32)
        if (cn[k] > best) { best = cn[k]; bk = k; }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const T ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int ok = __shfl_xor_sync(0xffffffffu, bk, o);
        if (ob > best || (ob == best && ok < bk)) { best = ob; bk = ok; }
      }
      if (bk != j) {
        for (int i = lane; i < m; i += 32) {
          const T x = A[i * PLDT + j];
          A[i * PLDT + j] = A[i * PLDT + bk];
          A[i * PLDT + bk] = x;
        }
        if (lane == 0) {
          const T c = cn[j]; cn[j] = cn[bk]; cn[bk] = c;
          const int p = piv[j]; piv[j] = piv[bk]; piv[bk] = p;
        }
      }
      __syncwarp();
      T s2 = T(0);
      for (int i = j + 1 + lane; i < m; i += 32) s2 += A[i * PLDT + j] * A[i * PLDT + j];
      s2 = pwarp_sum(s2);
      const T x0 = A[j * PLDT + j];
      if (s2 == T(0)) {
        if (lane == 0) tau[j] = T(0);
      } else {
        const T mu = sqrt(x0 * x0 + s2);
        const T be = x0 <= T(0) ? mu : -mu;
        const T sc = T(1) / (x0 - be);
        for (int i = j + 1 + lane; i < m; i += 32) A[i * PLDT + j] *= sc;
        if (lane == 0) { tau[j] = (be - x0) / be; A[j * PLDT + j] = be; }
      }
    }
    __syncthreads();
    const T tj = tau[j];
    for (int k = j + 1 + warp; k < n; k += PT / 32) {
      T w = lane == 0 ? A[j * PLDT + k] : T(0);
      for (int i = j + 1 + lane; i < m; i += 32) w += A[i * PLDT + j] * A[i * PLDT + k];
      w = pwarp_sum(w) * tj;
      if (lane == 0) A[j * PLDT + k] -= w;
      T nn = T(0);
      for (int i = j + 1 + lane; i < m; i += 32) {
        const T x = A[i * PLDT + k] - w * A[i * PLDT + j];
        A[i * PLDT + k] = x;
        nn += x * x;
      }
      nn = pwarp_sum(nn);
      if (lane == 0) cn[k] = nn;
    }
    __syncthreads();
  }
}

// Rotation of one Jacobi pair (alpha = |a|^2, beta = |b|^2, gamma = a . b): the tangent t of
// the angle that makes the rows orthogonal, computed in float32 after an exact
// power-of-two rescale (B300's float64 divide and square root take ~700 cycles each),
// then c = 1 / sqrt(1 + t^2) by two Newton steps from the float32 reciprocal square root,
// so that c^2 (1 + t^2) = 1 to float64 rounding: (c, s = c t) is an exact rotation whose
// angle is the Jacobi angle to ~1e-7; the residual inner product is left to the next sweep.
__device__ __forceinline__ void p_rotation(double al, double be, double ga, double &t, double &cs,
                                           double &sn) {
  const long long bits = __double_as_longlong(fmax(al, be));
  const int e = int((bits >> 52) & 0x7ff) - 1023;
  const double sc = __longlong_as_double((long long)(1023 - e) << 52);   // 2^-e, exact
  const float d = float((be - al) * sc), g2 = 2.f * float(ga * sc);
  const float zf = d / g2;
  float tf;
  if (fabsf(zf) > 1e18f) tf = 0.5f / zf;
  else tf = (zf >= 0.f ? 1.f : -1.f) / (fabsf(zf) + sqrtf(1.f + zf * zf));
  t = double(tf);
  const double x = 1.0 + t * t;
  double y = double(rsqrtf(float(x)));
  y = y * (1.5 - 0.5 * x * y * y);
  y = y * (1.5 - 0.5 * x * y * y);
  cs = y;
  sn = y * t;
}

// float32: the plain Jacobi rotation (float32 division and square root are cheap); c and
// s form an exact rotation to float32 rounding.
__device__ __forceinline__ void p_rotation(float al, float be, float ga, float &t, float &cs, float &sn) {
  const float zeta = (be - al) / (2.f * ga);
  t = fabsf(zeta) > 1e18f ? 0.5f / zeta : (zeta >= 0.f ? 1.f : -1.f) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
  cs = 1.f / sqrtf(1.f + t * t);
  sn = cs * t;
}

// One-sided Jacobi on the nr rows of B (ld PLDT): inner products over the first nc
// columns, rotations over nc + nu columns. Round-robin (circle) schedule, 16 lanes per
// row pair. The squared row norms are measured exactly at the start of every sweep and
// updated within it (alpha - t gamma, beta + t gamma), so a round computes one inner
// product per pair. A pair is rotated while |gamma| > tol sqrt(alpha beta), tol = 8
// sqrt(nc) eps, unless either row is below eps x the largest row (rounding noise).
// Returns the sweeps taken.
template <typename T>
__device__ int p_jacobi(T *B, int nr, int nc, int nu, int *sh_flag, T *nrm2) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (nr <= 1) return 0;
  constexpr int TPP = 16;
  const int P = nr + (nr & 1), np = P / 2;
  const int g = tid / TPP, gl = tid % TPP;
  // tol = 8 sqrt(nc) eps in float64, 4 sqrt(nc) eps in float32 (rows orthogonal closer to the
  // rounding floor at float32's cheap rounds)
  const T eps = T(Num<T>::eps());
  const T tol2 = T(sizeof(T) == 4 ? 16 : 64) * eps * eps * T(nc > 4 ? nc : 4);
  __shared__ T sh_mx;
  int sweep = 0;
  for (; sweep < P_MAX_SWEEPS; ++sweep) {
    // exact squared norms, one warp per row
    for (int i = warp; i < nr; i += PT / 32) {
      T s2 = T(0);
      for (int x = lane; x < nc; x += 32) s2 += B[i * PLDT + x] * B[i * PLDT + x];
      s2 = pwarp_sum(s2);
      if (lane == 0) nrm2[i] = s2;
    }
    if (tid == 0) *sh_flag = 0;
    __syncthreads();
    if (tid == 0 && sweep == 0) {
      T mx = T(0);
      for (int i = 0; i < nr; ++i) mx = nrm2[i] > mx ? nrm2[i] : mx;
      sh_mx = mx;
    }
    __syncthreads();
    const T floor2 = sh_mx * eps * eps;
    for (int k = 0; k < P - 1; ++k) {
      int i = -1, j = -1;
      if (g < np) {
        const int p0 = g, p1 = P - 1 - g;
        i = p0 == 0 ? 0 : 1 + (p0 - 1 + k) % (P - 1);
        j = 1 + (p1 - 1 + k) % (P - 1);
        if (i >= nr || j >= nr) i = j = -1;
      }
      T ga = T(0);
      if (i >= 0) {
        const T *a = B + i * PLDT, *b = B + j * PLDT;
        for (int x = gl; x < nc; x += TPP) ga += a[x] * b[x];
      }
#pragma unroll
      for (int o = TPP / 2; o > 0; o >>= 1) ga += __shfl_xor_sync(0xffffffffu, ga, o);
      if (i >= 0) {
        const T al = nrm2[i], be = nrm2[j];
        if (al > floor2 && be > floor2 && ga * ga > tol2 * al * be) {
          T t, cs, sn;
          p_rotation(al, be, ga, t, cs, sn);
          T *a = B + i * PLDT, *b = B + j * PLDT;
          for (int x = gl; x < nc + nu; x += TPP) {
            const T av = a[x], bv = b[x];
            a[x] = cs * av - sn * bv;
            b[x] = sn * av + cs * bv;
          }
          __syncwarp(0xffffu << (tid & 16));   // the pair's 16 lanes have read the norms
          if (gl == 0) { nrm2[i] = al - t * ga; nrm2[j] = be + t * ga; *sh_flag = 1; }
        }
      }
      __syncthreads();
    }
    const int rotated = *sh_flag;
    __syncthreads();
    if (!rotated) break;
  }
  return sweep + 1;
}

template <typename T>
__global__ void __launch_bounds__(PT, 1) potts_build_kernel(Layout lay, int q) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *W = (T *)smem_raw;
  T *Ap = W + PottsSmem::oA, *Rb = W + PottsSmem::oR, *Cs = W + PottsSmem::oC;
  T *Th = W + PottsSmem::oT, *US = W + PottsSmem::oU, *tau = W + PottsSmem::oTau;
  T *sn = W + PottsSmem::oSn;
  __shared__ double sh_red[PT / 32];
  __shared__ T sh_nrm2[PD];   // Jacobi row norms
  __shared__ T sh_cn[PD];     // column norms of the pivoted QR
  __shared__ int sh_piv[PD], sh_ipiv[PD];
  __shared__ double sh_lam, sh_smax, sh_flops, sh_dsum;
  __shared__ T sh_rscale;
  __shared__ int sh_n, sh_flag, sh_keep, sh_kprev, sh_sweeps, sh_svds;
  __shared__ long long sh_clk[4];   // cycles of the row: phase A, Theta products, Jacobi, selection + stores
  long long t_mark = 0;
  __shared__ int sh_src[PD];
  __shared__ T sh_Bh[PQ * PQ], sh_Bv[PQ * PQ];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int chi = lay.chi;
  const int64_t chi2 = int64_t(chi) * chi;
  const double beta = lay.beta;
  const int64_t site_vals = int64_t(q) * chi2;
  unsigned char *slot = (unsigned char *)lay.env_scratch + int64_t(blockIdx.x) * lay.env_slot_bytes;
  T *Qstore = (T *)slot;                                               // L_max panels PM x PD
  int2 *info = (int2 *)(slot + align256(int64_t(lay.L_max) * PM * PD * sizeof(T)));   // (kprev, kq) per site

  for (;;) {
    if (tid == 0) sh_n = atomicAdd(lay.counter, 1);
    __syncthreads();
    const int idx = sh_n;
    __syncthreads();
    if (idx >= lay.n_real) break;
    const int n = lay.order[idx];
    const RealInfo ri = lay.reals[n];
    const int L = ri.L;
    if (lay.flags[n] & FLAG_BAD_J) continue;   // uniform
    const float *jr = lay.jr + ri.site_off, *jd = lay.jd + ri.site_off;
    T *cache_n = (T *)lay.cache + ri.cache_off * site_vals;
    int2 *bonds_n = lay.bonds + ri.bond_off;
    if (tid == 0) sh_lam = 0.0;
    for (int r = L - 1; r >= 0; --r) {
      const bool bottom = (r == L - 1);
      const T *prev = bottom ? nullptr : cache_n + int64_t(r + 1) * L * site_vals;
      const int2 *bprev = bottom ? nullptr : bonds_n + int64_t(r + 1) * (L + 1);
      T *dst_row = cache_n + int64_t(r) * L * site_vals;
      // row constants: the normalisations of the row's Boltzmann matrices
      {
        double acc = 0.0;
        for (int c = tid; c < L; c += PT) {
          if (c < L - 1) acc += beta * fmax((double)jr[r * L + c], 0.0);
          if (!bottom) acc += beta * fmax((double)jd[r * L + c], 0.0);
        }
        acc = pwarp_sum(acc);
        if (lane == 0) sh_red[warp] = acc;
        __syncthreads();
        if (tid == 0) {
          double s = 0.0;
          for (int w = 0; w < PT / 32; ++w) s += sh_red[w];
          sh_lam += s;
          sh_kprev = 1;
          Rb[0] = T(1);
          sh_flops = 0.0; sh_dsum = 0.0; sh_sweeps = 0; sh_svds = 0;
          for (int f = 0; f < 4; ++f) sh_clk[f] = 0;
          t_mark = clock64();
        }
        __syncthreads();
      }
      // ===================== phase A: MPO x MPS with the carried R, QR sweep
      for (int c = 0; c < L; ++c) {
        const int Dl = bottom ? 1 : bprev[c].x, Dr = bottom ? 1 : bprev[c + 1].x;
        const bool last = (c == L - 1);
        const int Bdim = last ? 1 : q;
        const int kprev = sh_kprev;
        if (tid < q * q) {
          const int a = tid / q, b = tid % q;
          sh_Bh[tid] = T(last ? 1.0 : pweight(beta, (double)jr[r * L + c], a == b));
          sh_Bv[tid] = T(bottom ? 0.0 : pweight(beta, (double)jd[r * L + c], a == b));
        }
        __syncthreads();
        // C[s][a'][b'] = sum_n Bv[s, n] A_c[n][a'][b'] of the row below (1 on the bottom row)
        for (int e = tid; e < q * Dl * Dr; e += PT) {
          const int s = e / (Dl * Dr), rem = e % (Dl * Dr), a = rem / Dr, b = rem % Dr;
          T acc;
          if (bottom) {
            acc = T(1);
          } else {
            acc = T(0);
            const T *site = prev + int64_t(c) * site_vals;
            for (int nn = 0; nn < q; ++nn) acc += sh_Bv[s * q + nn] * site[(int64_t(nn) * chi + a) * chi + b];
          }
          Cs[(s * PCH + a) * PCH + b] = acc;
        }
        __syncthreads();
        // T[(k, s), (b, b')] = Bh[s, b] sum_a' R[k, (s, a')] C[s][a'][b'] (site 0: R = 1, a' = 0)
        const int m = kprev * q, ncol = Bdim * Dr;
        for (int e = tid; e < m * ncol; e += PT) {
          const int row = e / ncol, col = e % ncol;
          const int k = row / q, s = row % q, b = col / Dr, bb = col % Dr;
          T acc = T(0);
          if (c == 0) {
            acc = Cs[(s * PCH + 0) * PCH + bb];
          } else {
            const T *Rk = Rb + k * PD + s * Dl;
            for (int a = 0; a < Dl; ++a) acc += Rk[a] * Cs[(s * PCH + a) * PCH + bb];
          }
          Ap[row + col * PM] = sh_Bh[s * q + b] * acc;
        }
        __syncthreads();
        if (last) break;   // the last site starts phase B from the panel
        p_householder(Ap, m, ncol, tau);
        const int kq = min(m, ncol);
        // R = upper trapezoid (kq x ncol), normalised
        {
          double acc = 0.0;
          for (int e = tid; e < kq * ncol; e += PT) {
            const int i = e / ncol, b = e % ncol;
            if (b >= i) { const double v = double(Ap[i + b * PM]); acc += v * v; }
          }
          acc = pwarp_sum(acc);
          if (lane == 0) sh_red[warp] = acc;
          __syncthreads();
          if (tid == 0) {   // the scalar chain on one thread (not 16 warps on the float64 pipe)
            double nrm2 = 0.0;
            for (int w = 0; w < PT / 32; ++w) nrm2 += sh_red[w];
            const double nrm = sqrt(nrm2);
            const bool ok = nrm > 0.0 && isfinite(nrm);
            sh_rscale = ok ? T(1.0 / nrm) : T(0);
            if (ok) sh_lam += log(nrm);
            else set_flag(lay.flags, n, FLAG_NUMERIC);
          }
          __syncthreads();
          const T inv = sh_rscale;
          for (int e = tid; e < kq * ncol; e += PT) {
            const int i = e / ncol, b = e % ncol;
            Rb[i * PD + b] = (b >= i) ? Ap[i + b * PM] * inv : T(0);
          }
        }
        __syncthreads();
        p_form_q(Ap, tau, m, kq);
        T *qs = Qstore + int64_t(c) * PM * PD;
        for (int e = tid; e < m * kq; e += PT) {
          const int col = e / m, i = e % m;
          qs[i + col * PM] = Ap[i + col * PM];
        }
        if (tid == 0) {
          info[c] = make_int2(kprev, kq);
          sh_kprev = kq;
          // textbook flops: the MPO x MPS product, Householder QR with explicit Q
          const double mm = m, nn = ncol, kk = kq;
          sh_flops += 2.0 * mm * nn * (c == 0 ? 1.0 : Dl) + 2.0 * (2.0 * mm * nn * kk - 2.0 * kk * kk * kk / 3.0);
        }
        __syncthreads();
      }
      if (tid == 0) { const long long t1 = clock64(); sh_clk[0] += t1 - t_mark; t_mark = t1; }
      // ===================== phase B: truncating SVD sweep, right to left
      int kr = 1;   // kept bond to the right of the current site
      for (int c = L - 1; c >= 0; --c) {
        const int Dl = (c == L - 1) ? sh_kprev : info[c].x;   // left bond of site c
        const int nc = q * kr;
        // Theta[a][(s, j)]
        if (c == L - 1) {
          for (int e = tid; e < Dl * q; e += PT) {
            const int a = e / q, s = e % q;
            Th[a * PLDT + s] = Ap[(a * q + s) + 0 * PM];
          }
        } else {
          const int kq = info[c].y;
          const T *qs = Qstore + int64_t(c) * PM * PD;
          for (int e = tid; e < Dl * nc; e += PT) {
            const int a = e / nc, col = e % nc, s = col / kr, j = col % kr;
            T acc = T(0);
            for (int p = 0; p < kq; ++p) acc += qs[(a * q + s) + p * PM] * US[p * PCH + j];
            Th[a * PLDT + col] = acc;
          }
        }
        __syncthreads();
        if (tid == 0) { const long long t1 = clock64(); sh_clk[1] += t1 - t_mark; t_mark = t1; }
        T *site_dst = dst_row + int64_t(c) * site_vals;
        if (c == 0) {
          // site 0 (left bond 1): divided by its norm
          double acc = 0.0;
          for (int x = tid; x < nc; x += PT) acc += double(Th[x]) * double(Th[x]);
          acc = pwarp_sum(acc);
          if (lane == 0) sh_red[warp] = acc;
          __syncthreads();
          double nrm2 = 0.0;
          for (int w = 0; w < PT / 32; ++w) nrm2 += sh_red[w];
          const double nrm = sqrt(nrm2);
          const bool ok = nrm > 0.0 && isfinite(nrm);
          const T inv = ok ? T(1.0 / nrm) : T(0);
          for (int64_t e = tid; e < site_vals; e += PT) {
            const int s = int(e / chi2), rem = int(e % chi2), a = rem / chi, b = rem % chi;
            site_dst[e] = (a == 0 && b < kr) ? Th[s * kr + b] * inv : T(0);
          }
          if (tid == 0) {
            if (ok) sh_lam += log(nrm);
            else set_flag(lay.flags, n, FLAG_NUMERIC);
            bonds_n[int64_t(r) * (L + 1) + 0] = make_int2(1, 0);
            bonds_n[int64_t(r) * (L + 1) + L] = make_int2(1, 0);
            if (L > 1) bonds_n[int64_t(r) * (L + 1) + 1] = make_int2(kr, 0);
            lay.lam[ri.row_off + r] = sh_lam;
            if (lay.dbg_rowinfo) {   // the Ising build's row record: bond, sweeps and flops fields
              double *ro = lay.dbg_rowinfo + (ri.row_off + r) * 14;
              for (int f = 0; f < 14; ++f) ro[f] = 0.0;
              ro[5] = L > 1 ? sh_dsum / (L - 1) : 1.0;
              ro[6] = sh_svds;
              ro[7] = sh_svds > 0 ? double(sh_sweeps) / sh_svds : 0.0;
              for (int f = 0; f < 4; ++f) ro[8 + f] = double(sh_clk[f]);
              ro[13] = sh_flops;
            }
          }
          __syncthreads();
          break;
        }
        // QR preconditioning: Theta P = Q R (pivoted Householder), then the sweeps rotate the
        // rr = min(Dl, nc) rows of [R | Q^T], which end as S V^T P and U^T; one-sided Jacobi on
        // the graded triangular factor needs far fewer sweeps than on [Theta | I]
        // (Drmac & Veselic, SIAM J. Matrix Anal. Appl. 29, 2008). P is undone at the store.
        const int rr = min(Dl, nc);
        p_qr_pivot_rows(Th, Dl, nc, tau, sh_cn, sh_piv);
        for (int e = tid; e < Dl * rr; e += PT) {   // reflectors to Ap (column-major), R kept
          const int i = e / rr, j = e % rr;
          T v = T(0);
          if (i > j) { v = Th[i * PLDT + j]; Th[i * PLDT + j] = T(0); }
          Ap[i + j * PM] = v;
        }
        for (int b = tid; b < nc; b += PT) sh_ipiv[sh_piv[b]] = b;
        __syncthreads();
        p_form_q(Ap, tau, Dl, rr);
        for (int e = tid; e < rr * Dl; e += PT) {
          const int i = e / Dl, p = e % Dl;
          Th[i * PLDT + nc + p] = Ap[p + i * PM];
        }
        __syncthreads();
        const int nsw = p_jacobi(Th, rr, nc, Dl, &sh_flag, sh_nrm2);
        if (tid == 0) { const long long t1 = clock64(); sh_clk[2] += t1 - t_mark; t_mark = t1; }
        // singular values = row norms; keep the chi largest above cutoff x largest
        for (int i = tid; i < rr; i += PT) {
          T s2 = T(0);
          for (int x = 0; x < nc; ++x) s2 += Th[i * PLDT + x] * Th[i * PLDT + x];
          sn[i] = sqrt(s2);
        }
        __syncthreads();
        if (tid == 0) {
          T mx = T(0);
          for (int i = 0; i < rr; ++i) mx = sn[i] > mx ? sn[i] : mx;
          sh_smax = double(mx);
        }
        __syncthreads();
        const double smax = sh_smax, thr = smax * lay.cutoff;
        if (tid < rr) {
          const int i = tid;
          int rank = 0;
          for (int j = 0; j < rr; ++j) rank += (sn[j] > sn[i]) || (sn[j] == sn[i] && j < i);
          const bool keep = rank < chi && (sn[i] > thr || rank == 0);
          if (keep) sh_src[rank] = i;
        }
        if (tid == 0) {
          int kk = 0;
          for (int i = 0; i < rr; ++i) {
            int rank = 0;
            for (int j = 0; j < rr; ++j) rank += (sn[j] > sn[i]) || (sn[j] == sn[i] && j < i);
            kk += (rank < chi && (sn[i] > thr || rank == 0)) ? 1 : 0;
          }
          sh_keep = kk;
          sh_dsum += kk;
          if (nsw > 0) { sh_sweeps += nsw; sh_svds += 1; }
          // textbook flops: the Theta product and a Golub-Reinsch SVD of the Dl x nc matrix
          const double a = Dl > nc ? Dl : nc, b = Dl > nc ? nc : Dl;
          sh_flops += 4.0 * a * a * b + 8.0 * a * b * b + 9.0 * b * b * b;
          if (c < L - 1) sh_flops += 2.0 * Dl * q * double(info[c].y) * kr;
          if (smax > 0.0 && isfinite(smax)) sh_lam += log(smax);
          else set_flag(lay.flags, n, FLAG_NUMERIC);
        }
        __syncthreads();
        const int kk = sh_keep;
        // cache site c: A[s][a''][j] = V^T[a''][(s, j)]
        for (int64_t e = tid; e < site_vals; e += PT) {
          const int s = int(e / chi2), rem = int(e % chi2), a = rem / chi, b = rem % chi;
          T v = T(0);
          if (a < kk && b < kr) {
            const int i = sh_src[a];
            v = Th[i * PLDT + sh_ipiv[s * kr + b]] / sn[i];   // column (s, b) sits at ipiv
          }
          site_dst[e] = v;
        }
        // U S / s_max for site c - 1 (rows: the left bond of site c)
        const T inv = smax > 0.0 ? T(1.0 / smax) : T(0);
        for (int e = tid; e < Dl * kk; e += PT) {
          const int p = e / kk, a = e % kk;
          const int i = sh_src[a];
          US[p * PCH + a] = Th[i * PLDT + nc + p] * sn[i] * inv;
        }
        if (tid == 0) bonds_n[int64_t(r) * (L + 1) + c] = make_int2(kk, 0);
        kr = kk;
        __syncthreads();
        if (tid == 0) { const long long t1 = clock64(); sh_clk[3] += t1 - t_mark; t_mark = t1; }
      }
    }
  }
}

// log Z = lambda_0 + log sum over the top row's states (Eq. 6); one warp per realization.
template <typename T>
__global__ void potts_log_z_kernel(Layout lay, int q, double *logz) {
  const int n = blockIdx.x;
  const int lane = threadIdx.x;
  const RealInfo ri = lay.reals[n];
  const int L = ri.L, chi = lay.chi;
  const int64_t chi2 = int64_t(chi) * chi, site_vals = int64_t(q) * chi2;
  const T *row0 = (const T *)lay.cache + ri.cache_off * site_vals;
  const int2 *b0 = lay.bonds + ri.bond_off;
  double v = lane == 0 ? 1.0 : 0.0, lacc = 0.0;
  for (int c = 0; c < L; ++c) {
    const int Dl = b0[c].x, Dr = b0[c + 1].x;
    const T *A = row0 + int64_t(c) * site_vals;
    double acc = 0.0;
    for (int a = 0; a < Dl; ++a) {
      const double va = __shfl_sync(0xffffffffu, v, a);
      if (lane < Dr)
        for (int s = 0; s < q; ++s) acc += va * double(A[(int64_t(s) * chi + a) * chi + lane]);
    }
    const double nrm = sqrt(pwarp_sum(acc * acc));
    v = nrm > 0.0 ? acc / nrm : 0.0;
    lacc += log(nrm);
  }
  if (lane == 0) {
    const double val = lay.lam[ri.row_off] + lacc + log(fabs(v));
    logz[n] = val;
    if (!isfinite(val)) set_flag(lay.flags, n, FLAG_NUMERIC);
  }
}

constexpr int PS_CHAINS = 8;   // chains (warps) per sampler CTA

// Proposals (FORCED = false) or teacher-forced scores (FORCED = true) of S chains per
// realization; one warp per chain, lane b holds column b of the chain's vectors.
template <typename T, bool FORCED>
__global__ void __launch_bounds__(32 * PS_CHAINS) potts_sample_kernel(
    Layout lay, int q, int S, uint64_t seed, uint64_t prop_base, const uint8_t *in_states,
    uint8_t *out_states, double *out_logq, double *out_E) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *As = (T *)smem_raw;   // q x chi x chi of the current site
  const int bpr = (S + PS_CHAINS - 1) / PS_CHAINS;
  const int n = blockIdx.x / bpr;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int sid = (blockIdx.x % bpr) * PS_CHAINS + warp;
  const bool act = sid < S;
  const RealInfo ri = lay.reals[n];
  const int L = ri.L, chi = lay.chi;
  const int64_t chi2 = int64_t(chi) * chi, site_vals = int64_t(q) * chi2;
  const T *cache_n = (const T *)lay.cache + ri.cache_off * site_vals;
  const int2 *bonds_n = lay.bonds + ri.bond_off;
  const float *jr = lay.jr + ri.site_off, *jd = lay.jd + ri.site_off;
  const int64_t L2 = int64_t(L) * L;
  const double beta = lay.beta;
  T *rs = (T *)lay.samp_scratch + (ri.line_off * int64_t(lay.max_samples) + int64_t(act ? sid : 0) * L) * PCH;
  uint8_t *st = (FORCED ? nullptr : out_states + int64_t(S) * ri.site_off + int64_t(act ? sid : 0) * L2);
  const uint8_t *st_in = FORCED ? in_states + int64_t(S) * ri.site_off + int64_t(act ? sid : 0) * L2 : nullptr;
  auto state_at = [&](int i) -> int { return FORCED ? st_in[i] : st[i]; };
  double lq = 0.0, E = 0.0;
  int64_t group = -1;
  U64x4 words{};
  bool bad = false;
  auto stage = [&](const T *A) {
    __syncthreads();
    for (int64_t e = threadIdx.x; e < site_vals; e += blockDim.x) As[e] = A[e];
    __syncthreads();
  };
  for (int r = 0; r < L; ++r) {
    const T *row = cache_n + int64_t(r) * L * site_vals;
    const int2 *bd = bonds_n + int64_t(r) * (L + 1);
    // right pass: R_{L-1} = 1, R_c = T_{c+1}[s_up] R_{c+1}, normalised, spilled
    T Rv = lane == 0 ? T(1) : T(0);
    if (act && lane < PCH) rs[int64_t(L - 1) * PCH + lane] = Rv;
    for (int c = L - 2; c >= 0; --c) {
      stage(row + int64_t(c + 1) * site_vals);
      const int Dl = bd[c + 1].x, Dr = bd[c + 2].x;
      T w[PQ];
      const int su = (r > 0 && act) ? state_at((r - 1) * L + c + 1) : 0;
#pragma unroll
      for (int s = 0; s < PQ; ++s)
        w[s] = T((s < q && r > 0) ? pweight(beta, (double)jd[(r - 1) * L + c + 1], s == su) : (s < q ? 1.0 : 0.0));
      T acc = T(0);
      for (int b = 0; b < Dr; ++b) {
        const T rb = __shfl_sync(0xffffffffu, Rv, b);
        if (lane < Dl) {
          T t = T(0);
#pragma unroll
          for (int s = 0; s < PQ; ++s)
            if (s < q) t += w[s] * As[(s * chi + lane) * chi + b];
          acc += t * rb;
        }
      }
      const T nrm = sqrt(pwarp_sum(acc * acc));
      Rv = nrm > T(0) ? acc / nrm : T(0);
      if (act && lane < PCH) rs[int64_t(c) * PCH + lane] = lane < Dl ? Rv : T(0);
    }
    __syncwarp();
    // left sweep
    T lv = lane == 0 ? T(1) : T(0);
    for (int c = 0; c < L; ++c) {
      stage(row + int64_t(c) * site_vals);
      const int Dl = bd[c].x, Dr = bd[c + 1].x;
      const T Rc = (lane < Dr) ? rs[int64_t(c) * PCH + lane] : T(0);
      T v[PQ], rho[PQ];
#pragma unroll
      for (int s = 0; s < PQ; ++s) v[s] = T(0);
      for (int a = 0; a < Dl; ++a) {
        const T la = __shfl_sync(0xffffffffu, lv, a);
        if (lane < Dr) {
#pragma unroll
          for (int s = 0; s < PQ; ++s)
            if (s < q) v[s] += la * As[(s * chi + a) * chi + lane];
        }
      }
      const int i = r * L + c;
      const int su = (r > 0 && act) ? state_at((r - 1) * L + c) : 0;
      double tot = 0.0;
#pragma unroll
      for (int s = 0; s < PQ; ++s) {
        rho[s] = T(0);
        if (s < q) {
          rho[s] = fabs(pwarp_sum(v[s] * Rc));
          if (r > 0) rho[s] *= T(pweight(beta, (double)jd[(r - 1) * L + c], s == su));
          tot += double(rho[s]);
        }
      }
      int k;
      if (FORCED) {
        k = act ? st_in[i] : 0;
      } else {
        if ((i >> 2) != group) {
          group = i >> 2;
          words = philox4x64_10((uint64_t)group, prop_base + (uint64_t)(act ? sid : 0), (uint64_t)ri.gid,
                                 TAG_SPIN, seed, 0ull);
        }
        const double u = word_to_uniform(words.x[i & 3]);
        k = q - 1;
        double cum = 0.0;
        bool found = false;
#pragma unroll
        for (int s = 0; s < PQ - 1; ++s) {
          if (s < q - 1 && !found) {
            cum += double(rho[s]) / tot;
            if (u < cum) { k = s; found = true; }
          }
        }
      }
      if (!(tot > 0.0) || !isfinite(tot)) bad = true;
      double rk = double(rho[0]);
#pragma unroll
      for (int s = 1; s < PQ; ++s) rk = (s == k) ? double(rho[s]) : rk;
      lq += log(rk / tot);
      if (c > 0) E -= (double)jr[r * L + c - 1] * (k == state_at(i - 1) ? 1.0 : 0.0);
      if (r > 0) E -= (double)jd[(r - 1) * L + c] * (k == su ? 1.0 : 0.0);
      if (!FORCED && act && lane == 0) st[i] = (uint8_t)k;
      __syncwarp();
      T vk = v[0];
#pragma unroll
      for (int s = 1; s < PQ; ++s) vk = (s == k) ? v[s] : vk;
      const T nrm = sqrt(pwarp_sum(vk * vk));
      lv = nrm > T(0) ? vk / nrm : T(0);
    }
  }
  if (act && lane == 0) {
    out_logq[int64_t(n) * S + sid] = lq;
    out_E[int64_t(n) * S + sid] = E;
    if (bad) set_flag(lay.flags, n, FLAG_NUMERIC);
  }
}

}  // namespace

int64_t potts_slot_bytes(int L_max, int esz) {
  return align256(int64_t(L_max) * PM * PD * esz) + align256(int64_t(L_max) * 8);
}

// q and chi limits of the Potts kernels (panel sizes in shared memory)
bool potts_supported(int q, int chi) { return q >= 3 && q <= PQ && chi <= PCH && q * q * chi <= PM; }

int potts_scratch_ch() { return PCH; }

template <typename T>
static cudaError_t launch_potts_build_t(const Layout &lay, int q, cudaStream_t st) {
  const int bytes = PottsSmem::n * int(sizeof(T));
  cudaError_t e = cudaFuncSetAttribute(potts_build_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(lay.counter, 0, sizeof(int32_t), st);
  if (e != cudaSuccess) return e;
  potts_build_kernel<T><<<lay.env_slots, PT, bytes, st>>>(lay, q);
  return cudaGetLastError();
}

// prec: 0 = float64, 1 = float32 (build, cache and sampling contractions)
cudaError_t launch_potts_build(const Layout &lay, int q, int prec, cudaStream_t st) {
  return prec == 1 ? launch_potts_build_t<float>(lay, q, st) : launch_potts_build_t<double>(lay, q, st);
}

cudaError_t launch_potts_log_z(const Layout &lay, int q, int prec, double *logz, cudaStream_t st) {
  if (prec == 1) potts_log_z_kernel<float><<<lay.n_real, 32, 0, st>>>(lay, q, logz);
  else potts_log_z_kernel<double><<<lay.n_real, 32, 0, st>>>(lay, q, logz);
  return cudaGetLastError();
}

template <typename T>
static void launch_potts_sample_t(const Layout &lay, int q, int S, uint64_t seed, uint64_t base,
                                  const uint8_t *in, uint8_t *out, double *lq, double *E, cudaStream_t st) {
  const int bpr = (S + PS_CHAINS - 1) / PS_CHAINS;
  const size_t smem = size_t(q) * lay.chi * lay.chi * sizeof(T);
  if (in) potts_sample_kernel<T, true><<<lay.n_real * bpr, 32 * PS_CHAINS, smem, st>>>(lay, q, S, seed, base, in, out, lq, E);
  else potts_sample_kernel<T, false><<<lay.n_real * bpr, 32 * PS_CHAINS, smem, st>>>(lay, q, S, seed, base, in, out, lq, E);
}

cudaError_t launch_potts_sample(const Layout &lay, int q, int prec, int S, uint64_t seed, uint64_t base,
                                const uint8_t *in, uint8_t *out, double *lq, double *E, cudaStream_t st) {
  if (prec == 1) launch_potts_sample_t<float>(lay, q, S, seed, base, in, out, lq, E, st);
  else launch_potts_sample_t<double>(lay, q, S, seed, base, in, out, lq, E, st);
  return cudaGetLastError();
}

}  // namespace tnmc
