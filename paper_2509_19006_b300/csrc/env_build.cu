// Boundary-MPS environment build (Sec. 2.2, Sec. 3.2, Fig. 2), one CTA per
// disorder realization, persistent over the batch (Sec. 3.4).
//
// For row r = L-1 .. 0 the kernel applies the row's transfer MPO to the MPS of
// row r+1 (the bond doubles) and compresses it back to chi:
//   phase A  left-to-right Householder QR sweep (left-canonical form);
//   phase B  right-to-left SVD sweep with one-sided Jacobi, keeping the chi
//            largest singular values at every bond.
// The MPS is held in parity form (see common.cuh): the MPO then never needs
// to be materialised. With normalised Boltzmann weights
//   exp(beta J s s') = cosh(beta J) (1 + t s s'),  t = tanh(beta J),
// the vertical bond of site c multiplies the odd part A(-) of the site by
// t_v = tanh(beta Jv[r][c]) (the even part by 1), and the horizontal bond
// (c, c+1) adds a two-valued index k to the bond: the new bond index is
// (k, a) with parity k xor par(a), and in parity form the new site matrix is
//   N[(k_l, a), (k_r, b)] = w(k_r) * Ct[a, b],  w(0) = 1, w(1) = t_h,
// with Ct the old site matrix whose odd-parity (off-diagonal) blocks are
// scaled by t_v. Every factor dropped by the normalisation (log cosh,
// log 2 cosh, norms) is accumulated into the float64 log scale lambda_r.
//
// The MPO x MPS product is block diagonal in the parity sectors, so each QR
// and SVD splits into two independent problems of half the size, which the
// two halves of the CTA (256 threads each) solve concurrently.
#include "common.cuh"
#include <cstdio>

namespace tnmc {

namespace {

constexpr int ENV_THREADS = 512;
constexpr int JACOBI_MAX_SWEEPS = 40;

template <typename T, int CH>
struct EnvPlan {
  static constexpr int LDA = 2 * CH;                 // rows of the column-major A / Q panels
  static constexpr int64_t CH2 = int64_t(CH) * CH;
  // phase A (units of T)
  static constexpr int64_t oCp = 0;                  // CH x CH, row-major (ld CH)
  static constexpr int64_t oR = CH2;                 // 2 x (CH x CH), row-major (ld CH)
  static constexpr int64_t oA = 3 * CH2;             // 2 x (2CH x CH), column-major (ld 2CH)
  static constexpr int64_t oQf = 7 * CH2;            // 2 x (2CH x CH), column-major (ld 2CH)
  // phase B (aliases phase A)
  static constexpr int64_t oQc = 0;                  // 2CH x 2CH, column-major (ld 2CH); later V^T
  static constexpr int LDT = 2 * CH;                 // row length of Theta | U^T
  static constexpr int64_t oTh = 4 * CH2;            // 2CH x 2CH, row-major (ld LDT)
  static constexpr int64_t oUS = 8 * CH2;            // 2 x (CH x CH), row-major (ld CH)
  static constexpr int64_t oTau = 11 * CH2;          // 2 x CH
  static constexpr int64_t oSn = oTau + 2 * CH;      // 2CH singular values
  static constexpr int64_t nT = oSn + 2 * CH;
  static constexpr int64_t bytes = nT * int64_t(sizeof(T));
  static constexpr bool in_smem = bytes <= 200 * 1024;
  // global scratch per slot: Q of every site + per-site dims (+ the arena when not in smem)
  static __host__ __device__ int64_t q_bytes(int L_max) { return align256(int64_t(L_max) * LDA * LDA * sizeof(T)); }
  static __host__ __device__ int64_t info_bytes(int L_max) { return align256(int64_t(L_max) * sizeof(int4)); }
  static __host__ __device__ int64_t slot_bytes(int L_max) {
    return q_bytes(L_max) + info_bytes(L_max) + (in_smem ? 0 : align256(bytes));
  }
};

__device__ __forceinline__ void half_barrier(int half) {
  asm volatile("bar.sync %0, %1;" ::"r"(1 + half), "r"(256) : "memory");
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T, int W>
__device__ __forceinline__ T group_sum(T v) {
#pragma unroll
  for (int o = W / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Householder QR of the m x n column-major panel A (ld LDA) by one half of
// the CTA: R in the upper trapezoid, reflectors v (v_j = 1 implied) below the
// diagonal, their coefficients in tau. (LAPACK's geqr2 scheme: beta = -sign(x0)|x|.)
template <typename T, int LDA>
__device__ void householder_qr(T *A, int m, int n, T *tau, int half, int ht) {
  const int hw = ht >> 5, lane = ht & 31;
  const int kq = min(m, n);
  for (int j = 0; j < kq; ++j) {
    if (hw == 0) {
      T *col = A + int64_t(j) * LDA;
      T s2 = 0;
      for (int i = j + 1 + lane; i < m; i += 32) s2 += col[i] * col[i];
      s2 = warp_sum(s2);
      const T x0 = col[j];
      if (s2 == T(0)) {
        if (lane == 0) tau[j] = T(0);
      } else {
        const T mu = Num<T>::sqrt_(x0 * x0 + s2);
        const T beta = x0 <= T(0) ? mu : -mu;
        const T scale = T(1) / (x0 - beta);
        for (int i = j + 1 + lane; i < m; i += 32) col[i] *= scale;
        if (lane == 0) { tau[j] = (beta - x0) / beta; col[j] = beta; }
      }
    }
    half_barrier(half);
    const T tj = tau[j];
    if (tj != T(0)) {
      const T *v = A + int64_t(j) * LDA;
      for (int k = j + 1 + hw; k < n; k += 8) {
        T *ck = A + int64_t(k) * LDA;
        T w = lane == 0 ? ck[j] : T(0);
        for (int i = j + 1 + lane; i < m; i += 32) w += v[i] * ck[i];
        w = warp_sum(w) * tj;
        if (lane == 0) ck[j] -= w;
        for (int i = j + 1 + lane; i < m; i += 32) ck[i] -= w * v[i];
      }
    }
    half_barrier(half);
  }
}

// Explicit Q (m x kq, column-major, ld LDA) from the reflectors left in A.
template <typename T, int LDA>
__device__ void form_q(const T *A, const T *tau, T *Q, int m, int kq, int half, int ht) {
  const int hw = ht >> 5, lane = ht & 31;
  for (int idx = ht; idx < m * kq; idx += 256) {
    const int i = idx % m, l = idx / m;
    Q[int64_t(l) * LDA + i] = (i == l) ? T(1) : T(0);
  }
  half_barrier(half);
  for (int j = kq - 1; j >= 0; --j) {
    const T tj = tau[j];
    if (tj != T(0)) {
      const T *v = A + int64_t(j) * LDA;
      for (int l = j + hw; l < kq; l += 8) {
        T *ql = Q + int64_t(l) * LDA;
        T w = lane == 0 ? ql[j] : T(0);
        for (int i = j + 1 + lane; i < m; i += 32) w += v[i] * ql[i];
        w = warp_sum(w) * tj;
        if (lane == 0) ql[j] -= w;
        for (int i = j + 1 + lane; i < m; i += 32) ql[i] -= w * v[i];
      }
    }
    half_barrier(half);
  }
}

// Round-robin (circle method) schedule: in round k, seat s holds player
// 0 (s = 0) or 1 + (s - 1 + k) mod (P - 1); seats p and P-1-p play.
__device__ __forceinline__ int seat_player(int seat, int k, int P) {
  return seat == 0 ? 0 : 1 + (seat - 1 + k) % (P - 1);
}

// One-sided (Hestenes) Jacobi on the rows of the nr x nc row-major matrix B
// (ld ldb) by one half of the CTA: rotate row pairs until all rows are
// mutually orthogonal to within tol. Afterwards row i = s_i v_i^T with s_i
// a singular value and v_i the right singular vector. The rotations are also
// applied to the nu extra columns that follow (an identity block on entry),
// which then hold U^T, so that U S V^T reproduces B to rounding even though
// the rows are only orthogonal to tol. Rotation: for rows a,
// b with alpha = |a|^2, beta = |b|^2, gamma = a.b, zeta = (beta - alpha) / (2 gamma),
// t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)), c = 1 / sqrt(1 + t^2), s = c t:
// a <- c a - s b, b <- s a + c b (Golub & Van Loan, Sec. 8.6.3).
template <typename T, int CH>
__device__ void jacobi_rows(T *B, int nr, int nc, int nu, int ldb, int half, int ht,
                            volatile int *lastrot) {
  constexpr int PAIRS = CH / 2 > 0 ? CH / 2 : 1;
  constexpr int TPP = (256 / PAIRS) < 32 ? (256 / PAIRS) : 32;
  if (nr <= 1) return;  // uniform over the half
  const int P = nr + (nr & 1);
  const int gi = ht / TPP, gl = ht % TPP;
  const T tol = T(2) * Num<T>::eps() * Num<T>::sqrt_(T(nc > 4 ? nc : 4));
  for (int sweep = 0; sweep < JACOBI_MAX_SWEEPS; ++sweep) {
    for (int k = 0; k < P - 1; ++k) {
      int i = -1, j = -1;
      if (gi < P / 2) {
        i = seat_player(gi, k, P);
        j = seat_player(P - 1 - gi, k, P);
        if (i >= nr || j >= nr) i = j = -1;
      }
      T al = 0, be = 0, ga = 0;
      if (i >= 0) {
        const T *a = B + int64_t(i) * ldb, *b = B + int64_t(j) * ldb;
        for (int x = gl; x < nc; x += TPP) {
          const T av = a[x], bv = b[x];
          al += av * av; be += bv * bv; ga += av * bv;
        }
      }
      al = group_sum<T, TPP>(al);
      be = group_sum<T, TPP>(be);
      ga = group_sum<T, TPP>(ga);
      if (i >= 0 && ga != T(0) && fabs(ga) > tol * Num<T>::sqrt_(al * be)) {
        const T zeta = (be - al) / (T(2) * ga);
        const T az = fabs(zeta);
        T t;
        if (az > T(1) / Num<T>::eps()) t = T(0.5) / zeta;
        else t = (zeta >= T(0) ? T(1) : T(-1)) / (az + Num<T>::sqrt_(T(1) + zeta * zeta));
        const T cs = T(1) / Num<T>::sqrt_(T(1) + t * t), sn = cs * t;
        T *a = B + int64_t(i) * ldb, *b = B + int64_t(j) * ldb;
        for (int x = gl; x < nc + nu; x += TPP) {
          const T av = a[x], bv = b[x];
          a[x] = cs * av - sn * bv;
          b[x] = sn * av + cs * bv;
        }
        if (gl == 0) *lastrot = sweep;
      }
      half_barrier(half);
    }
    if (*lastrot < sweep) break;  // no rotation in this sweep (all threads agree)
  }
}

template <typename T>
__device__ __forceinline__ double log_cosh(double x) {
  const double ax = fabs(x);
  return ax + log1p(exp(-2.0 * ax)) - 0.6931471805599453;
}

template <typename T, int CH>
__global__ void __launch_bounds__(ENV_THREADS, 1) env_build_kernel(Layout lay) {
  using P = EnvPlan<T, CH>;
  constexpr int LDA = P::LDA;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double sh_red[ENV_THREADS / 32];
  __shared__ double sh_lam;
  __shared__ int sh_n, sh_kap0, sh_kap1, sh_newE, sh_newO, sh_ntr, sh_dmax;
  __shared__ double sh_dsum;
  __shared__ int sh_lastrot[2];
  __shared__ double sh_gap, sh_disc;

  const int tid = threadIdx.x, half = tid >> 8, ht = tid & 255;
  const int lane = tid & 31, warp = tid >> 5;
  const int chi = lay.chi;
  const double beta = lay.beta;

  unsigned char *slot = (unsigned char *)lay.env_scratch + int64_t(blockIdx.x) * lay.env_slot_bytes;
  T *Qstore = (T *)slot;
  int4 *info = (int4 *)(slot + P::q_bytes(lay.L_max));
  T *W = P::in_smem ? (T *)smem_raw
                    : (T *)(slot + P::q_bytes(lay.L_max) + P::info_bytes(lay.L_max));
  T *Cp = W + P::oCp;
  T *Rb = W + P::oR;
  T *Ab = W + P::oA;
  T *Qf = W + P::oQf;
  T *Qc = W + P::oQc;
  T *Th = W + P::oTh;
  constexpr int LDT = P::LDT;
  T *US = W + P::oUS;
  T *tau = W + P::oTau;
  T *sn = W + P::oSn;
  T *cache = (T *)lay.cache;

  for (;;) {
    if (tid == 0) sh_n = atomicAdd(lay.counter, 1);
    __syncthreads();
    const int idx = sh_n;
    __syncthreads();
    if (idx >= lay.n_real) break;
    const int n = lay.order[idx];
    const RealInfo ri = lay.reals[n];
    const int L = ri.L;
    const float *jr = lay.jr + ri.site_off;
    const float *jd = lay.jd + ri.site_off;
    T *cache_n = cache + ri.site_off * int64_t(chi) * chi;
    int2 *bonds_n = lay.bonds + ri.bond_off;
    if (lay.flags[n] & FLAG_BAD_J) continue;  // uniform: read by all threads after the barrier

    if (tid == 0) sh_lam = 0.0;
    for (int r = L - 1; r >= 0; --r) {
      const bool trivial_prev = (r == L - 1);
      const T *cprev = cache_n + int64_t(r + 1) * L * chi * chi;  // unused when trivial_prev
      const int2 *bprev = bonds_n + int64_t(r + 1) * (L + 1);
      // ---- row constants: sum log cosh(beta Jh) + sum log 2 cosh(beta Jv) (row r < L-1)
      {
        double acc = 0.0;
        for (int c = tid; c < L; c += ENV_THREADS) {
          if (c < L - 1) acc += log_cosh<T>(beta * (double)jr[r * L + c]);
          if (r < L - 1) acc += log_cosh<T>(beta * (double)jd[r * L + c]) + 0.6931471805599453;
        }
        acc = warp_sum(acc);
        if (lane == 0) sh_red[warp] = acc;
        __syncthreads();
        if (tid == 0) {
          double s = 0.0;
          for (int w = 0; w < ENV_THREADS / 32; ++w) s += sh_red[w];
          sh_lam += s;
          sh_kap0 = 1; sh_kap1 = 0;
          sh_gap = 1e300; sh_disc = 0.0; sh_ntr = 0; sh_dmax = 0; sh_dsum = 0.0;
        }
        // R of the (absent) site -1: the 1 x 1 identity of the trivial left bond
        if (tid == 0) Rb[0] = T(1);
        __syncthreads();
      }

      // ================= phase A: MPO application + left-to-right QR sweep
      for (int c = 0; c < L; ++c) {
        const int2 bc = trivial_prev ? make_int2(1, 0) : bprev[c];
        const int2 bn = trivial_prev ? make_int2(1, 0) : bprev[c + 1];
        const int Dc = bc.x + bc.y, Dn = bn.x + bn.y;
        const T tv = (r < L - 1) ? Num<T>::tanh_(T(beta) * T(jd[r * L + c])) : T(0);
        const T th = (c < L - 1) ? Num<T>::tanh_(T(beta) * T(jr[r * L + c])) : T(0);
        // 1. Ct: previous-row site with its odd-parity blocks scaled by t_v
        for (int e = tid; e < Dc * Dn; e += ENV_THREADS) {
          const int a = e / Dn, b = e % Dn;
          T v = trivial_prev ? T(1) : cprev[int64_t(c) * chi * chi + int64_t(a) * chi + b];
          if ((a >= bc.x) != (b >= bn.x)) v *= tv;
          Cp[a * CH + b] = v;
        }
        __syncthreads();
        // 2. Y_q = R_q x (rows of Ct in sector-q order), scattered into the QR panels
        const int k0 = sh_kap0, k1 = sh_kap1, m = k0 + k1;
        for (int e = tid; e < m * Dn; e += ENV_THREADS) {
          const int i = e / Dn, b = e % Dn;
          const int q = (i >= k0) ? 1 : 0;
          const int ip = q ? i - k0 : i;
          const T *Rrow = Rb + q * P::CH2 + int64_t(ip) * CH;
          T acc = 0;
          if (q == 0) {
            for (int a = 0; a < Dc; ++a) acc += Rrow[a] * Cp[a * CH + b];
          } else {
            for (int a2 = 0; a2 < Dc; ++a2) {
              const int a = (a2 < bc.y) ? bc.x + a2 : a2 - bc.y;
              acc += Rrow[a2] * Cp[a * CH + b];
            }
          }
          if (c < L - 1) {
            const int par = (b >= bn.x) ? 1 : 0;
            const int pos0 = par ? b - bn.x : b;
            const int pos1 = par ? b : bn.y + b;
            Ab[par * (LDA * CH) + int64_t(pos0) * LDA + i] = acc;
            Ab[(1 - par) * (LDA * CH) + int64_t(pos1) * LDA + i] = th * acc;
          } else {
            Th[int64_t(i) * LDT] = acc;  // last site: one column (trivial right bond)
          }
        }
        if (tid == 0) info[c] = make_int4(k0, k1, 0, 0);
        __syncthreads();
        if (c == L - 1) break;
        // 3. QR of each parity sector of the new right bond (both are m x Dn)
        T *Aq = Ab + half * (LDA * CH);
        householder_qr<T, LDA>(Aq, m, Dn, tau + half * CH, half, ht);
        __syncthreads();
        const int kq = min(m, Dn);
        // 4. R = upper trapezoid; normalise both sectors together
        {
          double acc = 0.0;
          for (int e = tid; e < 2 * kq * Dn; e += ENV_THREADS) {
            const int q = e / (kq * Dn), rem = e % (kq * Dn), i = rem / Dn, b = rem % Dn;
            if (b >= i) { const double v = (double)Ab[q * (LDA * CH) + int64_t(b) * LDA + i]; acc += v * v; }
          }
          acc = warp_sum(acc);
          if (lane == 0) sh_red[warp] = acc;
          __syncthreads();
          double nrm2 = 0.0;
          for (int w = 0; w < ENV_THREADS / 32; ++w) nrm2 += sh_red[w];
          const double nrm = sqrt(nrm2);
          const bool ok = nrm > 0.0 && isfinite(nrm);
          if (tid == 0) {
            if (ok) sh_lam += log(nrm);
            else set_flag(lay.flags, n, FLAG_NUMERIC);
          }
          const T inv = ok ? T(1.0 / nrm) : T(0);
          for (int e = tid; e < 2 * kq * Dn; e += ENV_THREADS) {
            const int q = e / (kq * Dn), rem = e % (kq * Dn), i = rem / Dn, b = rem % Dn;
            Rb[q * P::CH2 + int64_t(i) * CH + b] =
                (b >= i) ? Ab[q * (LDA * CH) + int64_t(b) * LDA + i] * inv : T(0);
          }
        }
        // 5. explicit Q of each sector
        form_q<T, LDA>(Aq, tau + half * CH, Qf + half * (LDA * CH), m, kq, half, ht);
        __syncthreads();
        // 6. store Q_c = [Q_0 | Q_1] (m x 2kq, column-major) for phase B
        T *qs = Qstore + int64_t(c) * LDA * LDA;
        for (int e = tid; e < 2 * kq * m; e += ENV_THREADS) {
          const int col = e / m, i = e % m;
          const int q = col / kq, l = col % kq;
          qs[int64_t(col) * LDA + i] = Qf[q * (LDA * CH) + int64_t(l) * LDA + i];
        }
        if (tid == 0) { info[c].z = kq; sh_kap0 = kq; sh_kap1 = kq; }
        __syncthreads();
      }

      // ================= phase B: right-to-left truncating SVD sweep
      int curE = 1, curO = 0;  // right bond of the current site, parity-sector dims
      for (int c = L - 1; c >= 0; --c) {
        const int4 inf = info[c];
        const int k0 = inf.x, k1 = inf.y, m = k0 + k1;
        const int N = curE + curO;
        if (c < L - 1) {
          const int kq = inf.z;
          const T *qs = Qstore + int64_t(c) * LDA * LDA;
          for (int e = tid; e < 2 * kq * m; e += ENV_THREADS) {
            const int col = e / m, i = e % m;
            Qc[int64_t(col) * LDA + i] = qs[int64_t(col) * LDA + i];
          }
          __syncthreads();
          // Theta = Q_c x blockdiag(US_0, US_1)
          for (int e = tid; e < m * N; e += ENV_THREADS) {
            const int i = e / N, j = e % N;
            const int q = (j >= curE) ? 1 : 0, jp = q ? j - curE : j;
            const T *Qcol = Qc + int64_t(q * kq) * LDA + i;
            const T *Ucol = US + q * P::CH2 + jp;
            T acc = 0;
            for (int p = 0; p < kq; ++p) acc += Qcol[int64_t(p) * LDA] * Ucol[p * CH];
            Th[int64_t(i) * LDT + j] = acc;
          }
          __syncthreads();
        }
        if (c == 0) {
          // site 0: left bond trivial (m = 1); divide by the norm
          double acc = 0.0;
          for (int j = tid; j < N; j += ENV_THREADS) { const double v = (double)Th[j]; acc += v * v; }
          acc = warp_sum(acc);
          if (lane == 0) sh_red[warp] = acc;
          __syncthreads();
          double nrm2 = 0.0;
          for (int w = 0; w < ENV_THREADS / 32; ++w) nrm2 += sh_red[w];
          const double nrm = sqrt(nrm2);
          const bool ok = nrm > 0.0 && isfinite(nrm);
          const T inv = ok ? T(1.0 / nrm) : T(0);
          T *dst = cache_n + int64_t(r) * L * chi * chi;
          for (int e = tid; e < chi * chi; e += ENV_THREADS) {
            const int a = e / chi, b = e % chi;
            dst[e] = (a == 0 && b < N) ? Th[b] * inv : T(0);
          }
          if (tid == 0) {
            if (ok) sh_lam += log(nrm);
            else set_flag(lay.flags, n, FLAG_NUMERIC);
            bonds_n[int64_t(r) * (L + 1) + 0] = make_int2(1, 0);
            bonds_n[int64_t(r) * (L + 1) + L] = make_int2(1, 0);
            if (L > 1) bonds_n[int64_t(r) * (L + 1) + 1] = make_int2(curE, curO);
            lay.lam[ri.row_off + r] = sh_lam;
            if (lay.dbg_rowinfo) {
              double *ro = lay.dbg_rowinfo + (ri.row_off + r) * 6;
              ro[0] = sh_lam + 0.34657359027997264 * L;  // log ||F_r||: parity form has norm 2^(-L/2)
              ro[1] = sh_gap; ro[2] = sh_disc; ro[3] = sh_ntr;
              ro[4] = sh_dmax; ro[5] = L > 1 ? sh_dsum / (L - 1) : 1.0;
            }
          }
          __syncthreads();
          break;
        }
        // identity block after Theta: the rotations accumulate U^T there
        for (int e = tid; e < m * CH; e += ENV_THREADS) {
          const int i = e / CH, p = e % CH;
          const int base = (i >= k0) ? k0 : 0;
          Th[int64_t(i) * LDT + N + p] = (p == i - base) ? T(1) : T(0);
        }
        if (tid == 0) { sh_lastrot[0] = -1; sh_lastrot[1] = -1; }
        __syncthreads();
        // SVD of each row-parity block (one per half)
        {
          const int rows = half ? k1 : k0;
          T *Bq = Th + int64_t(half ? k0 : 0) * LDT;
          jacobi_rows<T, CH>(Bq, rows, N, rows, LDT, half, ht, &sh_lastrot[half]);
        }
        __syncthreads();
        // singular values = row norms
        for (int i = tid; i < m; i += ENV_THREADS) {
          T s2 = 0;
          for (int j = 0; j < N; ++j) { const T v = Th[int64_t(i) * LDT + j]; s2 += v * v; }
          sn[i] = Num<T>::sqrt_(s2);
        }
        __syncthreads();
        // selection of the chi largest (ties: lower index first); new position in its sector
        T smax = 0;
        for (int i = 0; i < m; ++i) smax = sn[i] > smax ? sn[i] : smax;
        const T thr = smax * T(lay.cutoff);
        __shared__ int sh_keep[2 * 64 * 2];   // per candidate: new index in the bond, or -1
        __shared__ int sh_src[64];            // kept bond index -> candidate row
        for (int i = tid; i < m; i += ENV_THREADS) {
          const T si = sn[i];
          int rank = 0, pos = 0;
          const int qi = (i >= k0) ? 1 : 0;
          for (int j = 0; j < m; ++j) {
            const bool before = (sn[j] > si) || (sn[j] == si && j < i);
            rank += before;
            if (before && ((j >= k0) ? 1 : 0) == qi && sn[j] > thr) pos += 1;  // provisional
          }
          sh_keep[i] = (rank < chi && si > thr) ? (qi << 16) | pos : -1;
        }
        __syncthreads();
        if (tid == 0) {
          int ne = 0, no = 0;
          double kept_min = 1e300, drop_max = 0.0, tot = 0.0, drop = 0.0;
          for (int i = 0; i < m; ++i) {
            const double s = (double)sn[i];
            tot += s * s;
            if (sh_keep[i] >= 0) {
              if (i < k0) ++ne; else ++no;
              kept_min = s < kept_min ? s : kept_min;
            } else {
              drop += s * s;
              drop_max = s > drop_max ? s : drop_max;
            }
          }
          // positions counted above include only candidates above threshold, which are
          // exactly the kept ones ranked before i within its sector (kept set = top-K)
          sh_newE = ne; sh_newO = no;
          sh_dmax = max(sh_dmax, ne + no);
          sh_dsum += ne + no;
          if (drop_max > 0.0) {
            const double gap = kept_min / drop_max - 1.0;
            sh_gap = gap < sh_gap ? gap : sh_gap;
            sh_ntr += 1;
          }
          if (tot > 0.0) { const double d = drop / tot; sh_disc = d > sh_disc ? d : sh_disc; }
          if (smax > T(0) && isfinite((double)smax)) sh_lam += log((double)smax);
          else set_flag(lay.flags, n, FLAG_NUMERIC);
        }
        __syncthreads();
        const int ne = sh_newE, no = sh_newO, nk = ne + no;
        // V^T rows in the new bond order (even kept rows, then odd), into the Qc region
        T *Vt = Qc;
        for (int e = tid; e < m * N; e += ENV_THREADS) {
          const int i = e / N, j = e % N;
          const int kp = sh_keep[i];
          if (kp >= 0) {
            const int q = kp >> 16, pos = kp & 0xffff;
            const int row = q ? ne + pos : pos;
            Vt[int64_t(row) * CH + j] = Th[int64_t(i) * LDT + j] / sn[i];
            if (j == 0) sh_src[row] = i;
          }
        }
        if (lay.dbg_spectra && tid < m && sh_keep[tid] >= 0) {
          int rank = 0;
          for (int j = 0; j < m; ++j) rank += (sn[j] > sn[tid]) || (sn[j] == sn[tid] && j < tid);
          lay.dbg_spectra[(ri.bond_off + int64_t(r) * (L + 1) + c) * chi + rank] =
              (double)sn[tid] / (double)smax;
        }
        __syncthreads();
        // cache row r, site c
        {
          T *dst = cache_n + (int64_t(r) * L + c) * chi * chi;
          for (int e = tid; e < chi * chi; e += ENV_THREADS) {
            const int a = e / chi, b = e % chi;
            dst[e] = (a < nk && b < N) ? Vt[int64_t(a) * CH + b] : T(0);
          }
        }
        // U S from the accumulated rotations, per sector, divided by the largest singular value
        {
          const T inv = smax > T(0) ? T(1) / smax : T(0);
          for (int e = tid; e < (k0 * ne + k1 * no); e += ENV_THREADS) {
            int q, p, k;
            if (e < k0 * ne) { q = 0; p = e / ne; k = e % ne; }
            else { const int e2 = e - k0 * ne; q = 1; p = e2 / no; k = e2 % no; }
            const int i = sh_src[q ? ne + k : k];
            US[q * P::CH2 + int64_t(p) * CH + k] = Th[int64_t(i) * LDT + N + p] * sn[i] * inv;
          }
        }
        if (tid == 0) bonds_n[int64_t(r) * (L + 1) + c + 1] = make_int2(curE, curO);
        curE = ne; curO = no;
        __syncthreads();
      }
    }
  }
}

}  // namespace

template <typename T, int CH>
static int64_t env_slot_bytes_t(int L_max) { return EnvPlan<T, CH>::slot_bytes(L_max); }

int64_t env_slot_bytes(int prec, int CH, int L_max) {
  if (prec == 0) {
    switch (CH) {
      case 8: return env_slot_bytes_t<double, 8>(L_max);
      case 16: return env_slot_bytes_t<double, 16>(L_max);
      case 32: return env_slot_bytes_t<double, 32>(L_max);
      case 64: return env_slot_bytes_t<double, 64>(L_max);
    }
  } else {
    switch (CH) {
      case 8: return env_slot_bytes_t<float, 8>(L_max);
      case 16: return env_slot_bytes_t<float, 16>(L_max);
      case 32: return env_slot_bytes_t<float, 32>(L_max);
      case 64: return env_slot_bytes_t<float, 64>(L_max);
    }
  }
  return -1;
}

template <typename T, int CH>
static cudaError_t launch_env_t(const Layout &lay, cudaStream_t st) {
  using P = EnvPlan<T, CH>;
  const int smem = P::in_smem ? int(P::bytes) : 0;
  cudaError_t e = cudaFuncSetAttribute(env_build_kernel<T, CH>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(lay.counter, 0, sizeof(int32_t), st);
  if (e != cudaSuccess) return e;
  env_build_kernel<T, CH><<<lay.env_slots, ENV_THREADS, smem, st>>>(lay);
  return cudaGetLastError();
}

cudaError_t launch_env_build(const Layout &lay, int prec, int CH, cudaStream_t st) {
  if (prec == 0) {
    switch (CH) {
      case 8: return launch_env_t<double, 8>(lay, st);
      case 16: return launch_env_t<double, 16>(lay, st);
      case 32: return launch_env_t<double, 32>(lay, st);
      case 64: return launch_env_t<double, 64>(lay, st);
    }
  } else {
    switch (CH) {
      case 8: return launch_env_t<float, 8>(lay, st);
      case 16: return launch_env_t<float, 16>(lay, st);
      case 32: return launch_env_t<float, 32>(lay, st);
      case 64: return launch_env_t<float, 64>(lay, st);
    }
  }
  return cudaErrorInvalidValue;
}

}  // namespace tnmc
