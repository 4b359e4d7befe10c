// Boundary-MPS environment build (Sec. 2.2, Sec. 3.2, Fig. 2), one CTA per
// disorder realization, persistent over the batch (Sec. 3.4).
//
// For row r = L-1 .. 0 the kernel applies the row's transfer MPO to the MPS of
// row r+1 (the bond doubles) and compresses it back to chi:
//   phase A  left-to-right Householder QR sweep (left-canonical form);
//   phase B  right-to-left SVD sweep with one-sided Jacobi, keeping the chi
//            largest singular values at every bond; in float64 each Jacobi
//            runs on the triangular factor of a Householder QR of the site
//            matrix (far fewer sweeps).
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
// two halves of the CTA (256 threads each) solve concurrently. The float64
// build of at most (SM count / 2) realizations runs as pairs of CTAs (2-CTA
// clusters): the second CTA of a pair rotates sector 1's Jacobi SVDs on its own
// SM, its rows exchanged through distributed shared memory.
//
// With checkpointed environments (Layout::ckpt_every) a launch builds either all
// rows, keeping every K-th row, or one K-row segment from the checkpoint below
// it (Layout::seg_begin, seg_end); see cache_slot in common.cuh.
#include "common.cuh"
#include "tcmma.cuh"

#include <type_traits>

namespace tnmc {

namespace {

constexpr int ENV_THREADS = 512;
constexpr int JACOBI_MAX_SWEEPS = 30;

template <typename TC, typename TS, int CH>
struct EnvPlan {
  static constexpr int LDA = 2 * CH;                 // rows of the column-major QR panels
  static constexpr int LDT = 2 * CH + 1;             // row stride of Theta | U^T (odd: no bank conflicts between rows)
  static constexpr int64_t CH2 = int64_t(CH) * CH;
  // phase A (units of TC)
  static constexpr int64_t oR = 0;                   // 2 x (CH x CH), row-major (ld CH)
  static constexpr int64_t oA = 2 * CH2;             // 2 x (2CH x CH), column-major (ld 2CH); Q in place
  // phase B (aliases phase A; Theta must not alias R while the last site's GEMM reads R)
  static constexpr int64_t oUS = 0;                  // 2 x (CH x CH), row-major (ld CH)
  static constexpr int64_t oTh = 2 * CH2;            // 2CH x 2CH, row-major (ld LDT)
  static constexpr int64_t oTau = oTh + 2 * CH * LDT;  // 2 x CH
  static constexpr int64_t oSn = oTau + 2 * CH;      // 2CH singular values
  static constexpr int64_t nT = oSn + 2 * CH;
  static constexpr int64_t bytes = nT * int64_t(sizeof(TC));
  static constexpr bool in_smem = bytes <= 220 * 1024;
  static constexpr bool split_carry = sizeof(TC) != sizeof(TS);
  // global scratch per slot: Q of every site, per-site dims, the float64 carry
  // of the previous row when the cache is stored narrower, and the work arena
  // when it does not fit in shared memory
  static __host__ __device__ int64_t q_bytes(int L_max) {
    return align256(int64_t(L_max) * LDA * LDA * sizeof(TC));
  }
  static __host__ __device__ int64_t info_bytes(int L_max) {
    return align256(int64_t(L_max) * sizeof(int4));
  }
  static __host__ __device__ int64_t carry_bytes(int L_max, int chi) {
    return split_carry ? align256(int64_t(2) * L_max * chi * chi * sizeof(TC)) : 0;
  }
  static __host__ __device__ int64_t slot_bytes(int L_max, int chi) {
    return q_bytes(L_max) + info_bytes(L_max) + carry_bytes(L_max, chi) +
           (in_smem ? 0 : align256(bytes));
  }
};

__device__ __forceinline__ void half_barrier(int half) {
  asm volatile("bar.sync %0, %1;" ::"r"(1 + half), "r"(256) : "memory");
}

// ---- two-CTA clusters (float64 build with at most 74 realizations): the
// second CTA of a cluster runs the Jacobi SVD of parity sector 1 on its own
// SM, its rows shipped through distributed shared memory.
__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.aligned;\nbarrier.cluster.wait.aligned;" ::: "memory");
}
// address of the same shared variable in CTA `rank` of this cluster (generic)
template <typename T>
__device__ __forceinline__ T *peer_ptr(T *p, unsigned rank) {
  uint64_t out;
  asm volatile("mapa.u64 %0, %1, %2;" : "=l"(out) : "l"(reinterpret_cast<uint64_t>(p)), "r"(rank));
  return reinterpret_cast<T *>(out);
}
__device__ __forceinline__ void fence_cluster() { asm volatile("fence.acq_rel.cluster;" ::: "memory"); }
__device__ __forceinline__ void store_release_cluster(unsigned *p, unsigned v) {
  asm volatile("st.release.cluster.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned load_acquire_cluster(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.cluster.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
// Wait until *p == want, at most `budget` cycles; false if the wait ran out.
__device__ __forceinline__ bool wait_flag(const unsigned *p, unsigned want, long long budget) {
  const long long t0 = clock64();
  while (load_acquire_cluster(p) != want) {
    if (clock64() - t0 > budget) return false;
    __nanosleep(200);
  }
  return true;
}
constexpr long long CLUSTER_WAIT_CYCLES = 40000000000ll;   // ~20 s at 2 GHz

// Sum over a group of W lanes in double-float: a compensated reduction (each level one
// TwoSum of the leading words, the exact error and the trailing words summed in float32,
// renormalised at the end). Its absolute error ~ u^2 (|x_1| + ... + |x_W|) is the order of
// the accurate double-word additions it replaces, at about half their latency; the inputs
// may be unnormalised dot-product accumulators.
template <int W>
__device__ __forceinline__ dfloat jgroup_sum_df(dfloat v) {
  float h = v.hi, l = v.lo;
#pragma unroll
  for (int o = W / 2; o > 0; o >>= 1) {
    const float oh = __shfl_xor_sync(0xffffffffu, h, o), ol = __shfl_xor_sync(0xffffffffu, l, o);
    float s, e;
    df::two_sum(h, oh, s, e);
    h = s;
    l += ol + e;
  }
  float s, e;
  df::two_sum(h, l, s, e);
  return dfloat(s, e);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
  if constexpr (std::is_same<T, dfloat>::value) {
    return jgroup_sum_df<32>(v);
  } else {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += shfl_xor(v, o);
    return v;
  }
}

// Inner-loop arithmetic, generic over the element type: plain expressions in float32
// and float64, the fused double-float forms of dfloat.cuh for double-float (dot
// products accumulate unnormalised and are finished before use).
template <typename T>
__device__ __forceinline__ void dacc(T &acc, T x, T y) { acc += x * y; }
__device__ __forceinline__ void dacc(dfloat &acc, dfloat x, dfloat y) { df::dot_step(acc, x, y); }
template <typename T>
__device__ __forceinline__ T dfin(T acc) { return acc; }
__device__ __forceinline__ dfloat dfin(dfloat acc) { return df::finish(acc); }
template <typename T>
__device__ __forceinline__ T axmy(T x, T w, T v) { return x - w * v; }      // x - w v
__device__ __forceinline__ dfloat axmy(dfloat x, dfloat w, dfloat v) { return df::axmy(x, w, v); }
template <typename T>
__device__ __forceinline__ void rotate(T &a, T &b, T cs, T sn) {             // (a, b) <- (c a - s b, s a + c b)
  const T av = a, bv = b;
  a = cs * av - sn * bv;
  b = sn * av + cs * bv;
}
__device__ __forceinline__ void rotate(dfloat &a, dfloat &b, dfloat cs, dfloat sn) {
  const dfloat av = a, bv = b;
  a = df::lin2(cs, av, sn, bv);
  b = df::lin2(cs, bv, df::neg(sn), av);
}

// the column-norm comparison of the pivoted QR (float64, or the leading word of a double-float)
__device__ __forceinline__ double pivot_key(double v) { return v; }
__device__ __forceinline__ float pivot_key(float v) { return v; }
__device__ __forceinline__ float pivot_key(dfloat v) { return v.hi; }

template <typename T, int W>
__device__ __forceinline__ T group_sum(T v) {
  if constexpr (std::is_same<T, dfloat>::value) {
    return jgroup_sum_df<W>(v);
  } else {
#pragma unroll
    for (int o = W / 2; o > 0; o >>= 1) v += shfl_xor(v, o);
    return v;
  }
}

// Householder QR of an m x n panel by one half of the CTA, element (i, j) at
// A[i * RS + j * CS]: R in the upper trapezoid, reflectors v (v_j = 1 implied)
// below the diagonal, their coefficients in tau. (LAPACK's geqr2 scheme:
// beta = -sign(x0)|x|.) RS = 1 is a column-major panel, CS = 1 a row-major one.
//
// With PIVOT (the float64 and double-float preconditioning QR) the columns are pivoted
// (Businger & Golub, 1965: at step j the remaining column of largest norm below row j is
// swapped into place; LAPACK's geqp3 order): piv[k] receives the original index of column k and cn
// holds the norms below the current row, recomputed exactly in each update pass (no
// downdating). The triangular factor is then graded, and one-sided Jacobi on its rows
// needs about half the sweeps (Drmac & Veselic, "New fast and accurate Jacobi SVD
// algorithm", SIAM J. Matrix Anal. Appl. 29, 2008).
template <typename T, int RS, int CS, bool PIVOT = false>
__device__ void householder_qr_strided(T *A, int m, int n, T *tau, int half, int ht, T *cn = nullptr,
                                       int *piv = nullptr) {
  const int hw = ht >> 5, lane = ht & 31;
  const int kq = min(m, n);
  if constexpr (PIVOT) {
    static_assert(sizeof(T) == 8 || std::is_same<T, float>::value, "pivoted QR of the Jacobi preconditioner");
    constexpr int G = 8;
    const int grp = ht / G, gl = ht % G;
    for (int k0 = 0; k0 < n; k0 += 256 / G) {           // uniform trip count over the half
      const int k = k0 + grp;
      T s2 = 0;
      if (k < n)
        for (int i = gl; i < m; i += G) dacc(s2, A[int64_t(i) * RS + int64_t(k) * CS], A[int64_t(i) * RS + int64_t(k) * CS]);
      s2 = group_sum<T, G>(dfin(s2));
      if (k < n && gl == 0) { cn[k] = s2; piv[k] = k; }
    }
    half_barrier(half);
  }
  for (int j = 0; j < kq; ++j) {
    if (hw == 0) {
      if constexpr (PIVOT) {
        // the remaining column of largest norm (ties: lower index) swapped into column j
        using K = decltype(pivot_key(T()));
        K best = K(-1);
        int bk = j;
        for (int k = j + lane; k < n; k += 32) {
          const K v = pivot_key(cn[k]);
          if (v > best) { best = v; bk = k; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const K ov = __shfl_xor_sync(0xffffffffu, best, o);
          const int ok = __shfl_xor_sync(0xffffffffu, bk, o);
          if (ov > best || (ov == best && ok < bk)) { best = ov; bk = ok; }
        }
        if (bk != j) {
          for (int i = lane; i < m; i += 32) {
            const T x = A[int64_t(i) * RS + int64_t(j) * CS];
            A[int64_t(i) * RS + int64_t(j) * CS] = A[int64_t(i) * RS + int64_t(bk) * CS];
            A[int64_t(i) * RS + int64_t(bk) * CS] = x;
          }
          if (lane == 0) {
            const T c = cn[j]; cn[j] = cn[bk]; cn[bk] = c;
            const int p = piv[j]; piv[j] = piv[bk]; piv[bk] = p;
          }
        }
        __syncwarp();
      }
      T *col = A + int64_t(j) * CS;
      if constexpr (std::is_same<T, dfloat>::value) {
        // double-float: the column (x0 and below) scaled by a power of two that brings its
        // largest entry near 1, so the squares stay inside float32's range; the reflector
        // and tau do not depend on the scale, and beta is scaled back exactly
        float mx = 0.f;
        for (int i = j + lane; i < m; i += 32) mx = fmaxf(mx, fabsf(col[int64_t(i) * RS].hi));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        const float sc = mx > 0.f ? df::unit_scale(mx) : 1.f;
        T s2 = 0;
        for (int i = j + 1 + lane; i < m; i += 32) {
          const T v = df::scale2(col[int64_t(i) * RS], sc);
          dacc(s2, v, v);
        }
        s2 = warp_sum(dfin(s2));
        const T x0 = df::scale2(col[int64_t(j) * RS], sc);
        if (s2 == T(0)) {
          if (lane == 0) tau[j] = T(0);
        } else {
          const T mu = Num<T>::sqrt_(x0 * x0 + s2);
          const T beta = x0 <= T(0) ? mu : -mu;
          const T scale = T(1) / (x0 - beta);
          for (int i = j + 1 + lane; i < m; i += 32)
            col[int64_t(i) * RS] = df::scale2(col[int64_t(i) * RS], sc) * scale;
          if (lane == 0) { tau[j] = (beta - x0) / beta; col[int64_t(j) * RS] = df::scale2(beta, 1.f / sc); }
        }
      } else {
        T s2 = 0;
        for (int i = j + 1 + lane; i < m; i += 32) dacc(s2, col[int64_t(i) * RS], col[int64_t(i) * RS]);
        s2 = warp_sum(dfin(s2));
        const T x0 = col[int64_t(j) * RS];
        if (s2 == T(0)) {
          if (lane == 0) tau[j] = T(0);
        } else {
          const T mu = Num<T>::sqrt_(x0 * x0 + s2);
          const T beta = x0 <= T(0) ? mu : -mu;
          const T scale = T(1) / (x0 - beta);
          for (int i = j + 1 + lane; i < m; i += 32) col[int64_t(i) * RS] *= scale;
          if (lane == 0) { tau[j] = (beta - x0) / beta; col[int64_t(j) * RS] = beta; }
        }
      }
    }
    half_barrier(half);
    const T tj = tau[j];
    if (tj != T(0) || PIVOT) {   // pivoting refreshes the column norms even for a null reflector
      const T *v = A + int64_t(j) * CS;
      if constexpr (!std::is_same<T, double>::value || PIVOT) {
        // float32, double-float (and pivoting): 8 lanes per column (32 columns at a time),
        // 3-level reductions; at the float32 build's bonds a warp per column leaves most
        // lanes idle and pays 5 shuffle levels per column
        // (the trip count is uniform over the half: every lane reaches the shuffles)
        constexpr int G = 8;
        const int grp = ht / G, gl = ht % G;
        for (int k0 = j + 1; k0 < n; k0 += 256 / G) {
          const int k = k0 + grp;
          const bool on = k < n;
          T *ck = A + int64_t(on ? k : j) * CS;
          T w = (on && gl == 0) ? ck[int64_t(j) * RS] : T(0);
          if (on)
            for (int i = j + 1 + gl; i < m; i += G) dacc(w, v[int64_t(i) * RS], ck[int64_t(i) * RS]);
          w = group_sum<T, G>(dfin(w)) * tj;
          T nn = 0;
          if (on) {
            if (gl == 0) ck[int64_t(j) * RS] -= w;
            for (int i = j + 1 + gl; i < m; i += G) {
              const T x = axmy(ck[int64_t(i) * RS], w, v[int64_t(i) * RS]);
              ck[int64_t(i) * RS] = x;
              if constexpr (PIVOT) dacc(nn, x, x);
            }
          }
          if constexpr (PIVOT) {
            nn = group_sum<T, G>(dfin(nn));
            if (on && gl == 0) cn[k] = nn;
          }
        }
      } else {
        for (int k = j + 1 + hw; k < n; k += 8) {
          T *ck = A + int64_t(k) * CS;
          T w = lane == 0 ? ck[int64_t(j) * RS] : T(0);
          for (int i = j + 1 + lane; i < m; i += 32) dacc(w, v[int64_t(i) * RS], ck[int64_t(i) * RS]);
          w = warp_sum(dfin(w)) * tj;
          if (lane == 0) ck[int64_t(j) * RS] -= w;
          for (int i = j + 1 + lane; i < m; i += 32)
            ck[int64_t(i) * RS] = axmy(ck[int64_t(i) * RS], w, v[int64_t(i) * RS]);
        }
      }
    }
    half_barrier(half);
  }
}

// ---- double-float Householder QR and Q formation with one barrier per step.
// Reflector of column j (entries j.. of col, stride RS) by one warp: the column scaled by
// a power of two for the norm (float32's exponent range), as in householder_qr_strided.
template <int RS>
__device__ __forceinline__ void df_reflector(dfloat *col, int j, int m, dfloat *tau, int lane) {
  float mx = 0.f;
  for (int i = j + lane; i < m; i += 32) mx = fmaxf(mx, fabsf(col[int64_t(i) * RS].hi));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  const float sc = mx > 0.f ? df::unit_scale(mx) : 1.f;
  dfloat s2 = 0;
  for (int i = j + 1 + lane; i < m; i += 32) {
    const dfloat v = df::scale2(col[int64_t(i) * RS], sc);
    dacc(s2, v, v);
  }
  s2 = warp_sum(dfin(s2));
  const dfloat x0 = df::scale2(col[int64_t(j) * RS], sc);
  if (s2 == dfloat(0)) {
    if (lane == 0) tau[j] = dfloat(0);
  } else {
    const dfloat mu = Num<dfloat>::sqrt_(x0 * x0 + s2);
    const dfloat beta = x0 <= dfloat(0) ? mu : -mu;
    const dfloat scale = dfloat(1) / (x0 - beta);
    for (int i = j + 1 + lane; i < m; i += 32) col[int64_t(i) * RS] = df::scale2(col[int64_t(i) * RS], sc) * scale;
    if (lane == 0) { tau[j] = (beta - x0) / beta; col[int64_t(j) * RS] = df::scale2(beta, 1.f / sc); }
  }
}

// Householder QR (unpivoted) of the m x n panel A[i * RS + j * CS] by one half of the
// CTA with look-ahead: in step j the first warp applies reflector j to column j + 1 and
// at once computes reflector j + 1, while the other seven warps (8 lanes per column)
// apply reflector j to columns j + 2 ..; one barrier per step. Same results as the
// two-barrier form up to the order of the column-j+1 reductions.
template <int RS, int CS>
__device__ void householder_qr_la(dfloat *A, int m, int n, dfloat *tau, int half, int ht) {
  const int hw = ht >> 5, lane = ht & 31;
  const int kq = min(m, n);
  if (kq <= 0) return;   // uniform over the half
  if (hw == 0) df_reflector<RS>(A, 0, m, tau, lane);
  half_barrier(half);
  constexpr int G = 8;
  const int grp = (ht - 32) / G, gl = (ht - 32) % G;   // warps 1..7: 28 lane groups
  for (int j = 0; j < kq; ++j) {
    const dfloat tj = tau[j];
    const dfloat *v = A + int64_t(j) * CS;
    if (hw == 0) {
      if (j + 1 < n) {
        dfloat *c1 = A + int64_t(j + 1) * CS;
        if (tj != dfloat(0)) {
          dfloat w = lane == 0 ? c1[int64_t(j) * RS] : dfloat(0);
          for (int i = j + 1 + lane; i < m; i += 32) dacc(w, v[int64_t(i) * RS], c1[int64_t(i) * RS]);
          w = warp_sum(dfin(w)) * tj;
          if (lane == 0) c1[int64_t(j) * RS] -= w;
          for (int i = j + 1 + lane; i < m; i += 32)
            c1[int64_t(i) * RS] = axmy(c1[int64_t(i) * RS], w, v[int64_t(i) * RS]);
        }
        __syncwarp();
        if (j + 1 < kq) df_reflector<RS>(c1, j + 1, m, tau, lane);
      }
    } else if (tj != dfloat(0)) {
      for (int k0 = j + 2; k0 < n; k0 += 28) {   // uniform trip count over warps 1..7
        const int k = k0 + grp;
        const bool on = k < n;
        dfloat *ck = A + int64_t(on ? k : j) * CS;
        dfloat w = (on && gl == 0) ? ck[int64_t(j) * RS] : dfloat(0);
        if (on)
          for (int i = j + 1 + gl; i < m; i += G) dacc(w, v[int64_t(i) * RS], ck[int64_t(i) * RS]);
        w = group_sum<dfloat, G>(dfin(w)) * tj;
        if (on) {
          if (gl == 0) ck[int64_t(j) * RS] -= w;
          for (int i = j + 1 + gl; i < m; i += G)
            ck[int64_t(i) * RS] = axmy(ck[int64_t(i) * RS], w, v[int64_t(i) * RS]);
        }
      }
    }
    half_barrier(half);
  }
}

// Explicit Q from the reflectors (as form_q_inplace) with one barrier per step: column
// j + 1 becomes H_{j+1} e_{j+1} at the start of step j, by the lane group that then
// applies reflector j to it (the last step's update of it has passed the barrier).
template <int LDA>
__device__ void form_q_la(dfloat *A, const dfloat *tau, int m, int kq, int half, int ht) {
  constexpr int G = 8;
  const int grp = ht / G, gl = ht % G;
  for (int j = kq - 1; j >= 0; --j) {
    if (grp == 0 && j + 1 < kq) {
      const dfloat t1 = tau[j + 1];
      dfloat *q1 = A + int64_t(j + 1) * LDA;
      for (int i = gl; i < m; i += G) {
        if (i < j + 1) q1[i] = dfloat(0);
        else if (i == j + 1) q1[i] = dfloat(1) - t1;
        else q1[i] = -(t1 * q1[i]);
      }
    }
    if (ht < 32) __syncwarp();   // the finalised column is read by other lanes of group 0
    const dfloat tj = tau[j];
    if (tj != dfloat(0)) {
      const dfloat *v = A + int64_t(j) * LDA;
      for (int l0 = j + 1; l0 < kq; l0 += 256 / G) {   // uniform trip count over the half
        const int l = l0 + grp;
        const bool on = l < kq;
        dfloat *ql = A + int64_t(on ? l : j) * LDA;
        dfloat w = (on && gl == 0) ? ql[j] : dfloat(0);
        if (on)
          for (int i = j + 1 + gl; i < m; i += G) dacc(w, v[i], ql[i]);
        w = group_sum<dfloat, G>(dfin(w)) * tj;
        if (on) {
          if (gl == 0) ql[j] -= w;
          for (int i = j + 1 + gl; i < m; i += G) ql[i] = axmy(ql[i], w, v[i]);
        }
      }
    }
    half_barrier(half);
  }
  if (kq > 0 && grp == 0) {   // column 0
    const dfloat t0 = tau[0];
    for (int i = gl; i < m; i += G) {
      if (i == 0) A[0] = dfloat(1) - t0;
      else A[i] = -(t0 * A[i]);
    }
  }
  half_barrier(half);
}

// The column-major panel (ld LDA) of the left-to-right sweep.
template <typename T, int LDA>
__device__ __forceinline__ void householder_qr(T *A, int m, int n, T *tau, int half, int ht) {
  if constexpr (std::is_same<T, dfloat>::value) householder_qr_la<1, LDA>(A, m, n, tau, half, ht);
  else householder_qr_strided<T, 1, LDA>(A, m, n, tau, half, ht);
}

// Explicit Q (m x kq, column-major, ld LDA) formed in place of the reflectors
// left in A (LAPACK's org2r order: last reflector first; column j becomes
// H_j e_j once the columns to its right are final).
template <typename T, int LDA>
__device__ void form_q_2b(T *A, const T *tau, int m, int kq, int half, int ht) {
  const int hw = ht >> 5, lane = ht & 31;
  for (int j = kq - 1; j >= 0; --j) {
    const T tj = tau[j];
    if constexpr (std::is_same<T, float>::value) {
      if (tj != T(0)) {
      // float32: 8 lanes per column, 32 columns at a time (uniform trip count over the half)
      constexpr int G = 8;
      const int grp = ht / G, gl = ht % G;
      const T *v = A + int64_t(j) * LDA;
      for (int l0 = j + 1; l0 < kq; l0 += 256 / G) {
        const int l = l0 + grp;
        const bool on = l < kq;
        T *ql = A + int64_t(on ? l : j) * LDA;
        T w = (on && gl == 0) ? ql[j] : T(0);
        if (on)
          for (int i = j + 1 + gl; i < m; i += G) dacc(w, v[i], ql[i]);
        w = group_sum<T, G>(dfin(w)) * tj;
        if (on) {
          if (gl == 0) ql[j] -= w;
          for (int i = j + 1 + gl; i < m; i += G) ql[i] = axmy(ql[i], w, v[i]);
        }
      }
      }
    } else if (tj != T(0)) {
      const T *v = A + int64_t(j) * LDA;
      for (int l = j + 1 + hw; l < kq; l += 8) {
        T *ql = A + int64_t(l) * LDA;
        T w = lane == 0 ? ql[j] : T(0);
        for (int i = j + 1 + lane; i < m; i += 32) dacc(w, v[i], ql[i]);
        w = warp_sum(dfin(w)) * tj;
        if (lane == 0) ql[j] -= w;
        for (int i = j + 1 + lane; i < m; i += 32) ql[i] = axmy(ql[i], w, v[i]);
      }
    }
    half_barrier(half);
    if (hw == 0) {
      T *qj = A + int64_t(j) * LDA;
      for (int i = lane; i < m; i += 32) {
        if (i < j) qj[i] = T(0);
        else if (i == j) qj[i] = T(1) - tj;
        else qj[i] *= -tj;
      }
    }
    half_barrier(half);
  }
}

template <typename T, int LDA>
__device__ __forceinline__ void form_q_inplace(T *A, const T *tau, int m, int kq, int half, int ht) {
  if constexpr (std::is_same<T, dfloat>::value) form_q_la<LDA>(A, tau, m, kq, half, ht);
  else form_q_2b<T, LDA>(A, tau, m, kq, half, ht);
}


// Jacobi convergence test gamma^2 > tol^2 alpha beta. In double-float the products are
// fourth powers of the singular values, which underflow float32's range below ~1e-10 of
// the largest; the equivalent (gamma / alpha) (gamma / beta) > tol^2 stays in range.
template <typename T>
__device__ __forceinline__ bool not_converged(T ga, T al, T be, T tol2) { return ga * ga > tol2 * (al * be); }
__device__ __forceinline__ bool not_converged(dfloat ga, dfloat al, dfloat be, dfloat tol2) {
  if (!(al.hi > 0.f) || !(be.hi > 0.f)) return false;
  return __fdividef(ga.hi, al.hi) * __fdividef(ga.hi, be.hi) > tol2.hi;
}

// Jacobi rotation (c, s, t = s / c) that orthogonalises two rows with squared
// norms alpha, beta and inner product gamma. The angle only needs about float32
// accuracy (an inexact angle leaves a small residual for the next sweep); what
// must hold to working precision is c^2 + s^2 = 1, or the rotation would not
// be orthogonal. For float64, zeta and t come from float32 arithmetic after an
// exact power-of-two rescale, and the pair (c0, s0) is rescaled by the series
// 1 / sqrt(n) = 1 - d/2 + 3 d^2 / 8 (d = n - 1, small), which leaves
// c^2 + s^2 - 1 at rounding level. This keeps the float64 square roots and
// divisions (each a long sequence on the float64 pipe) off the critical path of
// every Jacobi round.
template <typename T>
__device__ __forceinline__ void rotation_params(T al, T be, T ga, T &cs, T &sn, T &t);
template <>
__device__ __forceinline__ void rotation_params<float>(float al, float be, float ga, float &cs,
                                                       float &sn, float &t) {
  const float num = be - al;
  const float zeta = __fdividef(num, 2.f * ga);
  const float az = fabsf(zeta);
  float tf;
  if (az > 1e15f) {
    tf = __fdividef(0.5f, zeta);
  } else {
    const float q = fmaf(zeta, zeta, 1.f);
    tf = copysignf(__fdividef(1.f, az + q * rsqrtf(q)), zeta);
  }
  if (num == 0.f) tf = 1.f;
  cs = rsqrtf(fmaf(tf, tf, 1.f));
  sn = cs * tf;
  t = tf;
}

template <>
__device__ __forceinline__ void rotation_params<double>(double al, double be, double ga, double &cs,
                                                        double &sn, double &t) {
  // zeta = num / den in float32: both are brought into float range by the
  // exponent of the larger one, read from its bit pattern (a power-of-two
  // scaling is exact); float64 arithmetic is left only for that scaling and
  // the orthogonality rescale below
  const double num = be - al, den = 2.0 * ga;
  const double big = fmax(fabs(num), fabs(den));
  int e = ((__double2hiint(big) >> 20) & 0x7ff) - 1023;
  e = max(min(e, 1022), -1022);
  const double sc = __hiloint2double((1023 - e) << 20, 0);   // 2^-e
  const float fn = (float)(num * sc), fd = (float)(den * sc);
  const float zeta = __fdividef(fn, fd);
  const float az = fabsf(zeta);
  float tf;
  if (az > 1e15f) {
    tf = __fdividef(0.5f, zeta);
  } else {
    const float q = fmaf(zeta, zeta, 1.f);
    tf = copysignf(__fdividef(1.f, az + q * rsqrtf(q)), zeta);
  }
  if (fn == 0.f) tf = 1.f;
  const float c0f = rsqrtf(fmaf(tf, tf, 1.f));
  const double c0 = c0f, s0 = (double)(c0f * tf);
  // c^2 + s^2 = 1 to working precision: rescale by 1/sqrt(1+d) ~ 1 - d/2 + 3d^2/8
  // (|d| ~ 1e-7 from the float32 pair; the series' remainder 5|d|^3/16 < 1e-20)
  const double d = fma(c0, c0, fma(s0, s0, -1.0));
  const double r = fma(d, fma(0.375, d, -0.5), 1.0);
  cs = c0 * r;
  sn = s0 * r;
  t = tf;
}

// Double-float rows: the angle in float32 from the leading words (double-float has
// float32's exponent range, so no rescale is needed), then c = c0 (1 - d/2 + 3 d^2 / 8)
// with d = c0^2 (1 + t^2) - 1 evaluated in double-float (|d| ~ 1e-7), so that
// c^2 (1 + t^2) = 1 to double-float precision; s = c t.
template <>
__device__ __forceinline__ void rotation_params<dfloat>(dfloat al, dfloat be, dfloat ga, dfloat &cs,
                                                        dfloat &sn, dfloat &t) {
  const float num = (be - al).hi, den = 2.f * ga.hi;
  const float zeta = __fdividef(num, den);
  const float az = fabsf(zeta);
  float tf;
  if (az > 1e15f) {
    tf = __fdividef(0.5f, zeta);
  } else {
    const float q = fmaf(zeta, zeta, 1.f);
    tf = copysignf(__fdividef(1.f, az + q * rsqrtf(q)), zeta);
  }
  if (num == 0.f) tf = 1.f;
  const float c0 = rsqrtf(fmaf(tf, tf, 1.f));
  // d = c0^2 (1 + t^2) - 1 (|d| ~ 1e-7) from the exact products c0^2 = p + e and
  // t^2 = tp + te: p (1 + tp) - 1 in one rounding (an FMA; p - 1 is exact), then the
  // small terms e (1 + tp) + p te in float32: absolute error ~1e-15
  float p, e, tp, te;
  df::two_prod(c0, c0, p, e);
  df::two_prod(tf, tf, tp, te);
  const float d = fmaf(p, tp, p - 1.f) + fmaf(e, 1.f + tp, p * te);
  const float corr = d * fmaf(0.375f, d, -0.5f);
  // c = c0 + c0 corr with the product exact, s = c t
  float ph, pl, ch, cl;
  df::two_prod(c0, corr, ph, pl);
  df::fast_two_sum(c0, ph, ch, cl);
  cl += pl;
  cs = dfloat(ch, cl);
  sn = df::mul(cs, tf);
  t = dfloat(tf);
}

// Float64 rows: the tangent t is the float32 value of the angle formula
// (zeta = (beta - alpha) / (2 gamma) taken in float32 after both operands are
// brought into float range by the exponent of the larger one, read from its bit
// pattern; a power-of-two scaling is exact), used exactly as a float64 number.
// c = 1 / sqrt(1 + t^2) starts from the float32 reciprocal square root c0 and is
// corrected by the series 1 / sqrt(1 + d) = 1 - d/2 + 3 d^2 / 8 with
// d = c0^2 (1 + t^2) - 1 (|d| ~ 1e-7; the series' remainder 5|d|^3/16 < 1e-20),
// so that c^2 (1 + t^2) = 1 to working precision. ic = c (1 + t^2) = 1 / c.
__device__ __forceinline__ void rotation_tangent_f64(double al, double be, double ga, double &t,
                                                     double &c, double &ic) {
  const double num = be - al, den = 2.0 * ga;
  const double big = fmax(fabs(num), fabs(den));
  int e = ((__double2hiint(big) >> 20) & 0x7ff) - 1023;
  e = max(min(e, 1022), -1022);
  const double sc = __hiloint2double((1023 - e) << 20, 0);   // 2^-e
  const float fn = (float)(num * sc), fd = (float)(den * sc);
  const float zeta = __fdividef(fn, fd);
  const float az = fabsf(zeta);
  float tf;
  if (az > 1e15f) {
    tf = __fdividef(0.5f, zeta);
  } else {
    const float q = fmaf(zeta, zeta, 1.f);
    tf = copysignf(__fdividef(1.f, az + q * rsqrtf(q)), zeta);
  }
  if (fn == 0.f) tf = 1.f;
  const double c0 = (double)rsqrtf(fmaf(tf, tf, 1.f));
  t = (double)tf;
  const double q = fma(t, t, 1.0);
  const double d = fma(c0 * c0, q, -1.0);
  c = c0 * fma(d, fma(0.375, d, -0.5), 1.0);
  ic = c * q;
}

// One-sided (Hestenes) Jacobi on the rows of the nr x nc row-major matrix B
// (ld ldb) by one half of the CTA: rotate row pairs until all rows are
// mutually orthogonal to within tol. Afterwards row i = s_i v_i^T with s_i
// a singular value and v_i the right singular vector. The rotations are also
// applied to the nu extra columns that follow (an identity block on entry),
// which then hold U^T, so that U S V^T reproduces B to rounding even though
// the rows are only orthogonal to tol. Rotation: for rows a, b with
// alpha = |a|^2, beta = |b|^2, gamma = a.b, zeta = (beta - alpha) / (2 gamma),
// t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)), c = 1 / sqrt(1 + t^2), s = c t:
// a <- c a - s b, b <- s a + c b, and then alpha <- alpha - t gamma,
// beta <- beta + t gamma (Golub & Van Loan, Sec. 8.6.3; de Rijk's cached
// norms, refreshed in the first round of every sweep).
//
// With SCALED (float64 rows) the rotations are scaled ("fast"): row i is held as d_i x B_i, and
// a rotation becomes two multiply-adds per element pair,
//   B_a <- B_a - (t d_b / d_a) B_b,   B_b <- B_b + (t d_a / d_b) B_a,
//   d_a <- c d_a,   d_b <- c d_b,
// instead of four float64 operations. This pays where both parity sectors share
// one SM's float64 pipe (one CTA per realization: 7 % faster at L = 96, chi = 64);
// with a sector per SM (CTA pairs) the rounds are latency-bound and the extra
// per-pair scale arithmetic costs more than the shorter rotations save.
// The transformation of the true rows d x B is exactly the rotation (c, s).
// Each row also keeps e_i = 1 / d_i, updated by 1/c = c (1 + t^2) and then one
// Newton step e <- e (2 - d e), so that d_i e_i = 1 to working precision. At the
// end of every sweep that rotated, each row is multiplied by its scale and the
// scales reset to 1; hence d = e = 1 in the first round of every sweep, and a
// scale never falls below cos(pi/4)^(nr-1) within a sweep.
//
// Only the warps that own a pair this round execute arithmetic: with float64
// on B300 every idle warp's instruction costs the whole SM issue slots.
// NT threads take part: 256 (one half of the CTA, ht = its thread index, synchronised by
// the half's named barrier) or 512 (the whole CTA, ht = threadIdx.x, __syncthreads).
// scl: 2 values per row (d_i, e_i), used with SCALED only.
template <typename T, int TPP, int NT = 256, bool SCALED = false>
__device__ int jacobi_rows(T *B, int nr, int nc, int nu, int ldb, int half, int ht,
                           volatile int *lastrot, T *nrm2, const int *perm, T *scl) {
  static_assert(NT == 256 || NT == 512, "a half or the whole CTA");
  static_assert(NT / TPP >= 32, "one lane group per row pair: up to 32 pairs (64 rows)");
  static_assert(!SCALED || std::is_same<T, double>::value, "scaled rotations are for float64 rows");
  if (nr <= 1) return 0;  // uniform over the half
  const int P = nr + (nr & 1);
  const int npairs = P / 2;
  // the second half's active pairs start on the third scheduler partition, so
  // both halves' float64 work spreads over all four partitions
  const int vt = (NT == 512 || !half) ? ht : ((ht + 192) & 255);
  const int gi = vt / TPP, gl = vt % TPP;
  const bool warp_active = (vt & ~31) < npairs * TPP;
  // The computed cosine of a pair carries a rounding error ~ sqrt(nc) eps, so
  // a tolerance at that floor never converges; 8 sqrt(nc) eps stops at the
  // rounding level. Rotations whose tangent is below eps change nothing.
  // float32 rounds are cheap, so float32 stops at 2 sqrt(nc) eps (more sweeps,
  // rows orthogonal closer to the rounding floor); float64 at 8 sqrt(nc) eps
  const T tf = sizeof(T) == 4 ? T(4) : T(64);
  const T tol2 = tf * Num<T>::eps() * Num<T>::eps() * T(nc > 4 ? nc : 4);
  auto sync = [half]() {
    if (NT == 512) __syncthreads(); else half_barrier(half);
  };
  for (int i = ht; i < nr; i += NT) {
    T s2 = 0;
    for (int x = 0; x < nc; ++x) { const T v = B[int64_t(i) * ldb + x]; dacc(s2, v, v); }
    nrm2[i] = dfin(s2);
    if (SCALED) { scl[2 * i] = T(1); scl[2 * i + 1] = T(1); }
  }
  sync();
  // Rows whose norm is below eps x the largest are rounding noise: rotating
  // them only stirs noise (a rotation with a larger row leaves their norm of
  // the same size, and they never pass any cutoff), so they are left alone.
  // A row is judged noise only on an exact norm (the first round of a sweep
  // measures every row); it then keeps that norm, since nothing rotates it.
  const T kNoise = T(-INFINITY);
  T floor2 = 0;
  if (warp_active) {
    T mx = 0;
    for (int i = 0; i < nr; ++i) mx = nrm2[i] > mx ? nrm2[i] : mx;
    floor2 = sizeof(T) == 8 ? mx * Num<T>::eps() * Num<T>::eps() : T(0);
  }
  sync();
  for (int sweep = 0; sweep < JACOBI_MAX_SWEEPS; ++sweep) {
    // Round-robin (circle method) schedule: in round k, seat s holds player 0
    // (s = 0) or 1 + (s - 1 + k) mod (P - 1), and seats p and P-1-p play. The
    // positions (s - 1 + k) mod (P - 1) of this lane's two seats advance by one
    // every round.
    int pa = gi - 1, pb = P - 2 - gi;
    for (int k = 0; k < P - 1; ++k) {
      if (warp_active) {
        const bool full = (k == 0);
        int i = -1, j = -1, solo = -1;
        if (gi < npairs) {
          i = gi == 0 ? 0 : 1 + pa;
          j = 1 + pb;
          pa = (pa + 1 == P - 1) ? 0 : pa + 1;
          pb = (pb + 1 == P - 1) ? 0 : pb + 1;
          if (i >= nr || j >= nr) {
            // odd row count: this row sits the round out, but its norm is still refreshed
            solo = (full && i < nr) ? perm[i] : ((full && j < nr) ? perm[j] : -1);
            i = j = -1;
          } else {
            i = perm[i];
            j = perm[j];
          }
        }
        // row scales (float64): read by every lane of the pair before the
        // shuffles below, written afterwards by the pair's first lane
        T di = 1, ei = 1, dj = 1, ej = 1;
        if (SCALED && i >= 0) {
          di = scl[2 * i]; ei = scl[2 * i + 1];
          dj = scl[2 * j]; ej = scl[2 * j + 1];
        }
        T al = 0, be = 0, ga = 0;
        if (i >= 0) {
          const T *a = B + int64_t(i) * ldb, *b = B + int64_t(j) * ldb;
          if (full) {
            for (int x = gl; x < nc; x += TPP) {
              const T av = a[x], bv = b[x];
              dacc(al, av, av); dacc(be, bv, bv); dacc(ga, av, bv);
            }
            al = dfin(al); be = dfin(be); ga = dfin(ga);
          } else {
            // two accumulators: halves the dependent multiply-add chain
            T g0 = 0, g1 = 0;
            int x = gl;
            for (; x + TPP < nc; x += 2 * TPP) {
              dacc(g0, a[x], b[x]);
              dacc(g1, a[x + TPP], b[x + TPP]);
            }
            if (x < nc) dacc(g0, a[x], b[x]);
            ga = dfin(g0) + dfin(g1);
          }
        } else if (solo >= 0) {
          const T *a = B + int64_t(solo) * ldb;
          for (int x = gl; x < nc; x += TPP) dacc(al, a[x], a[x]);
          al = dfin(al);
        }
        if constexpr (std::is_same<T, dfloat>::value) ga = jgroup_sum_df<TPP>(ga);
        else ga = group_sum<T, TPP>(ga);
        if (SCALED) ga *= di * dj;   // the true rows' inner product (d = 1 in a full round)
        if (full) {
          if constexpr (std::is_same<T, dfloat>::value) {
            al = jgroup_sum_df<TPP>(al);
            be = jgroup_sum_df<TPP>(be);
          } else {
            al = group_sum<T, TPP>(al);
            be = group_sum<T, TPP>(be);
          }
        } else if (i >= 0) {
          al = nrm2[i];
          be = nrm2[j];
        }
        __syncwarp();
        if (solo >= 0 && gl == 0) nrm2[solo] = al <= floor2 ? kNoise : al;
        bool rot = false;
        T cs = 1, sn = 0, t = 0;
        if (i >= 0) {
          // noise rows carry the sentinel from their exact measurement
          const bool quiet = full ? (al <= floor2 || be <= floor2) : (al == kNoise || be == kNoise);
          // convergence test without a square root: gamma^2 > tol^2 alpha beta
          rot = !quiet && ga != T(0) && not_converged(ga, al, be, tol2);
          if (rot) {
            if constexpr (SCALED) rotation_tangent_f64(al, be, ga, t, cs, sn);   // sn = 1 / c
            else rotation_params<T>(al, be, ga, cs, sn, t);
          }
          rot = rot && fabs(t) > Num<T>::eps();
        }
        if (rot) {
          T *a = B + int64_t(i) * ldb, *b = B + int64_t(j) * ldb;
          if constexpr (SCALED) {
            const T ta = t * dj * ei, tb = t * di * ej;
            for (int x = gl; x < nc + nu; x += TPP) {
              const T av = a[x], bv = b[x];
              a[x] = fma(-ta, bv, av);
              b[x] = fma(tb, av, bv);
            }
          } else {
            for (int x = gl; x < nc + nu; x += TPP) rotate(a[x], b[x], cs, sn);
          }
        }
        if (i >= 0 && gl == 0) {
          if (rot) {
            nrm2[i] = al - t * ga; nrm2[j] = be + t * ga; *lastrot = sweep;
            if (SCALED) {
              const T ndi = di * cs, ndj = dj * cs;
              T nei = ei * sn, nej = ej * sn;
              nei *= fma(-ndi, nei, T(2));
              nej *= fma(-ndj, nej, T(2));
              scl[2 * i] = ndi; scl[2 * i + 1] = nei;
              scl[2 * j] = ndj; scl[2 * j + 1] = nej;
            }
          }
          else if (full) { nrm2[i] = al <= floor2 ? kNoise : al; nrm2[j] = be <= floor2 ? kNoise : be; }
        }
      }
      sync();
    }
    if (SCALED && *lastrot == sweep) {
      // fold the scales into the rows (all threads agree on lastrot)
      for (int i = ht >> 5; i < nr; i += NT / 32) {
        const T d = scl[2 * i];
        if (d != T(1))
          for (int x = ht & 31; x < nc + nu; x += 32) B[int64_t(i) * ldb + x] *= d;
      }
      sync();
      for (int i = ht; i < nr; i += NT) { scl[2 * i] = T(1); scl[2 * i + 1] = T(1); }
      sync();
    }
    if (*lastrot < sweep) return sweep + 1;  // no rotation in this sweep (all threads agree)
  }
  return JACOBI_MAX_SWEEPS;
}

// Kernel layouts of the environment build, chosen at run time (Layout::variant):
//   bits 0-1, Jacobi of a sector in a CTA pair (float64 and double-float):
//     0 = the precision's default (float64: 8 lanes per row pair on half the CTA;
//     double-float: 16 lanes on the whole CTA), 1 = 8 lanes on the whole CTA,
//     2 = 8 lanes on half the CTA;
//   bit 2, one CTA per realization even where CTA pairs fit;
//   bit 3, Jacobi of the one-CTA build (both sectors, one per half): 0 = 4 lanes per
//     row pair, 1 = 8 lanes;
//   bit 4, float32 build (FP32, TF32, BF16) on pairs of CTAs where they fit (float32's
//     default is one CTA per realization); bits 0-1 then choose its Jacobi as above
//     (0 = 16 lanes on the whole CTA);
//   bit 5, float32 build: the Jacobi preconditioned by a pivoted QR, as float64 and
//     double-float always are (fewer sweeps; the float32 Householder Q is orthogonal only to
//     float32 rounding, so the float32 truncation is a little less accurate).
// Every layout computes the same method; they differ in rounding only.
enum : int32_t { VARIANT_PAIR_MASK = 3, VARIANT_ONE_CTA = 4, VARIANT_SINGLE_8 = 8, VARIANT_FP32_PAIRS = 16,
                 VARIANT_FP32_QRPRE = 32 };

template <typename TC>
__device__ __forceinline__ int jacobi_in_pair(int variant, TC *B, int nr, int nc, int nu, int ldb, int tid,
                                              volatile int *lastrot, TC *nrm2, const int *perm, TC *scl) {
  int code = variant & VARIANT_PAIR_MASK;
  if (code == 0) code = std::is_same<TC, double>::value ? 2 : 0;
  if (code == 1) return jacobi_rows<TC, 8, 512>(B, nr, nc, nu, ldb, 0, tid, lastrot, nrm2, perm, scl);
  if (code == 2)
    return tid < 256 ? jacobi_rows<TC, 8>(B, nr, nc, nu, ldb, 0, tid, lastrot, nrm2, perm, scl) : 0;
  return jacobi_rows<TC, 16, 512>(B, nr, nc, nu, ldb, 0, tid, lastrot, nrm2, perm, scl);
}

// Non-negative floating-point values order like their bit patterns.
__device__ __forceinline__ long long order_key(double x) { return __double_as_longlong(x); }
__device__ __forceinline__ long long order_key(float x) { return (long long)__float_as_int(x); }
__device__ __forceinline__ long long order_key(dfloat x) { return order_key(double(x)); }

__device__ __forceinline__ double log_cosh(double x) {
  const double ax = fabs(x);
  return ax + log1p(exp(-2.0 * ax)) - 0.6931471805599453;
}

// TC: arithmetic of the build (and the carry between rows); TS: cache storage.
// ---- the TF32 / BF16 contraction modes of the float32 build: the two dense products of
// a site on the tensor cores (tcmma.cuh), each operand rounded to TF32 or BF16 as it is
// loaded, float32 accumulation. Rows are already normalised by the row's log scale (the
// factors removed from R and U S go into lambda_r), so the products stay in range.
//
// Phase A: Y_q = R_q x Ct (sector q's rows), the same operands, rows and panel writes as
// the CUDA-core loop of the kernel. Tiles of 16 rows x 8 columns, dealt to the warps.
template <int MODE, int CH>
__device__ void mpo_product_tc(const float *Rb, const float *Cp, int chi, int k0, int k1, int2 bc,
                               int2 bn, float tv, float th, bool last, float *Ab, float *Th, int warp,
                               int lane) {
  constexpr int LDA = 2 * CH, LDT = 2 * CH + 1;
  constexpr int64_t CH2 = int64_t(CH) * CH;
  const int Dc = bc.x + bc.y, Dn = bn.x + bn.y;
  const int mt0 = (k0 + 15) >> 4, mt1 = (k1 + 15) >> 4, ntn = (Dn + 7) >> 3;
  const int ntile = (mt0 + mt1) * ntn;
  const int g = lane >> 2, t = lane & 3;
  for (int tile = warp; tile < ntile; tile += ENV_THREADS / 32) {   // uniform over the warp
    const int mtq = tile / ntn, nt = tile - mtq * ntn;
    const int q = mtq >= mt0 ? 1 : 0;
    const int kq = q ? k1 : k0;
    const int i0 = (q ? mtq - mt0 : mtq) * 16;
    const float *Rq = Rb + q * CH2;
    auto A = [&](int i, int a2) { return (i < kq && a2 < Dc) ? Rq[i * CH + a2] : 0.f; };
    auto B = [&](int a2, int b) {
      if (a2 >= Dc || b >= Dn) return 0.f;
      const int a = q == 0 ? a2 : ((a2 < bc.y) ? bc.x + a2 : a2 - bc.y);
      const float v = Cp[int64_t(a) * chi + b];
      return ((a >= bc.x) != (b >= bn.x)) ? v * tv : v;
    };
    float c[4];
    tc_tile<MODE>(c, Dc, i0, nt * 8, lane, A, B);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int il = i0 + g + ((u & 2) ? 8 : 0), b = nt * 8 + 2 * t + (u & 1);
      if (il >= kq || b >= Dn) continue;
      const int i = (q ? k0 : 0) + il;
      if (!last) {
        const int pb = b >= bn.x ? 1 : 0;
        const int pos0 = pb ? b - bn.x : b, pos1 = pb ? b : bn.y + b;
        Ab[pb * (LDA * CH) + int64_t(pos0) * LDA + i] = c[u];
        Ab[(1 - pb) * (LDA * CH) + int64_t(pos1) * LDA + i] = th * c[u];
      } else {
        Th[int64_t(i) * LDT] = c[u];
      }
    }
  }
}

// Phase B: Theta = Q_c x blockdiag(US_0, US_1), Q_c (m x 2 kq, column-major, ld 2 CH)
// from the slot scratch; the column tiles of each sector use that sector's block.
template <int MODE, int CH>
__device__ void theta_product_tc(const float *qs, const float *US, int m, int kq, int curE, int curO,
                                 float *Th, int warp, int lane) {
  constexpr int LDA = 2 * CH, LDT = 2 * CH + 1;
  constexpr int64_t CH2 = int64_t(CH) * CH;
  const int mtn = (m + 15) >> 4, nt0 = (curE + 7) >> 3, nt1 = (curO + 7) >> 3;
  const int ntile = mtn * (nt0 + nt1);
  const int g = lane >> 2, t = lane & 3;
  for (int tile = warp; tile < ntile; tile += ENV_THREADS / 32) {   // uniform over the warp
    const int mt = tile / (nt0 + nt1), ntq = tile - mt * (nt0 + nt1);
    const int q = ntq >= nt0 ? 1 : 0;
    const int Nq = q ? curO : curE;
    const int n0 = (q ? ntq - nt0 : ntq) * 8;
    const float *Qq = qs + int64_t(q * kq) * LDA;
    const float *Uq = US + q * CH2;
    auto A = [&](int i, int p) { return (i < m && p < kq) ? Qq[int64_t(p) * LDA + i] : 0.f; };
    auto B = [&](int p, int jp) { return (p < kq && jp < Nq) ? Uq[p * CH + jp] : 0.f; };
    float c[4];
    tc_tile<MODE>(c, kq, mt * 16, n0, lane, A, B);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = mt * 16 + g + ((u & 2) ? 8 : 0), jp = n0 + 2 * t + (u & 1);
      if (i < m && jp < Nq) Th[int64_t(i) * LDT + (q ? curE : 0) + jp] = c[u];
    }
  }
}

template <typename TC, typename TS, int CH, bool SPLIT>
__global__ void __launch_bounds__(ENV_THREADS, 1) env_build_kernel(Layout lay) {
  using P = EnvPlan<TC, TS, CH>;
  constexpr int LDA = P::LDA, LDT = P::LDT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double sh_red[ENV_THREADS / 32];
  __shared__ double sh_lam, sh_gap, sh_disc, sh_dsum, sh_flops;
  __shared__ int sh_n, sh_kap0, sh_kap1, sh_newE, sh_newO, sh_ntr, sh_dmax, sh_sweeps, sh_svds;
  __shared__ int sh_lastrot[2];
  __shared__ int sh_keep[2 * CH];   // per candidate row: (sector << 16 | position) or -1
  __shared__ int sh_src[2 * CH];    // Jacobi row order, then kept bond index -> candidate row
  // float64 and double-float preconditioning QR with column pivoting: per sector, the column
  // norms and the permutation (piv: position -> original column; ipiv: original column ->
  // position)
  // the pivoted QR that preconditions the Jacobi: always in float64 and double-float, in
  // the float32 build when its layout asks (VARIANT_FP32_QRPRE; uniform over the CTA)
  const bool qrpre = sizeof(TC) == 8 || (lay.variant & VARIANT_FP32_QRPRE);
  __shared__ TC sh_cn[2 * CH];
  __shared__ int sh_piv[2 * CH], sh_ipiv[2 * CH];
  __shared__ long long sh_key[2 * CH];   // ordering keys of the singular values
  __shared__ TC Bnrm[2 * CH];        // squared row norms cached by the Jacobi sweeps
  __shared__ TC sh_scl[4 * CH];      // Jacobi row scales (d, 1/d) of float64 rows, per sector
  __shared__ TC sh_tv, sh_th, sh_smax, sh_rscale;
  __shared__ long long sh_clk[5];    // cycles per phase of the current row (diagnostics)
  // cluster mode: task (rank 1 reads) and result (rank 0 reads) mailboxes
  __shared__ unsigned sh_task_seq, sh_done_seq, sh_sent;
  __shared__ int sh_task[5];         // U^T width, columns, stop, first row of sector 1 in the owner, rows
  __shared__ int sh_done_nsw, sh_helper_dead;
  long long t_mark = 0;

  const int tid = threadIdx.x, half = tid >> 8, ht = tid & 255;
  const int lane = tid & 31, warp = tid >> 5;
  const int chi = lay.chi;
  const int64_t chi2 = int64_t(chi) * chi;
  const double beta = lay.beta;

  const int slot_idx = SPLIT ? int(blockIdx.x >> 1) : int(blockIdx.x);
  unsigned char *slot = (unsigned char *)lay.env_scratch + int64_t(slot_idx) * lay.env_slot_bytes;
  TC *Qstore = (TC *)slot;
  int4 *info = (int4 *)(slot + P::q_bytes(lay.L_max));
  TC *carry = (TC *)(slot + P::q_bytes(lay.L_max) + P::info_bytes(lay.L_max));
  TC *W = P::in_smem ? (TC *)smem_raw
                     : (TC *)(slot + P::q_bytes(lay.L_max) + P::info_bytes(lay.L_max) +
                              P::carry_bytes(lay.L_max, chi));
  TC *Rb = W + P::oR;
  TC *Ab = W + P::oA;
  TC *US = W + P::oUS;
  TC *Th = W + P::oTh;
  TC *tau = W + P::oTau;
  TC *sn = W + P::oSn;

  static_assert(!SPLIT || P::in_smem, "cluster mode keeps Theta in shared memory");
  const long long wait_budget = lay.wait_cycles > 0 ? lay.wait_cycles : CLUSTER_WAIT_CYCLES;
  if (SPLIT) {
    if (tid == 0) { sh_task_seq = 0; sh_done_seq = 0; sh_sent = 0; sh_helper_dead = 0; }
    cluster_sync_all();   // both CTAs are running (and initialised) before any remote access
    if (cluster_rank() == 1) {
      // ---- helper: run sector 1's Jacobi for the other CTA until told to stop
      TC *peer_Th = peer_ptr(Th, 0u);
      __shared__ int sh_go;
      for (unsigned task_no = 1;; ++task_no) {
        if (tid == 0) {
          const bool ok = wait_flag(&sh_task_seq, task_no, wait_budget);
          sh_go = ok && sh_task[2] == 0;
          if (!ok) set_flag(lay.flags, 0, FLAG_TIMEOUT);
        }
        __syncthreads();
        fence_cluster();
        if (!sh_go) break;
        const int nu = sh_task[0], N = sh_task[1], row0 = sh_task[3], rows = sh_task[4];
        if (tid == 0) sh_lastrot[0] = -1;
        const int nsw = jacobi_in_pair<TC>(lay.variant, Th, rows, N, nu, LDT, tid, &sh_lastrot[0], Bnrm,
                                           sh_src, sh_scl);
        __syncthreads();
        // the rotated rows back into the owner's Theta, sector 1 at its row row0
        for (int e = tid; e < rows * (N + nu); e += ENV_THREADS) {
          const int r = e / (N + nu), x = e % (N + nu);
          peer_Th[int64_t(row0 + r) * LDT + x] = Th[int64_t(r) * LDT + x];
        }
        fence_cluster();
        __syncthreads();
        if (tid == 0) {
          *peer_ptr(&sh_done_nsw, 0u) = nsw;
          fence_cluster();
          store_release_cluster(peer_ptr(&sh_done_seq, 0u), task_no);
        }
      }
      cluster_sync_all();
      return;
    }
  }

  for (;;) {
    if (tid == 0) sh_n = atomicAdd(lay.counter, 1);
    __syncthreads();
    const int idx = sh_n;
    __syncthreads();
    if (idx >= lay.n_real) {
      if (SPLIT) {
        if (tid == 0) {
          *peer_ptr(&sh_task[2], 1u) = 1;   // stop
          fence_cluster();
          store_release_cluster(peer_ptr(&sh_task_seq, 1u), sh_sent + 1);
        }
        cluster_sync_all();
      }
      break;
    }
    const int n = lay.order[idx];
    const RealInfo ri = lay.reals[n];
    const int L = ri.L;
    const float *jr = lay.jr + ri.site_off;
    const float *jd = lay.jd + ri.site_off;
    TS *cache_n = (TS *)lay.cache + ri.cache_off * chi2;
    // rows of this launch: all (bottom-up), or one segment [a, b) rebuilt from
    // the checkpoint of row b (from the bottom row when b = L)
    const int K = lay.ckpt_every;
    int r_lo = lay.seg_begin < 0 ? 0 : lay.seg_begin;
    const int r_hi = lay.seg_begin < 0 ? L - 1 : min(lay.seg_end, L) - 1;
    if (lay.tune_rows > 0) r_lo = max(0, L - lay.tune_rows);   // a timing launch: the bottom rows
    if (r_lo > r_hi) continue;   // uniform: this realization has no row in the segment
    int2 *bonds_n = lay.bonds + ri.bond_off;
    if (lay.flags[n] & FLAG_BAD_J) continue;  // uniform: read by all threads after the barrier

    if (tid == 0) sh_lam = (r_hi < L - 1) ? lay.lam[ri.row_off + r_hi + 1] : 0.0;
    if (P::split_carry && K > 0 && lay.seg_begin >= 0 && r_hi < L - 1) {
      // a segment resumes the float64 build from the float64 copy of the checkpoint below it
      const double *src = lay.ckpt64 + (ri.ckpt_off + int64_t((r_hi + 1) / K) * L) * chi2;
      TC *dstc = carry + int64_t((r_hi + 1) & 1) * L * chi2;
      for (int64_t e = tid; e < int64_t(L) * chi2; e += ENV_THREADS) dstc[e] = TC(src[e]);
      __syncthreads();
    }
    for (int r = r_hi; r >= r_lo; --r) {
      const bool trivial_prev = (r == L - 1);
      // the previous row in the build's own precision
      const TC *cprev = P::split_carry ? carry + int64_t((r + 1) & 1) * L * chi2
                                       : (const TC *)(cache_n + cache_slot(r + 1, L, K, lay.seg_begin) * L * chi2);
      TC *ccur = P::split_carry ? carry + int64_t(r & 1) * L * chi2 : nullptr;
      TS *dst_row = cache_n + cache_slot(r, L, K, lay.seg_begin) * L * chi2;
      const int2 *bprev = bonds_n + int64_t(r + 1) * (L + 1);
      // ---- row constants: sum log cosh(beta Jh) + sum log 2 cosh(beta Jv) (row r < L-1)
      {
        double acc = 0.0;
        for (int c = tid; c < L; c += ENV_THREADS) {
          if (c < L - 1) acc += log_cosh(beta * (double)jr[r * L + c]);
          if (r < L - 1) acc += log_cosh(beta * (double)jd[r * L + c]) + 0.6931471805599453;
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
          sh_sweeps = 0; sh_svds = 0; sh_flops = 0.0;
          for (int q = 0; q < 5; ++q) sh_clk[q] = 0;
          Rb[0] = TC(1);  // R of the absent site -1: the 1 x 1 identity of the trivial left bond
        }
        __syncthreads();
      }

      // ================= phase A: MPO application + left-to-right QR sweep
      for (int c = 0; c < L; ++c) {
        const int2 bc = trivial_prev ? make_int2(1, 0) : bprev[c];
        const int2 bn = trivial_prev ? make_int2(1, 0) : bprev[c + 1];
        const int Dc = bc.x + bc.y, Dn = bn.x + bn.y;
        if (tid == 0) {
          sh_tv = (r < L - 1) ? Num<TC>::tanh_(TC(beta) * TC(jd[r * L + c])) : TC(0);
          sh_th = (c < L - 1) ? Num<TC>::tanh_(TC(beta) * TC(jr[r * L + c])) : TC(0);
        }
        __syncthreads();
        const TC tv = sh_tv, th = sh_th;
        const TC *Cp = cprev + int64_t(c) * chi2;
        if (tid == 0) t_mark = clock64();
        // Y_q = R_q x Ct[rows in sector-q order], Ct = previous site with its
        // odd-parity blocks scaled by t_v; scattered into the two QR panels
        const int k0 = sh_kap0, k1 = sh_kap1, m = k0 + k1;
        bool on_tc = false;   // the TF32 / BF16 modes: this product on the tensor cores
        if constexpr (std::is_same<TC, float>::value) {
          if (lay.tc_mode != TCMODE_NONE && !trivial_prev) {
            if (lay.tc_mode == TCMODE_TF32)
              mpo_product_tc<TCMODE_TF32, CH>(Rb, Cp, chi, k0, k1, bc, bn, tv, th, c == L - 1, Ab, Th, warp, lane);
            else
              mpo_product_tc<TCMODE_BF16, CH>(Rb, Cp, chi, k0, k1, bc, bn, tv, th, c == L - 1, Ab, Th, warp, lane);
            on_tc = true;
          }
        }
        for (int e = on_tc ? m * Dn : tid; e < m * Dn; e += ENV_THREADS) {
          const int i = e / Dn, b = e % Dn;
          const int q = (i >= k0) ? 1 : 0;
          const int ip = q ? i - k0 : i;
          const TC *Rrow = Rb + q * P::CH2 + int64_t(ip) * CH;
          const int pb = (b >= bn.x) ? 1 : 0;
          TC acc = 0;
          if (trivial_prev) {
            acc = Rrow[0];
          } else {
            // the previous row's site is read from global memory: loads batched eight at a
            // time ahead of the dependent multiply-adds (same arithmetic, same order)
            auto col_of = [&](int a2) { return q == 0 ? a2 : ((a2 < bc.y) ? bc.x + a2 : a2 - bc.y); };
            int a2 = 0;
            for (; a2 + 8 <= Dc; a2 += 8) {
              TC vb[8];
#pragma unroll
              for (int u = 0; u < 8; ++u) vb[u] = Cp[int64_t(col_of(a2 + u)) * chi + b];
#pragma unroll
              for (int u = 0; u < 8; ++u) {
                TC v = vb[u];
                if (((col_of(a2 + u) >= bc.x) ? 1 : 0) != pb) v *= tv;
                dacc(acc, Rrow[a2 + u], v);
              }
            }
            for (; a2 < Dc; ++a2) {
              const int a = col_of(a2);
              TC v = Cp[int64_t(a) * chi + b];
              if (((a >= bc.x) ? 1 : 0) != pb) v *= tv;
              dacc(acc, Rrow[a2], v);
            }
            acc = dfin(acc);
          }
          if (c < L - 1) {
            const int pos0 = pb ? b - bn.x : b;
            const int pos1 = pb ? b : bn.y + b;
            Ab[pb * (LDA * CH) + int64_t(pos0) * LDA + i] = acc;
            Ab[(1 - pb) * (LDA * CH) + int64_t(pos1) * LDA + i] = th * acc;
          } else {
            Th[int64_t(i) * LDT] = acc;  // last site: one column (trivial right bond)
          }
        }
        if (tid == 0) info[c] = make_int4(k0, k1, 0, 0);
        __syncthreads();
        if (tid == 0) { const long long t1 = clock64(); sh_clk[0] += t1 - t_mark; t_mark = t1; }
        if (c == L - 1) break;
        // QR of each parity sector of the new right bond (both are m x Dn)
        TC *Aq = Ab + half * (LDA * CH);
        householder_qr<TC, LDA>(Aq, m, Dn, tau + half * CH, half, ht);
        __syncthreads();
        const int kq = min(m, Dn);
        if (tid == 0 && lay.dbg_rowinfo) {   // the row records' flop count
          const double mm = m, nn = kq;
          sh_flops += 2.0 * (2.0 * (2.0 * mm * nn * nn - 2.0 * nn * nn * nn / 3.0))  // QR + Q, 2 sectors
                      + 2.0 * mm * Dn * Dc;                                          // MPO x MPS product
        }
        // R = upper trapezoid; both sectors normalised together
        {
          // squared norm: double-float rows sum in double-float, float32 rows in float32 (the
          // norm only picks a scale; log Z adds the log of the float32 scale applied), float64
          // rows in float64. The scalar chain (sum over warps, root, reciprocal, log) runs on
          // one thread: run by all 16 warps it queued 16 copies on the slow float64 pipe
          using TA = typename std::conditional<std::is_same<TC, double>::value, double, TC>::type;
          TA acc = TA(0.0);
          for (int e = tid; e < 2 * kq * Dn; e += ENV_THREADS) {
            const int q = e / (kq * Dn), rem = e % (kq * Dn), i = rem / Dn, b = rem % Dn;
            if (b >= i) { const TA v = TA(Ab[q * (LDA * CH) + int64_t(b) * LDA + i]); acc += v * v; }
          }
          acc = warp_sum(acc);
          if (lane == 0) sh_red[warp] = double(acc);
          __syncthreads();
          if (tid == 0) {
            double nrm2 = 0.0;
            for (int w = 0; w < ENV_THREADS / 32; ++w) nrm2 += sh_red[w];
            const double nrm = sqrt(nrm2);
            const bool ok = nrm > 0.0 && isfinite(nrm);
            const TC sc = ok ? TC(1.0 / nrm) : TC(0);
            if (!ok) set_flag(lay.flags, n, FLAG_NUMERIC);
            else if constexpr (std::is_same<TC, float>::value) sh_lam -= log(double(sc));
            else sh_lam += log(nrm);
            sh_rscale = sc;
          }
          __syncthreads();
          const TC inv = sh_rscale;
          for (int e = tid; e < 2 * kq * Dn; e += ENV_THREADS) {
            const int q = e / (kq * Dn), rem = e % (kq * Dn), i = rem / Dn, b = rem % Dn;
            Rb[q * P::CH2 + int64_t(i) * CH + b] =
                (b >= i) ? Ab[q * (LDA * CH) + int64_t(b) * LDA + i] * inv : TC(0);
          }
        }
        __syncthreads();
        // explicit Q of each sector, in place of its reflectors
        form_q_inplace<TC, LDA>(Aq, tau + half * CH, m, kq, half, ht);
        __syncthreads();
        if (tid == 0) { const long long t1 = clock64(); sh_clk[1] += t1 - t_mark; t_mark = t1; }
        // store Q_c = [Q_0 | Q_1] (m x 2kq, column-major) for phase B
        TC *qs = Qstore + int64_t(c) * LDA * LDA;
        for (int e = tid; e < 2 * kq * m; e += ENV_THREADS) {
          const int col = e / m, i = e % m;
          const int q = col / kq, l = col % kq;
          qs[int64_t(col) * LDA + i] = Ab[q * (LDA * CH) + int64_t(l) * LDA + i];
        }
        if (tid == 0) { info[c].z = kq; sh_kap0 = kq; sh_kap1 = kq; }
        __syncthreads();
        if (tid == 0) { const long long t1 = clock64(); sh_clk[0] += t1 - t_mark; t_mark = t1; }
      }

      // ================= phase B: right-to-left truncating SVD sweep
      int curE = 1, curO = 0;  // right bond of the current site, parity-sector dims
      for (int c = L - 1; c >= 0; --c) {
        const int4 inf = info[c];
        const int k0 = inf.x, k1 = inf.y, m = k0 + k1;
        const int N = curE + curO;
        TS *dst = dst_row + int64_t(c) * chi2;
        TC *cdst = P::split_carry ? ccur + int64_t(c) * chi2 : nullptr;
        if (tid == 0) t_mark = clock64();
        if (c < L - 1) {
          // Theta = Q_c x blockdiag(US_0, US_1); Q_c streamed from the slot scratch
          const int kq = inf.z;
          const TC *qs = Qstore + int64_t(c) * LDA * LDA;
          bool on_tc = false;   // the TF32 / BF16 modes: this product on the tensor cores
          if constexpr (std::is_same<TC, float>::value) {
            if (lay.tc_mode != TCMODE_NONE) {
              if (lay.tc_mode == TCMODE_TF32)
                theta_product_tc<TCMODE_TF32, CH>(qs, US, m, kq, curE, curO, Th, warp, lane);
              else
                theta_product_tc<TCMODE_BF16, CH>(qs, US, m, kq, curE, curO, Th, warp, lane);
              on_tc = true;
            }
          }
          for (int e = on_tc ? m * N : tid; e < m * N; e += ENV_THREADS) {
            const int i = e / N, j = e % N;
            const int q = (j >= curE) ? 1 : 0, jp = q ? j - curE : j;
            const TC *Qcol = qs + int64_t(q * kq) * LDA + i;
            const TC *Ucol = US + q * P::CH2 + jp;
            TC acc = 0;
            int p = 0;
            for (; p + 8 <= kq; p += 8) {   // Q_c from global memory: loads batched ahead
              TC qb[8];
#pragma unroll
              for (int u = 0; u < 8; ++u) qb[u] = Qcol[int64_t(p + u) * LDA];
#pragma unroll
              for (int u = 0; u < 8; ++u) dacc(acc, qb[u], Ucol[(p + u) * CH]);
            }
            for (; p < kq; ++p) dacc(acc, Qcol[int64_t(p) * LDA], Ucol[p * CH]);
            Th[int64_t(i) * LDT + j] = dfin(acc);
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
          const TC inv = ok ? TC(1.0 / nrm) : TC(0);
          for (int e = tid; e < chi2; e += ENV_THREADS) {
            const int a = e / chi, b = e % chi;
            const TC v = (a == 0 && b < N) ? Th[b] * inv : TC(0);
            dst[e] = TS(v);
            if (P::split_carry) cdst[e] = v;
          }
          if (tid == 0) {
            if (ok) sh_lam += log(nrm);
            else set_flag(lay.flags, n, FLAG_NUMERIC);
            bonds_n[int64_t(r) * (L + 1) + 0] = make_int2(1, 0);
            bonds_n[int64_t(r) * (L + 1) + L] = make_int2(1, 0);
            if (L > 1) bonds_n[int64_t(r) * (L + 1) + 1] = make_int2(curE, curO);
            lay.lam[ri.row_off + r] = sh_lam;
            if (lay.dbg_rowinfo) {
              double *ro = lay.dbg_rowinfo + (ri.row_off + r) * 14;
              ro[0] = sh_lam + 0.34657359027997264 * L;  // log ||F_r||: parity form has norm 2^(-L/2)
              ro[1] = sh_gap; ro[2] = sh_disc; ro[3] = sh_ntr;
              ro[4] = sh_dmax; ro[5] = L > 1 ? sh_dsum / (L - 1) : 1.0;
              ro[6] = sh_svds; ro[7] = sh_svds > 0 ? double(sh_sweeps) / sh_svds : 0.0;
              for (int q = 0; q < 5; ++q) ro[8 + q] = double(sh_clk[q]);
              ro[13] = sh_flops;
            }
          }
          __syncthreads();
          break;
        }
        // The rows the sweeps rotate, per parity sector (k_s rows of Theta, N columns).
        // float32: the rows of Theta with an identity block after them, in which the
        // rotations accumulate U^T, so that U S V^T reproduces Theta to rounding.
        // float64, QR-preconditioned: Theta_s = Q_s R_s (Householder, by the sector's half
        // of the CTA), and the sweeps rotate the r_s = min(k_s, N) rows of [R_s | Q_s^T]:
        // the rotated rows are still S V^T and the block ends as J Q_s^T = U^T. One-sided
        // Jacobi on the triangular factor needs far fewer sweeps (8-9 against 18-25 on
        // graded test spectra reaching 1e-12..1e-20, same accuracy). Rows r_s .. k_s - 1
        // (rank <= N) are zero and never kept.
        const int r0 = qrpre ? min(k0, N) : k0, r1 = qrpre ? min(k1, N) : k1;
        if (qrpre) {
          const int ks = half ? k1 : k0, rs = half ? r1 : r0;
          TC *As = Th + int64_t(half ? k0 : 0) * LDT;
          TC *ts = tau + half * CH;
          TC *Qb = US + half * P::CH2;   // free until this site's U S is written
          householder_qr_strided<TC, LDT, 1, true>(As, ks, N, ts, half, ht, sh_cn + half * CH,
                                                   sh_piv + half * CH);
          for (int b = ht; b < N; b += 256) sh_ipiv[half * CH + sh_piv[half * CH + b]] = b;
          // the reflectors to Q's column-major buffer, R's lower part cleared
          for (int e = ht; e < ks * rs; e += 256) {
            const int i = e / rs, j = e % rs;
            TC v = TC(0);
            if (i > j) { v = As[int64_t(i) * LDT + j]; As[int64_t(i) * LDT + j] = TC(0); }
            Qb[int64_t(j) * CH + i] = v;
          }
          half_barrier(half);
          form_q_inplace<TC, CH>(Qb, ts, ks, rs, half, ht);
          for (int e = ht; e < ks * CH; e += 256) {
            const int i = e / CH, p = e % CH;
            As[int64_t(i) * LDT + N + p] = (i < rs && p < ks) ? Qb[int64_t(i) * CH + p] : TC(0);
          }
          __syncthreads();
        } else {
          for (int e = tid; e < m * CH; e += ENV_THREADS) {
            const int i = e / CH, p = e % CH;
            const int base = (i >= k0) ? k0 : 0;
            Th[int64_t(i) * LDT + N + p] = (p == i - base) ? TC(1) : TC(0);
          }
        }
        if (tid == 0) { sh_lastrot[0] = -1; sh_lastrot[1] = -1; }
        // rows in decreasing norm (de Rijk's ordering speeds up the sweeps)
        for (int i = tid; i < m; i += ENV_THREADS) {
          TC s2 = 0;
          for (int j = 0; j < N; ++j) { const TC v = Th[int64_t(i) * LDT + j]; dacc(s2, v, v); }
          sh_key[i] = order_key(dfin(s2));
        }
        __syncthreads();
        for (int i = tid; i < m; i += ENV_THREADS) {
          const int base = (i >= k0) ? k0 : 0, end = (i >= k0) ? m : k0;
          int rank = 0;
          for (int j = base; j < end; ++j)
            rank += (sh_key[j] > sh_key[i]) || (sh_key[j] == sh_key[i] && j < i);
          sh_src[base + rank] = i - base;   // sector-local row at sorted position
        }
        __syncthreads();
        if (tid == 0) { const long long t1 = clock64(); sh_clk[2] += t1 - t_mark; t_mark = t1; }
        if (SPLIT && !sh_helper_dead) {
          // cluster mode: sector 1 (two rows or more) goes to the helper CTA, sector 0 is
          // rotated here (each sector has an SM to itself)
          const bool send = r1 >= 2;
          if (send) {
            TC *hTh = peer_ptr(Th, 1u);
            int *hsrc = peer_ptr(sh_src, 1u);
            for (int e = tid; e < r1 * (N + k1); e += ENV_THREADS) {
              const int r = e / (N + k1), x = e % (N + k1);
              hTh[int64_t(r) * LDT + x] = Th[int64_t(k0 + r) * LDT + x];
            }
            for (int r = tid; r < k1; r += ENV_THREADS) hsrc[r] = sh_src[k0 + r];
            fence_cluster();
            __syncthreads();
            if (tid == 0) {
              int *h_task = peer_ptr(sh_task, 1u);
              h_task[0] = k1;   // width of the U^T block
              h_task[1] = N;
              h_task[2] = 0;
              h_task[3] = k0;   // the row where sector 1 starts here
              h_task[4] = r1;   // rows to rotate
              fence_cluster();
              store_release_cluster(peer_ptr(&sh_task_seq, 1u), ++sh_sent);
            }
          }
          // 8 lanes per row pair on one half (measured: faster than 4 lanes, and than
          // 16 lanes over the whole CTA, whose barrier costs more than its warps gain)
          const int nsw0 = jacobi_in_pair<TC>(lay.variant, Th, r0, N, k0, LDT, tid, &sh_lastrot[0], Bnrm,
                                              sh_src, sh_scl);
          if (tid == 0) {
            if (nsw0 > 0) { sh_sweeps += nsw0; sh_svds += 1; }
            if (send) {
              if (wait_flag(&sh_done_seq, sh_sent, wait_budget)) {
                if (sh_done_nsw > 0) { sh_sweeps += sh_done_nsw; sh_svds += 1; }
              } else {
                set_flag(lay.flags, n, FLAG_TIMEOUT);
                sh_helper_dead = 1;
              }
            }
          }
          __syncthreads();
          if (send && sh_helper_dead) {   // the helper gave up: rotate sector 1 here
            const int nsw1 = jacobi_rows<TC, 16, 512>(Th + int64_t(k0) * LDT, r1, N, k1, LDT, 0, tid,
                                                      &sh_lastrot[1], Bnrm + CH, sh_src + k0,
                                                      sh_scl + 2 * CH);
            if (tid == 0 && nsw1 > 0) { sh_sweeps += nsw1; sh_svds += 1; }
          }
        } else {
          const int rows = half ? k1 : k0;
          TC *Bq = Th + int64_t(half ? k0 : 0) * LDT;
          const int rr = half ? r1 : r0;
          TC *nb = Bnrm + (half ? CH : 0), *sc = sh_scl + (half ? 2 * CH : 0);
          const int *pp = sh_src + (half ? k0 : 0);
          const int nsw = (lay.variant & VARIANT_SINGLE_8)
                              ? jacobi_rows<TC, 8, 256>(Bq, rr, N, rows, LDT, half, ht, &sh_lastrot[half], nb, pp, sc)
                              : jacobi_rows<TC, 4, 256, std::is_same<TC, double>::value>(
                                    Bq, rr, N, rows, LDT, half, ht, &sh_lastrot[half], nb, pp, sc);
          if (ht == 0 && nsw > 0) { atomicAdd(&sh_sweeps, nsw); atomicAdd(&sh_svds, 1); }
        }
        __syncthreads();
        if (SPLIT) fence_cluster();   // the helper's rows, acquired by one thread, for all
        if (tid == 0) { const long long t1 = clock64(); sh_clk[3] += t1 - t_mark; t_mark = t1; }
        // singular values = row norms
        for (int i = tid; i < m; i += ENV_THREADS) {
          TC s2 = 0;
          for (int j = 0; j < N; ++j) { const TC v = Th[int64_t(i) * LDT + j]; dacc(s2, v, v); }
          const TC si = Num<TC>::sqrt_(dfin(s2));
          sn[i] = si;
          sh_key[i] = order_key(si);
        }
        __syncthreads();
        if (warp == 0) {
          long long km = 0;
          for (int i = lane; i < m; i += 32) km = sh_key[i] > km ? sh_key[i] : km;
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            const long long other = __shfl_xor_sync(0xffffffffu, km, o);
            km = other > km ? other : km;
          }
          if (lane == 0) {
            TC smx = 0;
            for (int i = 0; i < m; ++i) if (sh_key[i] == km) { smx = sn[i]; break; }
            sh_smax = smx;
          }
        }
        __syncthreads();
        // keep the chi largest above cutoff x largest (ties: lower index first)
        const TC smax = sh_smax;
        const TC thr = smax * TC(lay.cutoff);
        const long long kthr = order_key(thr);
        for (int i = tid; i < m; i += ENV_THREADS) {
          const long long ki = sh_key[i];
          int rank = 0, pos = 0;
          const int qi = (i >= k0) ? 1 : 0;
          for (int j = 0; j < m; ++j) {
            const long long kj = sh_key[j];
            const bool before = (kj > ki) || (kj == ki && j < i);
            rank += before;
            if (before && ((j >= k0) ? 1 : 0) == qi) pos += 1;
          }
          const TC si = sn[i];
          const bool keep = rank < chi && ki > kthr;
          sh_keep[i] = keep ? (qi << 16) | pos : -1;
          if (keep && lay.dbg_spectra)
            lay.dbg_spectra[(ri.bond_off + int64_t(r) * (L + 1) + c) * chi + rank] =
                (double)si / (double)smax;
        }
        __syncthreads();
        if (warp == 0) {
          // kept counts per sector over warp 0; for the row records also the cut gap and the
          // discarded weight (float64 work kept off the build unless asked for)
          const bool stats = lay.dbg_rowinfo != nullptr;
          int ne = 0, no = 0;
          double kept_min = 1e300, drop_max = 0.0, tot = 0.0, drop = 0.0;
          for (int i = lane; i < m; i += 32) {
            const bool kept = sh_keep[i] >= 0;
            if (kept) { if (i < k0) ++ne; else ++no; }
            if (stats) {
              const double s = (double)sn[i];
              tot += s * s;
              if (kept) {
                kept_min = s < kept_min ? s : kept_min;
              } else {
                drop += s * s;
                drop_max = s > drop_max ? s : drop_max;
              }
            }
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            ne += __shfl_xor_sync(0xffffffffu, ne, o);
            no += __shfl_xor_sync(0xffffffffu, no, o);
          }
          if (stats) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
              tot += __shfl_xor_sync(0xffffffffu, tot, o);
              drop += __shfl_xor_sync(0xffffffffu, drop, o);
              const double km = __shfl_xor_sync(0xffffffffu, kept_min, o);
              const double dm = __shfl_xor_sync(0xffffffffu, drop_max, o);
              kept_min = km < kept_min ? km : kept_min;
              drop_max = dm > drop_max ? dm : drop_max;
            }
          }
          if (lane == 0) {
            sh_newE = ne; sh_newO = no;
            if (stats) {
              sh_dmax = max(sh_dmax, ne + no);
              sh_dsum += ne + no;
              if (drop_max > 0.0) {
                const double gap = kept_min / drop_max - 1.0;
                sh_gap = gap < sh_gap ? gap : sh_gap;
                sh_ntr += 1;
              }
              if (tot > 0.0) { const double d = drop / tot; sh_disc = d > sh_disc ? d : sh_disc; }
            }
          }
        } else if (tid == 32) {   // the log scale of this site, beside warp 0's counts
          if (smax > TC(0) && isfinite((double)smax)) sh_lam += log((double)smax);
          else set_flag(lay.flags, n, FLAG_NUMERIC);
        }
        __syncthreads();
        const int ne = sh_newE, no = sh_newO, nk = ne + no;
        if (tid == ENV_THREADS - 32 && lay.dbg_rowinfo) {   // the row records' flop count, off warp 0
          for (int q = 0; q < 2; ++q) {
            const double rq = q ? k1 : k0;
            const double a = rq > N ? rq : N, b = rq > N ? N : rq;
            if (b > 0) sh_flops += 4.0 * a * a * b + 8.0 * a * b * b + 9.0 * b * b * b;
          }
          if (c < L - 1) sh_flops += 2.0 * m * N * inf.z;
        }
        // a kept candidate's position within its sector counts the kept candidates of that
        // sector ranked before it (the kept set is the top of the ranking, so all of them)
        for (int i = tid; i < m; i += ENV_THREADS) {
          const int kp = sh_keep[i];
          if (kp >= 0) sh_src[(kp >> 16) ? ne + (kp & 0xffff) : (kp & 0xffff)] = i;
          Bnrm[i] = kp >= 0 ? TC(1) / sn[i] : TC(0);   // reciprocal singular values
        }
        __syncthreads();
        // cache row r, site c: V^T rows in the new bond order (even kept rows, then odd)
        for (int e = tid; e < chi2; e += ENV_THREADS) {
          const int a = e / chi, b = e % chi;
          TC v = TC(0);
          if (a < nk && b < N) {
            const int i = sh_src[a];
            // pivoted preconditioning: column b of the site sits at position ipiv[b] of the rows
            const int bb = qrpre ? sh_ipiv[(i >= k0 ? CH : 0) + b] : b;
            v = Th[int64_t(i) * LDT + bb] * Bnrm[i];
          }
          dst[e] = TS(v);
          if (P::split_carry) cdst[e] = v;
        }
        // U S from the accumulated rotations, per sector, divided by the largest singular value
        {
          const TC inv = smax > TC(0) ? TC(1) / smax : TC(0);
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
        if (tid == 0) { const long long t1 = clock64(); sh_clk[4] += t1 - t_mark; t_mark = t1; }
      }
      // MIXED with checkpoints: keep the float64 row of every checkpoint (full build only;
      // the next row reads this buffer and writes the other one)
      if (P::split_carry && K > 0 && lay.seg_begin < 0 && r % K == 0) {
        double *ck = lay.ckpt64 + (ri.ckpt_off + int64_t(r / K) * L) * chi2;
        for (int64_t e = tid; e < int64_t(L) * chi2; e += ENV_THREADS) ck[e] = double(ccur[e]);
      }
    }
  }
}

}  // namespace

// Kernel variants: mode 0 = float64 build and cache; 1 = float32 build and
// cache; 2 = float64 build with a float32 cache (the float64 carry between
// rows stays in the slot scratch); 3 = double-float build and cache.
template <typename TC, typename TS>
static int64_t env_slot_bytes_ts(int CH, int L_max, int chi) {
  switch (CH) {
    case 8: return EnvPlan<TC, TS, 8>::slot_bytes(L_max, chi);
    case 16: return EnvPlan<TC, TS, 16>::slot_bytes(L_max, chi);
    case 32: return EnvPlan<TC, TS, 32>::slot_bytes(L_max, chi);
    case 64: return EnvPlan<TC, TS, 64>::slot_bytes(L_max, chi);
  }
  return -1;
}

int64_t env_slot_bytes(int mode, int CH, int L_max, int chi) {
  if (mode == 0) return env_slot_bytes_ts<double, double>(CH, L_max, chi);
  if (mode == 1) return env_slot_bytes_ts<float, float>(CH, L_max, chi);
  if (mode == 3) return env_slot_bytes_ts<dfloat, dfloat>(CH, L_max, chi);
  return env_slot_bytes_ts<double, float>(CH, L_max, chi);
}

template <typename TC, typename TS, int CH, bool SPLIT>
static cudaError_t launch_env_t(const Layout &lay, cudaStream_t st) {
  using P = EnvPlan<TC, TS, CH>;
  const int smem = P::in_smem ? int(P::bytes) : 0;
  cudaError_t e = cudaFuncSetAttribute(env_build_kernel<TC, TS, CH, SPLIT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(lay.counter, 0, sizeof(int32_t), st);
  if (e != cudaSuccess) return e;
  if (!SPLIT) {
    env_build_kernel<TC, TS, CH, false><<<lay.env_slots, ENV_THREADS, smem, st>>>(lay);
    return cudaGetLastError();
  }
  // pairs of CTAs: the second of each pair serves sector 1's Jacobi SVDs
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(2 * lay.env_slots);
  cfg.blockDim = dim3(ENV_THREADS);
  cfg.dynamicSmemBytes = size_t(smem);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, env_build_kernel<TC, TS, CH, true>, lay);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

template <typename TC, typename TS>
static cudaError_t launch_env_ts(const Layout &lay, int CH, bool split, cudaStream_t st) {
  if (split) {
    switch (CH) {
      case 8: return launch_env_t<TC, TS, 8, true>(lay, st);
      case 16: return launch_env_t<TC, TS, 16, true>(lay, st);
      case 32: return launch_env_t<TC, TS, 32, true>(lay, st);
      case 64: return launch_env_t<TC, TS, 64, true>(lay, st);
    }
    return cudaErrorInvalidValue;
  }
  switch (CH) {
    case 8: return launch_env_t<TC, TS, 8, false>(lay, st);
    case 16: return launch_env_t<TC, TS, 16, false>(lay, st);
    case 32: return launch_env_t<TC, TS, 32, false>(lay, st);
    case 64: return launch_env_t<TC, TS, 64, false>(lay, st);
  }
  return cudaErrorInvalidValue;
}

// The float64 and double-float builds run as CTA pairs (one SM per parity sector's
// Jacobi) when the pairs of all realizations fit on the GPU at once (2 x realizations
// <= SMs; 74 pairs on a 148-SM B300); the float32 build does so when its layout asks.
cudaError_t launch_env_build(const Layout &lay, int mode, int CH, cudaStream_t st) {
  if (mode == 0 || mode == 3 || (mode == 1 && (lay.variant & VARIANT_FP32_PAIRS))) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const bool pairs = 2 * lay.env_slots <= sms && !(lay.variant & VARIANT_ONE_CTA);
    if (mode == 3) return launch_env_ts<dfloat, dfloat>(lay, CH, pairs, st);
    if (mode == 1) return launch_env_ts<float, float>(lay, CH, pairs, st);
    return launch_env_ts<double, double>(lay, CH, pairs, st);
  }
  if (mode == 1) return launch_env_ts<float, float>(lay, CH, false, st);
  return launch_env_ts<double, float>(lay, CH, false, st);
}

}  // namespace tnmc
