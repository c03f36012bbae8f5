// Row-wise WQ assembly by sum factorisation, fused with the CSR value stores.
//
// For a row i = (i1, i2, i3) and a column j in I_i the WQ entries are
// (Eq. (massquadrature), Eq. (sumfactorization), extended to Eq. (stiff) with
// the term (l, m) integrated by the rule of kind (delta_kl, delta_km) in
// direction k):
//
//   s_ij = sum_{l,m} sum_{q3} w3 B3 sum_{q2} w2 B2 sum_{q1} w1 B1 c_lm(q1,q2,q3)
//
// Each block owns a tile of rows (a range of i1, a range of i2, one i3) and runs
// the three mode products of Eq. (sumfactorization) for all its rows at once,
// sharing the intermediate tensors between neighbouring rows (the paper applies
// them row by row, Algorithm 3):
//
//   stage 3:  T3[q1,q2]    = sum_{q3 in Q_i3 n Q_j3} w3(i3,q3) B3(j3,q3) c_lm(q1,q2,q3)
//   stage 2:  H2[q1,i2,q2] = sum_{terms of a class} w2^{(a2,b2)}(i2,q2) T3[q1,q2]
//             G_g[q1,i2,j2] += sum_{q2 in Q_i2 n Q_j2} B2^{(b2)}(j2,q2) H2[q1,i2,q2]
//   stage 1:  h_b[q1]      = sum_{a} w1^{(a,b)}(i1,q1) G_{(a,b)}[q1,i2,j2]
//             s[i1,j1]     = sum_{b} sum_{q1 in Q_i1 n Q_j1} B1^{(b)}(j1,q1) h_b[q1]
//
// The nine terms (l, m) fall into six classes of equal (test, trial) kind in
// directions 1 and trial kind in direction 2, which lets stage 2 contract the
// trial B-splines once per class; stage 1 contracts them once per trial kind.
// Products with a B-spline that vanishes at the point are skipped (the q-sums
// run over the intersection of the two supports). Values go straight to their
// CSR position: row_ptr is closed form in the band prefix sums.
#include <algorithm>

#include "wq_internal.h"

namespace wq {

struct AsmDir {
  int n;
  const int* q0;
  const int* nq;
  const double* w;       // [4][n][NQ]
  const double* bt;      // [2][n][NQ]
  const int64_t* prefix; // [n+1]
};

struct AsmArgs {
  AsmDir d[3];
  int NQ;
  const double* coef;    // [7][N_QP]
  const double* kappa;   // NULL or [N_QP]
  int64_t nqp_total;
  int nqp1, nqp2;
  void* vals;
  int nt1, nt2;          // tiles per direction 1, 2
  int T1M, T2M;          // largest tile extents
  int W1M, W2M;          // largest point windows of a tile
};

// Term (l, m) of Eq. (stiff), ordered by class; class c covers terms
// [kClassStart[c], kClassStart[c+1]).
__constant__ int kTermL[9] = {0, 0, 0, 1, 2, 1, 2, 1, 2};
__constant__ int kTermM[9] = {0, 1, 2, 0, 0, 1, 1, 2, 2};
__constant__ int kClassStart[7] = {0, 1, 2, 3, 5, 7, 9};
__constant__ int kSlot[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};

__device__ __forceinline__ int band_lo(int i, int p) { return i - p > 0 ? i - p : 0; }
__device__ __forceinline__ int band_w(int i, int p, int n) { return min(n - 1, i + p) - band_lo(i, p) + 1; }

template <typename T>
__device__ __forceinline__ T fmaT(T a, T b, T c);
template <>
__device__ __forceinline__ double fmaT<double>(double a, double b, double c) { return fma(a, b, c); }
template <>
__device__ __forceinline__ float fmaT<float>(float a, float b, float c) { return fmaf(a, b, c); }

struct SmemLayout {
  int w1, b1, w2, b2, a3, t3, h2, g, ints, total_real;  // offsets in Real elements, ints in int32
};

template <int P, bool MASS>
__host__ __device__ inline SmemLayout smem_layout(int NQ, int T1M, int T2M, int W1M, int W2M) {
  constexpr int NK = MASS ? 1 : 4, NB = MASS ? 1 : 2, NG = MASS ? 1 : 4, BW = 2 * P + 1;
  const int J1M = T1M + 2 * P, J2M = T2M + 2 * P;
  SmemLayout L;
  int o = 0;
  L.w1 = o; o += NK * T1M * NQ;
  L.b1 = o; o += NB * J1M * NQ;
  L.w2 = o; o += NK * T2M * NQ;
  L.b2 = o; o += NB * J2M * NQ;
  L.a3 = o; o += NK * NQ;
  L.t3 = o; o += W1M * W2M;
  L.h2 = o; o += T2M * NQ * W1M;
  L.g = o;  o += NG * T2M * BW * W1M;
  L.total_real = o;
  L.ints = 2 * (J1M + J2M);
  return L;
}

template <int P, bool MASS, typename Real, typename OutT>
__global__ void __launch_bounds__(256) k_assemble(AsmArgs A) {
  constexpr int BW = 2 * P + 1;
  constexpr int NK = MASS ? 1 : 4;   // weight kinds held per direction
  constexpr int NB = MASS ? 1 : 2;   // trial derivative orders
  constexpr int NG = MASS ? 1 : 4;   // stage-1 groups (a1, b1)
  constexpr int NCLASS = MASS ? 1 : 6;
  constexpr int MAXQ = 4 * P + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* sm = reinterpret_cast<Real*>(smem_raw);
  const int NQ = A.NQ;
  const SmemLayout L = smem_layout<P, MASS>(NQ, A.T1M, A.T2M, A.W1M, A.W2M);
  int* si = reinterpret_cast<int*>(sm + L.total_real);

  const int n1 = A.d[0].n, n2 = A.d[1].n, n3 = A.d[2].n;
  int bid = blockIdx.x;
  const int tile1 = bid % A.nt1;
  bid /= A.nt1;
  const int tile2 = bid % A.nt2;
  const int i3 = bid / A.nt2;
  const int i1a = (int)((int64_t)tile1 * n1 / A.nt1), i1b = (int)((int64_t)(tile1 + 1) * n1 / A.nt1);
  const int i2a = (int)((int64_t)tile2 * n2 / A.nt2), i2b = (int)((int64_t)(tile2 + 1) * n2 / A.nt2);
  const int T1 = i1b - i1a, T2 = i2b - i2a;
  const int j1a = band_lo(i1a, P), j1b = min(n1 - 1, i1b - 1 + P), J1 = j1b - j1a + 1;
  const int j2a = band_lo(i2a, P), j2b = min(n2 - 1, i2b - 1 + P), J2 = j2b - j2a + 1;
  const int J1M = A.T1M + 2 * P;
  int* q0j1 = si;
  int* nqj1 = si + J1M;
  int* q0j2 = si + 2 * J1M;
  int* nqj2 = q0j2 + (A.T2M + 2 * P);
  const int tid = threadIdx.x, nth = blockDim.x;

  // per-tile univariate tables into shared memory
  for (int e = tid; e < J1; e += nth) {
    q0j1[e] = A.d[0].q0[j1a + e];
    nqj1[e] = A.d[0].nq[j1a + e];
  }
  for (int e = tid; e < J2; e += nth) {
    q0j2[e] = A.d[1].q0[j2a + e];
    nqj2[e] = A.d[1].nq[j2a + e];
  }
  Real* w1s = sm + L.w1;  // [NK][T1M][NQ]
  Real* b1s = sm + L.b1;  // [NB][J1M][NQ]
  Real* w2s = sm + L.w2;  // [NK][T2M][NQ]
  Real* b2s = sm + L.b2;  // [NB][J2M][NQ]
  Real* a3s = sm + L.a3;  // [NK][NQ]
  Real* t3s = sm + L.t3;  // [W2][W1]
  Real* h2s = sm + L.h2;  // [T2][NQ][W1]
  Real* gs = sm + L.g;    // [NG][T2][BW][W1]
  for (int e = tid; e < NK * T1 * NQ; e += nth) {
    int t = e % NQ, r = e / NQ, il = r % T1, k = r / T1;
    w1s[(k * A.T1M + il) * NQ + t] = (Real)A.d[0].w[((size_t)k * n1 + i1a + il) * NQ + t];
  }
  for (int e = tid; e < NB * J1 * NQ; e += nth) {
    int t = e % NQ, r = e / NQ, jl = r % J1, b = r / J1;
    b1s[(b * J1M + jl) * NQ + t] = (Real)A.d[0].bt[((size_t)b * n1 + j1a + jl) * NQ + t];
  }
  for (int e = tid; e < NK * T2 * NQ; e += nth) {
    int t = e % NQ, r = e / NQ, il = r % T2, k = r / T2;
    w2s[(k * A.T2M + il) * NQ + t] = (Real)A.d[1].w[((size_t)k * n2 + i2a + il) * NQ + t];
  }
  const int J2M = A.T2M + 2 * P;
  for (int e = tid; e < NB * J2 * NQ; e += nth) {
    int t = e % NQ, r = e / NQ, jl = r % J2, b = r / J2;
    b2s[(b * J2M + jl) * NQ + t] = (Real)A.d[1].bt[((size_t)b * n2 + j2a + jl) * NQ + t];
  }
  __syncthreads();

  const int qw1 = q0j1[i1a - j1a];
  const int W1 = q0j1[i1b - 1 - j1a] + nqj1[i1b - 1 - j1a] - qw1;
  const int qw2 = q0j2[i2a - j2a];
  const int W2 = q0j2[i2b - 1 - j2a] + nqj2[i2b - 1 - j2a] - qw2;
  const int qi3 = A.d[2].q0[i3], ni3 = A.d[2].nq[i3];
  const int64_t plane = (int64_t)A.nqp1 * A.nqp2;
  const int64_t N1 = A.d[0].prefix[n1], N2 = A.d[1].prefix[n2];
  const int64_t P3i = A.d[2].prefix[i3];
  const int bw3 = band_w(i3, P, n3), jlo3 = band_lo(i3, P);
  OutT* vals = reinterpret_cast<OutT*>(A.vals);

  for (int t3 = 0; t3 < BW; ++t3) {
    const int j3 = i3 - P + t3;
    if (j3 < 0 || j3 >= n3) continue;
    const int qj3 = A.d[2].q0[j3], nj3 = A.d[2].nq[j3];
    const int lo3 = max(qi3, qj3), hi3 = min(qi3 + ni3, qj3 + nj3), n3o = hi3 - lo3;
    __syncthreads();  // previous iteration's readers of a3s, gs
    for (int e = tid; e < NK * n3o; e += nth) {
      int k = e / n3o, q = lo3 + e % n3o;
      int b = k & 1;
      double wv = A.d[2].w[((size_t)k * n3 + i3) * NQ + (q - qi3)];
      double bv = A.d[2].bt[((size_t)b * n3 + j3) * NQ + (q - qj3)];
      a3s[k * NQ + (q - lo3)] = (Real)(wv * bv);
    }
    for (int e = tid; e < NG * T2 * BW * W1; e += nth) gs[e] = (Real)0;
    __syncthreads();

    for (int c = 0; c < NCLASS; ++c) {
      const int tb = MASS ? 0 : kClassStart[c], te = MASS ? 1 : kClassStart[c + 1];
      const int lc = MASS ? 0 : kTermL[tb], mc = MASS ? 0 : kTermM[tb];
      const int grp = MASS ? 0 : 2 * (lc == 0) + (mc == 0);
      const int b2 = MASS ? 0 : (mc == 1);
      for (int e = tid; e < T2 * NQ * W1; e += nth) h2s[e] = (Real)0;
      for (int term = tb; term < te; ++term) {
        const int l = MASS ? 0 : kTermL[term], m = MASS ? 0 : kTermM[term];
        const int slot = MASS ? 6 : kSlot[l][m];
        const int k3 = MASS ? 0 : 2 * (l == 2) + (m == 2);
        const int k2 = MASS ? 0 : 2 * (l == 1) + (m == 1);
        const double* cs = A.coef + (int64_t)slot * A.nqp_total;
        __syncthreads();  // t3s free, h2s zeroed
        // stage 3: contract q3; two independent items per thread
        const Real* a3 = a3s + k3 * NQ;
        for (int e0 = tid; e0 < W1 * W2; e0 += 2 * nth) {
          const int e1 = e0 + nth;
          const bool two = e1 < W1 * W2;
          const int64_t base0 = (int64_t)(qw2 + e0 / W1) * A.nqp1 + (qw1 + e0 % W1);
          const int64_t base1 = two ? (int64_t)(qw2 + e1 / W1) * A.nqp1 + (qw1 + e1 % W1) : base0;
          const double* c0 = cs + (int64_t)lo3 * plane + base0;
          const double* c1 = cs + (int64_t)lo3 * plane + base1;
          Real acc0 = (Real)0, acc1 = (Real)0;
          if (A.kappa) {
            const double* k0 = A.kappa + (int64_t)lo3 * plane + base0;
            const double* k1 = A.kappa + (int64_t)lo3 * plane + base1;
#pragma unroll 4
            for (int q = 0; q < n3o; ++q) {
              acc0 = fmaT<Real>(a3[q], (Real)(c0[q * plane] * k0[q * plane]), acc0);
              acc1 = fmaT<Real>(a3[q], (Real)(c1[q * plane] * k1[q * plane]), acc1);
            }
          } else {
#pragma unroll 4
            for (int q = 0; q < n3o; ++q) {
              acc0 = fmaT<Real>(a3[q], (Real)c0[q * plane], acc0);
              acc1 = fmaT<Real>(a3[q], (Real)c1[q * plane], acc1);
            }
          }
          t3s[e0] = acc0;
          if (two) t3s[e1] = acc1;
        }
        __syncthreads();
        // stage 2a: fold the direction-2 test weights of this term into H2
        for (int e = tid; e < T2 * NQ * W1; e += nth) {
          const int q1l = e % W1, r = e / W1, t = r % NQ, il = r / NQ;
          const int jl = i2a + il - j2a;
          if (t >= nqj2[jl]) continue;
          const int q2 = q0j2[jl] + t;
          h2s[e] = fmaT<Real>(w2s[(k2 * A.T2M + il) * NQ + t], t3s[(q2 - qw2) * W1 + q1l], h2s[e]);
        }
      }
      __syncthreads();
      // stage 2b: contract q2 against the trial B-splines of direction 2. One item
      // per (q1, i2, half of the band): the q2 loop runs outside, the j2 outputs of
      // the half are independent accumulators.
      {
        constexpr int HB = P + 1;  // outputs per half: tt2 in [0, P] or [P+1, 2P]
        for (int e = tid; e < T2 * 2 * W1; e += nth) {
          const int q1l = e % W1, r = e / W1, half = r & 1, il = r >> 1;
          const int i2 = i2a + il, il2 = i2 - j2a;
          const int qi = q0j2[il2], ni = nqj2[il2];
          int lo[HB], hi[HB], jl[HB];
          Real acc[HB];
#pragma unroll
          for (int k = 0; k < HB; ++k) {
            const int tt2 = half * (P + 1) + k;
            const int j2 = i2 - P + tt2;
            acc[k] = (Real)0;
            if (tt2 < BW && j2 >= 0 && j2 < n2) {
              const int jj = j2 - j2a;
              jl[k] = jj;
              lo[k] = max(qi, q0j2[jj]);
              hi[k] = min(qi + ni, q0j2[jj] + nqj2[jj]);
            } else {
              jl[k] = 0;
              lo[k] = 1 << 30;
              hi[k] = -(1 << 30);
            }
          }
          const Real* hh = h2s + il * NQ * W1 + q1l;
          const Real* bb = b2s + b2 * J2M * NQ;
          for (int t = 0; t < ni; ++t) {
            const int q = qi + t;
            const Real hv = hh[t * W1];
#pragma unroll
            for (int k = 0; k < HB; ++k)
              if (q >= lo[k] && q < hi[k]) acc[k] = fmaT<Real>(bb[jl[k] * NQ + q - q0j2[jl[k]]], hv, acc[k]);
          }
#pragma unroll
          for (int k = 0; k < HB; ++k) {
            const int tt2 = half * (P + 1) + k;
            if (hi[k] > lo[k]) gs[((grp * T2 + il) * BW + tt2) * W1 + q1l] += acc[k];
          }
        }
      }
      __syncthreads();
    }

    // stage 1: contract q1 and store. The q1 loop runs outside; the 2p+1 outputs
    // of the row (one per j1) are independent accumulators.
    const int jl3 = j3 - jlo3;
    for (int e = tid; e < T1 * T2 * BW; e += nth) {
      const int il1 = e % T1, r = e / T1, tt2 = r % BW, il2 = r / BW;
      const int i1 = i1a + il1, i2 = i2a + il2, j2 = i2 - P + tt2;
      if (j2 < 0 || j2 >= n2) continue;
      const int qi1 = q0j1[i1 - j1a], ni1 = nqj1[i1 - j1a];
      int lo[BW], hi[BW], qj[BW];
      Real s[BW];
#pragma unroll
      for (int tt1 = 0; tt1 < BW; ++tt1) {
        const int j1 = i1 - P + tt1;
        s[tt1] = (Real)0;
        if (j1 >= 0 && j1 < n1) {
          qj[tt1] = q0j1[j1 - j1a];
          lo[tt1] = max(qi1, qj[tt1]);
          hi[tt1] = min(qi1 + ni1, qj[tt1] + nqj1[j1 - j1a]);
        } else {
          qj[tt1] = 0;
          lo[tt1] = 1 << 30;
          hi[tt1] = -(1 << 30);
        }
      }
      const int gstride = T2 * BW * W1;
      const Real* g0 = gs + (il2 * BW + tt2) * W1;   // group 0; group g at + g * gstride
      const Real* wk = w1s + il1 * NQ;               // kind 0; kind k at + k * T1M * NQ
      const int jrow0 = i1 - P - j1a;                // b1s row of tt1 = 0 (may be < 0)
      for (int q = qi1; q < qi1 + ni1; ++q) {
        const int gq = q - qw1, wq = q - qi1;
        Real h0, h1 = (Real)0;
        if (MASS) {
          h0 = wk[wq] * g0[gq];
        } else {
          // groups g = 2a+b: h_b = w^{(0,b)} G_{(0,b)} + w^{(1,b)} G_{(1,b)}
          h0 = fmaT<Real>(wk[wq], g0[gq], wk[wq + 2 * A.T1M * NQ] * g0[gq + 2 * gstride]);
          h1 = fmaT<Real>(wk[wq + A.T1M * NQ], g0[gq + gstride], wk[wq + 3 * A.T1M * NQ] * g0[gq + 3 * gstride]);
        }
#pragma unroll
        for (int tt1 = 0; tt1 < BW; ++tt1) {
          if (q >= lo[tt1] && q < hi[tt1]) {
            const int idx = (jrow0 + tt1) * NQ + q - qj[tt1];
            if (MASS)
              s[tt1] = fmaT<Real>(b1s[idx], h0, s[tt1]);
            else
              s[tt1] = fmaT<Real>(b1s[idx + J1M * NQ], h1, fmaT<Real>(b1s[idx], h0, s[tt1]));
          }
        }
      }
      const int64_t row = P3i * N2 * N1 +
                          (int64_t)bw3 * (A.d[1].prefix[i2] * N1 + (int64_t)band_w(i2, P, n2) * A.d[0].prefix[i1]);
      const int bw1 = band_w(i1, P, n1), bw2 = band_w(i2, P, n2);
      const int jlo1 = band_lo(i1, P), jlo2 = band_lo(i2, P);
      const int64_t base = row + ((int64_t)jl3 * bw2 + (j2 - jlo2)) * bw1 - jlo1;
#pragma unroll
      for (int tt1 = 0; tt1 < BW; ++tt1) {
        const int j1 = i1 - P + tt1;
        if (j1 >= 0 && j1 < n1) vals[base + j1] = (OutT)s[tt1];
      }
    }
  }
}

// Host-side closed forms of Q_i (same as the set-up kernels) for tile windows.
static void q_range_host(int i, int p, int n_el, int nqp, int* qs, int* qe) {
  int lo = std::max(0, i - p), hi = std::min(n_el, i + 1);
  *qs = lo == 0 ? 0 : 2 * lo + p;
  *qe = hi == n_el ? nqp - 1 : 2 * hi + p - 2;
}

static int max_window(const wq_plan_s* pl, int l, int nt) {
  const int n = (int)pl->n[l], p = pl->p, ne = n - p, nqp = (int)pl->nqp[l];
  int best = 0;
  for (int t = 0; t < nt; ++t) {
    int a = (int)((int64_t)t * n / nt), b = (int)((int64_t)(t + 1) * n / nt);
    if (b <= a) continue;
    int qs0, qe0, qs1, qe1;
    q_range_host(a, p, ne, nqp, &qs0, &qe0);
    q_range_host(b - 1, p, ne, nqp, &qs1, &qe1);
    best = std::max(best, qe1 - qs0 + 1);
  }
  return best;
}

struct TileChoice {
  int t1, t2;
};

static TileChoice tiles_for(int p) {
  (void)p;
  return TileChoice{16, 4};
}

template <int P, bool MASS, typename Real, typename OutT>
static wq_status launch_t(wq_plan_s* pl, const double* kappa, void* vals, cudaStream_t s) {
  AsmArgs A;
  for (int l = 0; l < 3; ++l) {
    A.d[l].n = pl->dir[l].n;
    A.d[l].q0 = pl->dir[l].q0;
    A.d[l].nq = pl->dir[l].nq;
    A.d[l].w = pl->dir[l].w;
    A.d[l].bt = pl->dir[l].bt;
    A.d[l].prefix = pl->dir[l].prefix;
  }
  A.NQ = pl->nq_max;
  A.coef = pl->coef;
  A.kappa = kappa;
  A.nqp_total = pl->n_qp_total;
  A.nqp1 = (int)pl->nqp[0];
  A.nqp2 = (int)pl->nqp[1];
  A.vals = vals;
  TileChoice tc = tiles_for(P);
  const int n1 = (int)pl->n[0], n2 = (int)pl->n[1], n3 = (int)pl->n[2];
  A.nt1 = (n1 + tc.t1 - 1) / tc.t1;
  A.nt2 = (n2 + tc.t2 - 1) / tc.t2;
  A.T1M = (n1 + A.nt1 - 1) / A.nt1;
  A.T2M = (n2 + A.nt2 - 1) / A.nt2;
  A.W1M = max_window(pl, 0, A.nt1);
  A.W2M = max_window(pl, 1, A.nt2);
  SmemLayout L = smem_layout<P, MASS>(A.NQ, A.T1M, A.T2M, A.W1M, A.W2M);
  size_t smem = sizeof(Real) * (size_t)L.total_real + sizeof(int) * (size_t)L.ints + 16;
  if (smem > 227 * 1024) return set_error(WQ_ERR_UNSUPPORTED, "tile does not fit in shared memory");
  auto kern = k_assemble<P, MASS, Real, OutT>;
  WQ_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
              "assembly kernel attributes");
  int64_t blocks = (int64_t)A.nt1 * A.nt2 * n3;
  kern<<<(unsigned)blocks, 256, smem, s>>>(A);
  count_launch();
  WQ_CUDA_TRY(cudaGetLastError(), "assembly kernel launch");
  return WQ_OK;
}

template <bool MASS, typename Real, typename OutT>
static wq_status dispatch(wq_plan_s* pl, const double* kappa, void* vals, cudaStream_t s) {
  switch (pl->p) {
    case 2: return launch_t<2, MASS, Real, OutT>(pl, kappa, vals, s);
    case 3: return launch_t<3, MASS, Real, OutT>(pl, kappa, vals, s);
    case 4: return launch_t<4, MASS, Real, OutT>(pl, kappa, vals, s);
    case 5: return launch_t<5, MASS, Real, OutT>(pl, kappa, vals, s);
    case 6: return launch_t<6, MASS, Real, OutT>(pl, kappa, vals, s);
    case 7: return launch_t<7, MASS, Real, OutT>(pl, kappa, vals, s);
    case 8: return launch_t<8, MASS, Real, OutT>(pl, kappa, vals, s);
    default: return set_error(WQ_ERR_UNSUPPORTED, "degree out of range");
  }
}

wq_status launch_assemble_f64(wq_plan_s* pl, bool mass, const double* kappa, double* vals, cudaStream_t s) {
  return mass ? dispatch<true, double, double>(pl, kappa, vals, s)
              : dispatch<false, double, double>(pl, kappa, vals, s);
}

wq_status launch_assemble_f32(wq_plan_s* pl, bool mass, const double* kappa, void* vals, int value_dtype,
                              cudaStream_t s) {
  if (value_dtype == WQ_VALUES_F32)
    return mass ? dispatch<true, float, float>(pl, kappa, vals, s) : dispatch<false, float, float>(pl, kappa, vals, s);
  return mass ? dispatch<true, float, double>(pl, kappa, vals, s) : dispatch<false, float, double>(pl, kappa, vals, s);
}

}  // namespace wq

using wq::set_error;

static wq_status assemble(wq_plan_t plan, bool mass, const double* kappa, void* vals, int value_dtype, int precision,
                          void* stream) {
  if (!plan || !vals) return set_error(WQ_ERR_INVALID_ARG, "NULL argument");
  if (value_dtype != WQ_VALUES_F64 && value_dtype != WQ_VALUES_F32)
    return set_error(WQ_ERR_INVALID_ARG, "unknown value dtype");
  cudaStream_t s = (cudaStream_t)stream;
  if (precision == WQ_PREC_FP64) {
    if (value_dtype != WQ_VALUES_F64) return set_error(WQ_ERR_INVALID_ARG, "FP64 contractions write FP64 values");
    return wq::launch_assemble_f64(plan, mass, kappa, (double*)vals, s);
  }
  if (precision == WQ_PREC_FP32) return wq::launch_assemble_f32(plan, mass, kappa, vals, value_dtype, s);
  return set_error(WQ_ERR_UNSUPPORTED, "unknown precision");
}

extern "C" wq_status wq_assemble_stiffness(wq_plan_t plan, const double* d_kappa, void* d_vals, int value_dtype,
                                           int precision, void* stream) {
  return assemble(plan, false, d_kappa, d_vals, value_dtype, precision, stream);
}

extern "C" wq_status wq_assemble_mass(wq_plan_t plan, const double* d_kappa, void* d_vals, int value_dtype,
                                      int precision, void* stream) {
  return assemble(plan, true, d_kappa, d_vals, value_dtype, precision, stream);
}

extern "C" wq_status wq_assemble_host(wq_plan_t plan, int which, const double* h_ctrl, double* d_vals, double* h_vals,
                                      void* stream) {
  if (!plan || !d_vals || !h_vals || (which != 0 && which != 1)) return set_error(WQ_ERR_INVALID_ARG, "bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  wq_status st = wq_plan_refresh(plan, h_ctrl, 0, stream);
  if (st != WQ_OK) return st;
  st = assemble(plan, which == 1, nullptr, d_vals, WQ_VALUES_F64, WQ_PREC_FP64, stream);
  if (st != WQ_OK) return st;
  WQ_CUDA_TRY(cudaMemcpyAsync(h_vals, d_vals, sizeof(double) * plan->nnz, cudaMemcpyDeviceToHost, s), "value copy");
  WQ_CUDA_TRY(cudaStreamSynchronize(s), "stream synchronize");
  return WQ_OK;
}
