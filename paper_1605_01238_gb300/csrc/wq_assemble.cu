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
#include <vector>

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
  int T1, T2;            // target tile extents (TileSplit)
  int T1M, T2M;          // largest tile extents
  int W1M, W2M;          // largest point windows of a tile
};

// Term (l, m) of Eq. (stiff), ordered by class; class c covers terms
// [kClassStart[c], kClassStart[c+1]).
__constant__ int kTermL[9] = {0, 0, 0, 1, 2, 1, 2, 1, 2};
__constant__ int kTermM[9] = {0, 1, 2, 0, 0, 1, 1, 2, 2};
__constant__ int kClassStart[7] = {0, 1, 2, 3, 5, 7, 9};
__constant__ int kSlot[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};

// Tiles of one direction: rows [0, p+1) and [n-p-1, n) have irregular point sets
// (their supports reach a boundary span); rows in between are regular:
// Q_i = [2i - p, 2i + p]. Each of the three segments is split into tiles of at
// most T rows, so a tile is either wholly regular or wholly boundary. When the
// regular segment is empty the whole range is one boundary segment.
struct TileSplit {
  int n, p, T;
  __host__ __device__ int seg_count(int len) const { return len > 0 ? (len + T - 1) / T : 0; }
  __host__ __device__ bool has_mid() const { return n - p - 1 > p + 1; }
  __host__ __device__ int count() const {
    if (!has_mid()) return seg_count(n);
    return 2 * seg_count(p + 1) + seg_count(n - 2 * (p + 1));
  }
  // bounds [a, b) of tile t and whether its rows are regular
  __host__ __device__ void tile(int t, int* a, int* b, bool* regular) const {
    int lo, len, k, m;
    if (!has_mid()) {
      lo = 0; len = n; m = seg_count(n); k = t; *regular = false;
    } else {
      const int nb = seg_count(p + 1), nm = seg_count(n - 2 * (p + 1));
      if (t < nb) { lo = 0; len = p + 1; m = nb; k = t; *regular = false; }
      else if (t < nb + nm) { lo = p + 1; len = n - 2 * (p + 1); m = nm; k = t - nb; *regular = true; }
      else { lo = n - p - 1; len = p + 1; m = nb; k = t - nb - nm; *regular = false; }
    }
    *a = lo + (int)((int64_t)k * len / m);
    *b = lo + (int)((int64_t)(k + 1) * len / m);
  }
};

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


// Stage 2b for one item (q1, i2) of a regular direction-2 tile: the 2P+1 outputs
// j2 = i2 - P + tt2 share the row's 2P+1 points; the (t, tt2) pattern is static.
template <int P, typename Real>
__device__ __forceinline__ void stage2b_regular(const Real* h2s, const Real* b2s, Real* gs, const int* q0j2, int il,
                                                int q1l, int i2a, int j2a, int NQ, int J2M, int W1, int T2, int b2,
                                                int grp) {
  constexpr int BW = 2 * P + 1;
  const int i2 = i2a + il;
  const int qi = q0j2[i2 - j2a];
  const Real* hh = h2s + il * NQ * W1 + q1l;
  int brow[BW];
  Real acc[BW];
#pragma unroll
  for (int tt2 = 0; tt2 < BW; ++tt2) {
    const int jl = i2 - P + tt2 - j2a;
    brow[tt2] = (b2 * J2M + jl) * NQ + qi - q0j2[jl];
    acc[tt2] = (Real)0;
  }
#pragma unroll
  for (int t = 0; t <= 2 * P; ++t) {
    const Real hv = hh[t * W1];
#pragma unroll
    for (int tt2 = 0; tt2 < BW; ++tt2)
      if (t >= 2 * tt2 - 2 * P && t <= 2 * tt2) acc[tt2] = fmaT<Real>(b2s[brow[tt2] + t], hv, acc[tt2]);
  }
  Real* g = gs + (grp * T2 + il) * BW * W1 + q1l;
#pragma unroll
  for (int tt2 = 0; tt2 < BW; ++tt2) g[tt2 * W1] += acc[tt2];
}

// Stage 1 for one (row i1, column block) of a regular direction-1 tile: the row's
// 2P+1 points t, the 2P+1 outputs j1 = i1 - P + tt1, pattern t in [2 tt1 - 2P, 2 tt1].
template <int P, bool MASS, typename Real, typename OutT>
__device__ __forceinline__ void stage1_regular(const Real* g0, const Real* wk, const Real* b1s, const int* q0j1,
                                               OutT* out, int i1, int j1a, int gq0, int qi1, int NQ, int J1M,
                                               int T1M, int gstride) {
  constexpr int BW = 2 * P + 1;
  int brow[BW];
  Real s[BW];
#pragma unroll
  for (int tt1 = 0; tt1 < BW; ++tt1) {
    const int jl = i1 - P + tt1 - j1a;
    brow[tt1] = jl * NQ + qi1 - q0j1[jl];
    s[tt1] = (Real)0;
  }
#pragma unroll
  for (int t = 0; t <= 2 * P; ++t) {
    const int gq = gq0 + t;
    Real h0, h1 = (Real)0;
    if (MASS) {
      h0 = wk[t] * g0[gq];
    } else {
      h0 = fmaT<Real>(wk[t], g0[gq], wk[t + 2 * T1M * NQ] * g0[gq + 2 * gstride]);
      h1 = fmaT<Real>(wk[t + T1M * NQ], g0[gq + gstride], wk[t + 3 * T1M * NQ] * g0[gq + 3 * gstride]);
    }
#pragma unroll
    for (int tt1 = 0; tt1 < BW; ++tt1) {
      if (t >= 2 * tt1 - 2 * P && t <= 2 * tt1) {
        if (MASS)
          s[tt1] = fmaT<Real>(b1s[brow[tt1] + t], h0, s[tt1]);
        else
          s[tt1] = fmaT<Real>(b1s[brow[tt1] + J1M * NQ + t], h1, fmaT<Real>(b1s[brow[tt1] + t], h0, s[tt1]));
      }
    }
  }
#pragma unroll
  for (int tt1 = 0; tt1 < BW; ++tt1) out[i1 - P + tt1] = (OutT)s[tt1];
}

// One tile (tile1, tile2, i3) of one matrix: the body shared by the per-plan
// kernel and the persistent batch kernel. smem_raw holds the tile's tables and
// intermediates (layout from smem_layout); all threads of the block take part.
template <int P, bool MASS, typename Real, typename OutT>
__device__ __forceinline__ void assemble_tile(const AsmArgs& A, int tile1, int tile2, int i3,
                                              unsigned char* smem_raw) {
  constexpr int BW = 2 * P + 1;
  constexpr int NK = MASS ? 1 : 4;   // weight kinds held per direction
  constexpr int NB = MASS ? 1 : 2;   // trial derivative orders
  constexpr int NG = MASS ? 1 : 4;   // stage-1 groups (a1, b1)
  constexpr int NCLASS = MASS ? 1 : 6;
  constexpr int MAXQ = 4 * P + 1;
  Real* sm = reinterpret_cast<Real*>(smem_raw);
  const int NQ = A.NQ;
  const SmemLayout L = smem_layout<P, MASS>(NQ, A.T1M, A.T2M, A.W1M, A.W2M);
  int* si = reinterpret_cast<int*>(sm + L.total_real);

  const int n1 = A.d[0].n, n2 = A.d[1].n, n3 = A.d[2].n;
  int i1a, i1b, i2a, i2b;
  bool reg1, reg2;
  TileSplit{n1, P, A.T1}.tile(tile1, &i1a, &i1b, &reg1);
  TileSplit{n2, P, A.T2}.tile(tile2, &i2a, &i2b, &reg2);
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
        // stage 3: contract q3; a thread takes its items two at a time when it has two
        const Real* a3 = a3s + k3 * NQ;
        for (int e0 = tid; e0 < W1 * W2; e0 += 2 * nth) {
          const int e1 = e0 + nth;
          const int64_t base0 = (int64_t)(qw2 + e0 / W1) * A.nqp1 + (qw1 + e0 % W1);
          const double* c0 = cs + (int64_t)lo3 * plane + base0;
          const double* k0 = A.kappa ? A.kappa + (int64_t)lo3 * plane + base0 : nullptr;
          Real acc0 = (Real)0;
          if (e1 < W1 * W2) {
            const int64_t base1 = (int64_t)(qw2 + e1 / W1) * A.nqp1 + (qw1 + e1 % W1);
            const double* c1 = cs + (int64_t)lo3 * plane + base1;
            Real acc1 = (Real)0;
            if (k0) {
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
            t3s[e1] = acc1;
          } else if (k0) {
#pragma unroll 4
            for (int q = 0; q < n3o; ++q) acc0 = fmaT<Real>(a3[q], (Real)(c0[q * plane] * k0[q * plane]), acc0);
          } else {
#pragma unroll 4
            for (int q = 0; q < n3o; ++q) acc0 = fmaT<Real>(a3[q], (Real)c0[q * plane], acc0);
          }
          t3s[e0] = acc0;
        }
        __syncthreads();
        // stage 2a: fold the direction-2 test weights of this term into H2
        if (reg2) {
          constexpr int NR = 2 * P + 1;  // |Q_i2| of regular rows; q2 - qw2 = 2 il + t
          for (int e = tid; e < T2 * NR * W1; e += nth) {
            const int q1l = e % W1, r = e / W1, t = r % NR, il = r / NR;
            Real* hp = h2s + (il * NQ + t) * W1 + q1l;
            *hp = fmaT<Real>(w2s[(k2 * A.T2M + il) * NQ + t], t3s[(2 * il + t) * W1 + q1l], *hp);
          }
        } else {
          for (int e = tid; e < T2 * NQ * W1; e += nth) {
            const int q1l = e % W1, r = e / W1, t = r % NQ, il = r / NQ;
            const int jl = i2a + il - j2a;
            if (t >= nqj2[jl]) continue;
            const int q2 = q0j2[jl] + t;
            h2s[e] = fmaT<Real>(w2s[(k2 * A.T2M + il) * NQ + t], t3s[(q2 - qw2) * W1 + q1l], h2s[e]);
          }
        }
      }
      __syncthreads();
      // stage 2b: contract q2 against the trial B-splines of direction 2.
      if (reg2) {
        // regular rows: t = q2 - q0(i2) in [0, 2P]; j2 = i2 - P + tt2 meets the row at
        // t in [2 tt2 - 2P, 2 tt2] n [0, 2P], a pattern fixed at compile time. One item
        // per (q1, i2) with the 2P+1 outputs j2 as independent accumulators.
        for (int e = tid; e < T2 * W1; e += nth)
          stage2b_regular<P, Real>(h2s, b2s, gs, q0j2, e / W1, e % W1, i2a, j2a, NQ, J2M, W1, T2, b2, grp);
      } else {
        for (int e = tid; e < T2 * BW * W1; e += nth) {
          const int q1l = e % W1, r = e / W1, tt2 = r % BW, il = r / BW;
          const int i2 = i2a + il, j2 = i2 - P + tt2;
          if (j2 < 0 || j2 >= n2) continue;
          const int il2 = i2 - j2a, jl2 = j2 - j2a;
          const int qi = q0j2[il2], qj = q0j2[jl2];
          const int lo = max(qi, qj), hi = min(qi + nqj2[il2], qj + nqj2[jl2]);
          Real acc = (Real)0;
          const Real* bb = b2s + (b2 * J2M + jl2) * NQ;
          const Real* hh = h2s + il * NQ * W1 + q1l;
          for (int q = lo; q < hi; ++q) acc = fmaT<Real>(bb[q - qj], hh[(q - qi) * W1], acc);
          gs[((grp * T2 + il) * BW + tt2) * W1 + q1l] += acc;
        }
      }
      __syncthreads();
    }

    // stage 1: contract q1 and store.
    const int jl3 = j3 - jlo3;
    for (int e = tid; e < T1 * T2 * BW; e += nth) {
      const int il1 = e % T1, r = e / T1, tt2 = r % BW, il2 = r / BW;
      const int i1 = i1a + il1, i2 = i2a + il2, j2 = i2 - P + tt2;
      if (j2 < 0 || j2 >= n2) continue;
      const int64_t row = P3i * N2 * N1 +
                          (int64_t)bw3 * (A.d[1].prefix[i2] * N1 + (int64_t)band_w(i2, P, n2) * A.d[0].prefix[i1]);
      const int bw1 = band_w(i1, P, n1), bw2 = band_w(i2, P, n2);
      const int jlo1 = band_lo(i1, P), jlo2 = band_lo(i2, P);
      const int64_t base = row + ((int64_t)jl3 * bw2 + (j2 - jlo2)) * bw1 - jlo1;
      const int gstride = T2 * BW * W1;
      const Real* g0 = gs + (il2 * BW + tt2) * W1;   // group 0; group g at + g * gstride
      const Real* wk = w1s + il1 * NQ;               // kind 0; kind k at + k * T1M * NQ
      const int qi1 = q0j1[i1 - j1a];
      if (reg1) {
        stage1_regular<P, MASS, Real, OutT>(g0, wk, b1s, q0j1, vals + base, i1, j1a, qi1 - qw1, qi1,
                                            NQ, J1M, A.T1M, gstride);
      } else {
        const int ni1 = nqj1[i1 - j1a];
        Real h0[MAXQ], h1[MAXQ];
        for (int t = 0; t < ni1; ++t) {
          const int gq = qi1 + t - qw1;
          if (MASS) {
            h0[t] = wk[t] * g0[gq];
          } else {
            h0[t] = fmaT<Real>(wk[t], g0[gq], wk[t + 2 * A.T1M * NQ] * g0[gq + 2 * gstride]);
            h1[t] = fmaT<Real>(wk[t + A.T1M * NQ], g0[gq + gstride], wk[t + 3 * A.T1M * NQ] * g0[gq + 3 * gstride]);
          }
        }
#pragma unroll
        for (int tt1 = 0; tt1 < BW; ++tt1) {
          const int j1 = i1 - P + tt1;
          if (j1 < 0 || j1 >= n1) continue;
          const int qj = q0j1[j1 - j1a];
          const int lo = max(qi1, qj), hi = min(qi1 + ni1, qj + nqj1[j1 - j1a]);
          const Real* bb0 = b1s + (j1 - j1a) * NQ;
          Real s = (Real)0;
          if (MASS) {
            for (int q = lo; q < hi; ++q) s = fmaT<Real>(bb0[q - qj], h0[q - qi1], s);
          } else {
            const Real* bb1 = bb0 + J1M * NQ;
            for (int q = lo; q < hi; ++q)
              s = fmaT<Real>(bb1[q - qj], h1[q - qi1], fmaT<Real>(bb0[q - qj], h0[q - qi1], s));
          }
          vals[base + j1] = (OutT)s;
        }
      }
    }
  }
}


template <int P, bool MASS, typename Real, typename OutT>
__global__ void __launch_bounds__(256) k_assemble(AsmArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int bid = blockIdx.x;
  const int tile1 = bid % A.nt1;
  bid /= A.nt1;
  const int tile2 = bid % A.nt2;
  const int i3 = bid / A.nt2;
  assemble_tile<P, MASS, Real, OutT>(A, tile1, tile2, i3, smem_raw);
}

// ---------------------------------------------------------------------------
// Batched assembly: many patches of different size and degree, stiffness and/or
// mass, in one persistent launch. Work items (job, tile1, tile2, i3) are taken in
// order from an atomic counter (the host sorts them longest first); no block
// ever waits on another, so the loop ends when the list is exhausted.
struct BatchJob {
  AsmArgs A;
  int p;
  int mass;
};

struct BatchItem {
  int job, tile1, tile2, i3;
};

template <bool MASS>
__device__ __forceinline__ void batch_dispatch(const BatchJob& J, const BatchItem& it, unsigned char* smem) {
  switch (J.p) {
    case 2: assemble_tile<2, MASS, double, double>(J.A, it.tile1, it.tile2, it.i3, smem); break;
    case 3: assemble_tile<3, MASS, double, double>(J.A, it.tile1, it.tile2, it.i3, smem); break;
    case 4: assemble_tile<4, MASS, double, double>(J.A, it.tile1, it.tile2, it.i3, smem); break;
    case 5: assemble_tile<5, MASS, double, double>(J.A, it.tile1, it.tile2, it.i3, smem); break;
    case 6: assemble_tile<6, MASS, double, double>(J.A, it.tile1, it.tile2, it.i3, smem); break;
    case 7: assemble_tile<7, MASS, double, double>(J.A, it.tile1, it.tile2, it.i3, smem); break;
    case 8: assemble_tile<8, MASS, double, double>(J.A, it.tile1, it.tile2, it.i3, smem); break;
  }
}

__global__ void __launch_bounds__(256) k_assemble_batch(const BatchJob* jobs, const BatchItem* items, int n_items,
                                                        unsigned int* counter) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int next;
  for (;;) {
    if (threadIdx.x == 0) next = (int)atomicAdd(counter, 1u);
    __syncthreads();
    const int k = next;
    __syncthreads();  // every thread has read `next` before thread 0 overwrites it
    if (k >= n_items) break;
    const BatchItem it = items[k];
    const BatchJob& J = jobs[it.job];
    if (J.mass)
      batch_dispatch<true>(J, it, smem_raw);
    else
      batch_dispatch<false>(J, it, smem_raw);
    __syncthreads();  // shared memory is reused by the next item
  }
}

// Host-side closed forms of Q_i (same as the set-up kernels) for tile windows.
static void q_range_host(int i, int p, int n_el, int nqp, int* qs, int* qe) {
  int lo = std::max(0, i - p), hi = std::min(n_el, i + 1);
  *qs = lo == 0 ? 0 : 2 * lo + p;
  *qe = hi == n_el ? nqp - 1 : 2 * hi + p - 2;
}

static void tile_extents(const wq_plan_s* pl, int l, int T, int* count, int* max_rows, int* max_win) {
  const int n = (int)pl->n[l], p = pl->p, ne = n - p, nqp = (int)pl->nqp[l];
  TileSplit ts{n, p, T};
  *count = ts.count();
  *max_rows = 0;
  *max_win = 0;
  for (int t = 0; t < *count; ++t) {
    int a, b;
    bool reg;
    ts.tile(t, &a, &b, &reg);
    if (b <= a) continue;
    int qs0, qe0, qs1, qe1;
    q_range_host(a, p, ne, nqp, &qs0, &qe0);
    q_range_host(b - 1, p, ne, nqp, &qs1, &qe1);
    *max_rows = std::max(*max_rows, b - a);
    *max_win = std::max(*max_win, qe1 - qs0 + 1);
  }
}

struct TileChoice {
  int t1, t2;
};

static TileChoice tiles_for(const wq_plan_s* pl) {
  if (pl->tile[0] > 0 && pl->tile[1] > 0) return TileChoice{pl->tile[0], pl->tile[1]};
  return TileChoice{16, 4};
}

// Kernel arguments, tile counts and shared-memory size of one matrix of one plan.
template <int P, bool MASS, typename Real>
static size_t make_args(wq_plan_s* pl, const double* kappa, void* vals, AsmArgs* out) {
  AsmArgs& A = *out;
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
  TileChoice tc = tiles_for(pl);
  A.T1 = tc.t1;
  A.T2 = tc.t2;
  tile_extents(pl, 0, tc.t1, &A.nt1, &A.T1M, &A.W1M);
  tile_extents(pl, 1, tc.t2, &A.nt2, &A.T2M, &A.W2M);
  SmemLayout L = smem_layout<P, MASS>(A.NQ, A.T1M, A.T2M, A.W1M, A.W2M);
  return sizeof(Real) * (size_t)L.total_real + sizeof(int) * (size_t)L.ints + 16;
}

template <int P, bool MASS, typename Real, typename OutT>
static wq_status launch_t(wq_plan_s* pl, const double* kappa, void* vals, cudaStream_t s) {
  AsmArgs A;
  size_t smem = make_args<P, MASS, Real>(pl, kappa, vals, &A);
  const int n3 = (int)pl->n[2];
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

namespace wq {

// NURBS basis functions: value (i, j) times w_i w_j; one warp per row.
template <typename T>
__global__ void k_scale_rows_cols(T* __restrict__ v, const int64_t* __restrict__ row_ptr,
                                  const int32_t* __restrict__ col, const double* __restrict__ w, int64_t n_rows) {
  const int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32;
  const int lane = threadIdx.x & 31;
  if (r >= n_rows) return;
  const double wr = w[r];
  for (int64_t k = row_ptr[r] + lane; k < row_ptr[r + 1]; k += 32) v[k] = (T)((double)v[k] * (wr * w[col[k]]));
}

// Checked mode: flags a NaN or infinite value in the error word.
template <typename T>
__global__ void k_check_finite(const T* __restrict__ v, int64_t n, int* err) {
  bool bad = false;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    bad |= !isfinite(v[i]);
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(err, kErrNonFinite);
}

}  // namespace wq

using wq::set_error;

static wq_status read_error(wq_plan_t plan, cudaStream_t s) { return wq_sync_check(plan, (void*)s); }

static wq_status assemble(wq_plan_t plan, bool mass, const double* kappa, void* vals, int value_dtype, int precision,
                          void* stream) {
  if (!plan || !vals) return set_error(WQ_ERR_INVALID_ARG, "NULL argument");
  if (value_dtype == WQ_VALUES_DEFAULT) value_dtype = plan->opt.value_dtype;
  if (precision == WQ_PREC_DEFAULT) precision = plan->opt.precision;
  if (value_dtype != WQ_VALUES_F64 && value_dtype != WQ_VALUES_F32)
    return set_error(WQ_ERR_INVALID_ARG, "unknown value dtype");
  cudaStream_t s = (cudaStream_t)stream;
  if (precision == WQ_PREC_FP64 && value_dtype != WQ_VALUES_F64)
    return set_error(WQ_ERR_INVALID_ARG, "FP64 contractions write FP64 values");
  if (precision < WQ_PREC_FP64 || precision > WQ_PREC_TF32X3) return set_error(WQ_ERR_UNSUPPORTED, "unknown precision");
  const size_t vbytes = (value_dtype == WQ_VALUES_F64 ? sizeof(double) : sizeof(float)) * (size_t)plan->nnz;
  if (plan->opt.checked) {
    wq_status st = wq::check_device_range(plan, vals, vbytes, "d_vals");
    if (st == WQ_OK && kappa) st = wq::check_device_range(plan, kappa, sizeof(double) * plan->n_qp_total, "d_kappa");
    if (st != WQ_OK) return st;
  }
  if (plan->nurbs_basis && !mass)
    return set_error(WQ_ERR_UNSUPPORTED, "the stiffness matrix with NURBS basis functions is not provided");
  const bool staged = plan->algorithm == WQ_ALGO_STAGED || plan->algorithm == WQ_ALGO_AUTO;
  wq_status st;
  if (precision == WQ_PREC_MIXED || precision == WQ_PREC_F32X2 || precision == WQ_PREC_TF32X3 ||
      ((precision == WQ_PREC_FP64 || precision == WQ_PREC_FP32) && staged))
    st = wq::launch_staged(plan, mass, kappa, vals, value_dtype, precision, s);
  else if (precision == WQ_PREC_FP64)
    st = wq::launch_assemble_f64(plan, mass, kappa, (double*)vals, s);
  else
    st = wq::launch_assemble_f32(plan, mass, kappa, vals, value_dtype, s);
  if (st != WQ_OK) return st;
  if (plan->nurbs_basis) {
    const unsigned blocks = (unsigned)((plan->n_rows * 32 + 255) / 256);
    if (value_dtype == WQ_VALUES_F64)
      wq::k_scale_rows_cols<double><<<blocks, 256, 0, s>>>((double*)vals, plan->row_ptr, plan->col, plan->wts,
                                                             plan->n_rows);
    else
      wq::k_scale_rows_cols<float><<<blocks, 256, 0, s>>>((float*)vals, plan->row_ptr, plan->col, plan->wts,
                                                            plan->n_rows);
    wq::count_launch();
    WQ_CUDA_TRY(cudaGetLastError(), "NURBS basis scaling launch");
  }
  if (!plan->opt.checked) return WQ_OK;
  if (value_dtype == WQ_VALUES_F64)
    wq::k_check_finite<double><<<304, 256, 0, s>>>((const double*)vals, plan->nnz, plan->err);
  else
    wq::k_check_finite<float><<<304, 256, 0, s>>>((const float*)vals, plan->nnz, plan->err);
  wq::count_launch();
  WQ_CUDA_TRY(cudaGetLastError(), "value check launch");
  return read_error(plan, s);
}

extern "C" wq_status wq_plan_reserve(wq_plan_t plan, int precision, int value_dtype, int adjoint, void* stream) {
  if (!plan) return set_error(WQ_ERR_INVALID_ARG, "NULL plan");
  if (value_dtype == WQ_VALUES_DEFAULT) value_dtype = plan->opt.value_dtype;
  if (precision == WQ_PREC_DEFAULT) precision = plan->opt.precision;
  if (value_dtype != WQ_VALUES_F64 && value_dtype != WQ_VALUES_F32)
    return set_error(WQ_ERR_INVALID_ARG, "unknown value dtype");
  if (precision < WQ_PREC_FP64 || precision > WQ_PREC_TF32X3) return set_error(WQ_ERR_UNSUPPORTED, "unknown precision");
  if (precision == WQ_PREC_FP64 && value_dtype != WQ_VALUES_F64)
    return set_error(WQ_ERR_INVALID_ARG, "FP64 contractions write FP64 values");
  cudaStream_t s = (cudaStream_t)stream;
  const bool staged = plan->algorithm == WQ_ALGO_STAGED || plan->algorithm == WQ_ALGO_AUTO;
  wq_status st = WQ_OK;
  if (staged || precision == WQ_PREC_MIXED || precision == WQ_PREC_F32X2 || precision == WQ_PREC_TF32X3)
    st = wq::launch_staged(plan, false, nullptr, nullptr, value_dtype, precision, s);
  if (st == WQ_OK && adjoint) st = wq::reserve_adjoint(plan, s);
  return st;
}

extern "C" wq_status wq_plan_set_tiles(wq_plan_t plan, int t1, int t2) {
  if (!plan) return set_error(WQ_ERR_INVALID_ARG, "NULL plan");
  if (t1 < 0 || t2 < 0 || t1 > 64 || t2 > 64 || (t1 == 0) != (t2 == 0))
    return set_error(WQ_ERR_INVALID_ARG, "tile extents must both be 0 (default) or in 1..64");
  plan->tile[0] = t1;
  plan->tile[1] = t2;
  return WQ_OK;
}

extern "C" wq_status wq_plan_get_tiles(wq_plan_t plan, int* t1, int* t2) {
  if (!plan || !t1 || !t2) return set_error(WQ_ERR_INVALID_ARG, "NULL argument");
  *t1 = plan->tile[0];
  *t2 = plan->tile[1];
  return WQ_OK;
}

extern "C" wq_status wq_plan_set_algorithm(wq_plan_t plan, int algorithm) {
  if (!plan) return set_error(WQ_ERR_INVALID_ARG, "NULL plan");
  if (algorithm != WQ_ALGO_FUSED && algorithm != WQ_ALGO_STAGED && algorithm != WQ_ALGO_AUTO)
    return set_error(WQ_ERR_INVALID_ARG, "unknown algorithm");
  plan->algorithm = algorithm;
  return WQ_OK;
}

extern "C" wq_status wq_assemble_stiffness(wq_plan_t plan, const double* d_kappa, void* d_vals, int value_dtype,
                                           int precision, void* stream) {
  return assemble(plan, false, d_kappa, d_vals, value_dtype, precision, stream);
}

extern "C" wq_status wq_assemble_mass(wq_plan_t plan, const double* d_kappa, void* d_vals, int value_dtype,
                                      int precision, void* stream) {
  return assemble(plan, true, d_kappa, d_vals, value_dtype, precision, stream);
}

namespace {

// Copies the values of one slab of direction 3 back to the host on the plan's copy
// stream, after the assembly stream has reached the end of the slab's kernels.
struct HostCopy {
  wq_plan_s* pl;
  const double* d_vals;
  double* h_vals;
  std::vector<int64_t> P3;  // prefix sums of the band widths of direction 3
};

wq_status copy_slab(void* ctx, int i3a, int i3b, cudaStream_t s) {
  HostCopy* c = static_cast<HostCopy*>(ctx);
  const int64_t per = c->pl->nnz1[0] * c->pl->nnz1[1];  // values per band pair of direction 3
  const int64_t a = c->P3[i3a] * per, b = c->P3[i3b] * per;
  WQ_CUDA_TRY(cudaEventRecord(c->pl->slab_done, s), "slab event");
  WQ_CUDA_TRY(cudaStreamWaitEvent(c->pl->copy_stream, c->pl->slab_done, 0), "slab wait");
  WQ_CUDA_TRY(cudaMemcpyAsync(c->h_vals + a, c->d_vals + a, sizeof(double) * (size_t)(b - a), cudaMemcpyDeviceToHost,
                              c->pl->copy_stream),
              "value copy");
  return WQ_OK;
}

}  // namespace

extern "C" wq_status wq_assemble_host(wq_plan_t plan, int which, const double* h_ctrl, double* d_vals, double* h_vals,
                                      void* stream) {
  if (!plan || !h_vals || (which != 0 && which != 1)) return set_error(WQ_ERR_INVALID_ARG, "bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  wq_status st = wq_plan_refresh(plan, h_ctrl, 0, stream);
  if (st != WQ_OK) return st;
  const bool staged = plan->algorithm == WQ_ALGO_STAGED || plan->algorithm == WQ_ALGO_AUTO;
  if (!staged || plan->opt.checked || plan->nurbs_basis) {
    if (!d_vals) return set_error(WQ_ERR_INVALID_ARG, "d_vals is NULL");
    st = assemble(plan, which == 1, nullptr, d_vals, WQ_VALUES_F64, WQ_PREC_FP64, stream);
    if (st != WQ_OK) return st;
    WQ_CUDA_TRY(cudaMemcpyAsync(h_vals, d_vals, sizeof(double) * plan->nnz, cudaMemcpyDeviceToHost, s), "value copy");
    WQ_CUDA_TRY(cudaStreamSynchronize(s), "stream synchronize");
    return WQ_OK;
  }
  // page-locked host values the device can address (wq_host_alloc, or registered
  // memory): stage 1 stores straight into them, so the values cross the host link once,
  // as they are produced, with no second pass over device memory and no copy engine
  cudaPointerAttributes at{};
  void* h_dev = nullptr;
  const cudaError_t pe = cudaPointerGetAttributes(&at, h_vals);
  if (pe == cudaSuccess && at.type == cudaMemoryTypeHost)
    h_dev = at.devicePointer;
  else if (pe != cudaSuccess)
    cudaGetLastError();  // not memory the runtime knows: the copy path below
  if (h_dev) {
    wq::SlabHook hook;
    hook.host_vals = true;
    st = wq::launch_staged(plan, which == 1, nullptr, h_dev, WQ_VALUES_F64, WQ_PREC_FP64, s, &hook);
    if (st != WQ_OK) return st;
    WQ_CUDA_TRY(cudaStreamSynchronize(s), "stream synchronize");
    return WQ_OK;
  }
  if (!d_vals) return set_error(WQ_ERR_INVALID_ARG, "d_vals is NULL and h_vals is not device-addressable page-locked memory");
  if (!plan->copy_stream) {
    WQ_CUDA_TRY(cudaStreamCreateWithFlags(&plan->copy_stream, cudaStreamNonBlocking), "copy stream");
    WQ_CUDA_TRY(cudaEventCreateWithFlags(&plan->slab_done, cudaEventDisableTiming), "slab event");
  }
  HostCopy c{plan, d_vals, h_vals, std::vector<int64_t>(plan->n[2] + 1, 0)};
  const int n3 = (int)plan->n[2], p = plan->p;
  for (int i = 0; i < n3; ++i) c.P3[i + 1] = c.P3[i] + (std::min(n3 - 1, i + p) - std::max(0, i - p) + 1);
  wq::SlabHook hook;
  hook.rows = std::max(1, (n3 + 7) / 8);  // about eight slabs: the copies overlap all but the last one
  hook.after = copy_slab;
  hook.ctx = &c;
  st = wq::launch_staged(plan, which == 1, nullptr, d_vals, WQ_VALUES_F64, WQ_PREC_FP64, s, &hook);
  cudaError_t e1 = cudaStreamSynchronize(s), e2 = cudaStreamSynchronize(plan->copy_stream);
  if (st != WQ_OK) return st;
  WQ_CUDA_TRY(e1, "stream synchronize");
  WQ_CUDA_TRY(e2, "copy stream synchronize");
  return WQ_OK;
}

extern "C" wq_status wq_host_alloc(size_t bytes, void** h_ptr) {
  if (!h_ptr) return set_error(WQ_ERR_INVALID_ARG, "NULL argument");
  *h_ptr = nullptr;
  if (wq::fault("alloc")) return set_error(WQ_ERR_INJECTED, "injected allocation failure: page-locked host memory");
  cudaError_t e = cudaHostAlloc(h_ptr, bytes ? bytes : 16, cudaHostAllocDefault);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    *h_ptr = nullptr;
    return set_error(WQ_ERR_OOM, "page-locked host allocation failed");
  }
  WQ_CUDA_TRY(e, "page-locked host allocation");
  return WQ_OK;
}

extern "C" wq_status wq_host_free(void* h_ptr) {
  if (h_ptr) WQ_CUDA_TRY(cudaFreeHost(h_ptr), "page-locked host free");
  return WQ_OK;
}

// ---------------------------------------------------------------------------
// Batch host side.

namespace wq {

template <bool MASS>
static size_t job_args(wq_plan_s* pl, void* vals, AsmArgs* A) {
  switch (pl->p) {
    case 2: return make_args<2, MASS, double>(pl, nullptr, vals, A);
    case 3: return make_args<3, MASS, double>(pl, nullptr, vals, A);
    case 4: return make_args<4, MASS, double>(pl, nullptr, vals, A);
    case 5: return make_args<5, MASS, double>(pl, nullptr, vals, A);
    case 6: return make_args<6, MASS, double>(pl, nullptr, vals, A);
    case 7: return make_args<7, MASS, double>(pl, nullptr, vals, A);
    default: return make_args<8, MASS, double>(pl, nullptr, vals, A);
  }
}

}  // namespace wq

struct wq_batch_s {
  int device = 0;
  wq::BatchJob* jobs = nullptr;
  wq::BatchItem* items = nullptr;
  unsigned int* counter = nullptr;
  int n_items = 0;
  int grid = 0;
  size_t smem = 0;
  int64_t nnz_total = 0;
  int64_t kernels = 1;   // kernels one replay launches
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

static void free_batch(wq_batch_s* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->jobs) cudaFree(b->jobs);
  if (b->items) cudaFree(b->items);
  if (b->counter) cudaFree(b->counter);
  delete b;
}

// Staged batch: every patch's staged assembly (the three mode-product kernels of
// Eq. (sumfactorization), stiffness then mass) captured into one CUDA graph on
// up to eight parallel branches, patches assigned largest first to the least
// loaded branch, so that small patches run side by side and the graph fills the
// GPU. Each plan's FP64 staged scratch is reserved before the capture (nothing is
// allocated inside it).
static wq_status batch_staged(wq_batch_s* b, int count, const wq_plan_t* plans, void* const* d_stiffness,
                              void* const* d_mass, cudaStream_t stream) {
  std::vector<int> jobs;
  std::vector<double> cost;
  for (int k = 0; k < count; ++k) {
    const bool s_k = d_stiffness && d_stiffness[k], m_k = d_mass && d_mass[k];
    if (!s_k && !m_k) continue;
    wq_status st = wq_plan_reserve(plans[k], WQ_PREC_FP64, WQ_VALUES_F64, 0, stream);
    if (st != WQ_OK) return st;
    jobs.push_back(k);
    cost.push_back((double)plans[k]->nnz * ((s_k ? 3.0 : 0.0) + (m_k ? 1.0 : 0.0)));
    b->nnz_total += plans[k]->nnz * ((s_k ? 1 : 0) + (m_k ? 1 : 0));
  }
  if (jobs.empty()) return set_error(WQ_ERR_INVALID_ARG, "the batch has no output arrays");
  WQ_CUDA_TRY(cudaStreamSynchronize(stream), "batch reservation");
  const int nb = std::max(1, std::min<int>(8, (int)jobs.size()));
  std::vector<int> order(jobs.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
  std::vector<std::vector<int>> branch(nb);
  std::vector<double> load(nb, 0.0);
  for (int o : order) {
    const int t = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    branch[t].push_back(jobs[o]);
    load[t] += cost[o];
  }
  std::vector<cudaStream_t> bs(nb, nullptr);
  std::vector<cudaEvent_t> ev(nb + 1, nullptr);
  cudaStream_t cs = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  for (int t = 0; t < nb && e == cudaSuccess; ++t) e = cudaStreamCreateWithFlags(&bs[t], cudaStreamNonBlocking);
  for (int t = 0; t <= nb && e == cudaSuccess; ++t) e = cudaEventCreateWithFlags(&ev[t], cudaEventDisableTiming);
  wq_status st = WQ_OK;
  const int64_t launches0 = wq_launch_count();
  bool capturing = false;
  if (e == cudaSuccess) {
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    capturing = e == cudaSuccess;
  }
  if (capturing) {
    e = cudaEventRecord(ev[nb], cs);
    for (int t = 0; t < nb && e == cudaSuccess; ++t) e = cudaStreamWaitEvent(bs[t], ev[nb], 0);
    for (int t = 0; t < nb && e == cudaSuccess && st == WQ_OK; ++t) {
      for (int k : branch[t]) {
        if (st == WQ_OK && d_stiffness && d_stiffness[k])
          st = wq::launch_staged(plans[k], false, nullptr, d_stiffness[k], WQ_VALUES_F64, WQ_PREC_FP64, bs[t]);
        if (st == WQ_OK && d_mass && d_mass[k])
          st = wq::launch_staged(plans[k], true, nullptr, d_mass[k], WQ_VALUES_F64, WQ_PREC_FP64, bs[t]);
      }
      if (e == cudaSuccess) e = cudaEventRecord(ev[t], bs[t]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev[t], 0);
    }
    cudaError_t e2 = cudaStreamEndCapture(cs, &b->graph);
    if (e == cudaSuccess) e = e2;
  }
  if (e == cudaSuccess && st == WQ_OK) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
  b->kernels = wq_launch_count() - launches0;
  for (int t = 0; t < nb; ++t)
    if (bs[t]) cudaStreamDestroy(bs[t]);
  for (int t = 0; t <= nb; ++t)
    if (ev[t]) cudaEventDestroy(ev[t]);
  if (cs) cudaStreamDestroy(cs);
  if (st != WQ_OK) return st;
  if (e != cudaSuccess) return wq::cuda_error(e, "staged batch graph capture");
  b->n_items = (int)jobs.size();
  b->grid = nb;
  return WQ_OK;
}

extern "C" wq_status wq_batch_create(wq_batch_t* out, int count, const wq_plan_t* plans, void* const* d_stiffness,
                                     void* const* d_mass, void* stream) {
  if (!out || count <= 0 || !plans) return set_error(WQ_ERR_INVALID_ARG, "bad batch arguments");
  *out = nullptr;
  bool all_staged = true;
  for (int k = 0; k < count; ++k) {
    if (!plans[k]) return set_error(WQ_ERR_INVALID_ARG, "NULL plan in batch");
    if (plans[k]->nurbs_basis) return set_error(WQ_ERR_UNSUPPORTED, "NURBS basis functions are not batched");
    all_staged = all_staged && plans[k]->algorithm != WQ_ALGO_FUSED;
  }
  if (all_staged) {
    wq_batch_s* b = new wq_batch_s();
    cudaGetDevice(&b->device);
    wq_status st = batch_staged(b, count, plans, d_stiffness, d_mass, (cudaStream_t)stream);
    if (st != WQ_OK) {
      free_batch(b);
      return st;
    }
    *out = b;
    return WQ_OK;
  }
  std::vector<wq::BatchJob> jobs;
  std::vector<wq::BatchItem> items;
  std::vector<double> cost;
  size_t smem = 0;
  int64_t nnz_total = 0;
  for (int k = 0; k < count; ++k) {
    wq_plan_s* pl = plans[k];
    if (!pl) return set_error(WQ_ERR_INVALID_ARG, "NULL plan in batch");
    if (pl->nurbs_basis) return set_error(WQ_ERR_UNSUPPORTED, "NURBS basis functions are not batched");
    for (int mass = 0; mass < 2; ++mass) {
      void* vals = mass ? (d_mass ? d_mass[k] : nullptr) : (d_stiffness ? d_stiffness[k] : nullptr);
      if (!vals) continue;
      wq::BatchJob J;
      J.p = pl->p;
      J.mass = mass;
      size_t need = mass ? wq::job_args<true>(pl, vals, &J.A) : wq::job_args<false>(pl, vals, &J.A);
      if (need > 227 * 1024) return set_error(WQ_ERR_UNSUPPORTED, "a batch tile does not fit in shared memory");
      smem = std::max(smem, need);
      const int job = (int)jobs.size();
      jobs.push_back(J);
      nnz_total += pl->nnz;
      // per-row work ~ nnz per row x multiply-adds per nonzero (stiffness ~ 3x mass)
      const double b = 2.0 * pl->p + 1.0;
      const double row_cost = b * b * b * (mass ? 1.0 : 3.0) * (4.0 + b);
      wq::TileSplit t1{(int)pl->n[0], pl->p, J.A.T1}, t2{(int)pl->n[1], pl->p, J.A.T2};
      for (int a = 0; a < J.A.nt1; ++a) {
        int a0, a1;
        bool r;
        t1.tile(a, &a0, &a1, &r);
        for (int c = 0; c < J.A.nt2; ++c) {
          int c0, c1;
          t2.tile(c, &c0, &c1, &r);
          for (int i3 = 0; i3 < (int)pl->n[2]; ++i3) {
            items.push_back(wq::BatchItem{job, a, c, i3});
            cost.push_back(row_cost * (a1 - a0) * (c1 - c0));
          }
        }
      }
    }
  }
  if (jobs.empty()) return set_error(WQ_ERR_INVALID_ARG, "the batch has no output arrays");
  // longest first
  std::vector<int> order(items.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
  std::vector<wq::BatchItem> sorted(items.size());
  for (size_t i = 0; i < order.size(); ++i) sorted[i] = items[order[i]];

  wq_batch_s* b = new wq_batch_s();
  cudaGetDevice(&b->device);
  b->n_items = (int)sorted.size();
  b->smem = smem;
  b->nnz_total = nnz_total;
  auto fail = [&](cudaError_t e, const char* what) {
    free_batch(b);
    return wq::cuda_error(e, what);
  };
  cudaError_t e = cudaMalloc(&b->jobs, sizeof(wq::BatchJob) * jobs.size());
  if (e == cudaSuccess) e = cudaMalloc(&b->items, sizeof(wq::BatchItem) * sorted.size());
  if (e == cudaSuccess) e = cudaMalloc(&b->counter, sizeof(unsigned int));
  if (e != cudaSuccess) return fail(e, "batch allocation");
  e = cudaMemcpy(b->jobs, jobs.data(), sizeof(wq::BatchJob) * jobs.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(b->items, sorted.data(), sizeof(wq::BatchItem) * sorted.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return fail(e, "batch upload");
  e = cudaFuncSetAttribute(wq::k_assemble_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return fail(e, "batch kernel attributes");
  int per_sm = 0, sms = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, wq::k_assemble_batch, 256, smem);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
  if (e != cudaSuccess) return fail(e, "batch occupancy");
  b->grid = std::max(1, per_sm) * sms;
  // one graph: reset the work counter, then the persistent kernel
  cudaStream_t cs = nullptr;
  e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) return fail(e, "capture stream");
  e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->counter, 0, sizeof(unsigned int), cs);
  if (e == cudaSuccess) {
    wq::k_assemble_batch<<<b->grid, 256, smem, cs>>>(b->jobs, b->items, b->n_items, b->counter);
    e = cudaGetLastError();
  }
  cudaError_t e2 = cudaStreamEndCapture(cs, &b->graph);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
  cudaStreamDestroy(cs);
  if (e != cudaSuccess) return fail(e, "batch graph capture");
  *out = b;
  return WQ_OK;
}

extern "C" wq_status wq_batch_launch(wq_batch_t batch, void* stream) {
  if (!batch) return set_error(WQ_ERR_INVALID_ARG, "NULL batch");
  WQ_CUDA_TRY(cudaGraphLaunch(batch->exec, (cudaStream_t)stream), "batch graph launch");
  wq::count_launch((int)batch->kernels);
  return WQ_OK;
}

extern "C" wq_status wq_batch_assemble(wq_batch_t batch, void* stream) { return wq_batch_launch(batch, stream); }

extern "C" wq_status wq_batch_info(wq_batch_t batch, int64_t* n_items, int64_t* nnz_total, int* grid) {
  if (!batch) return set_error(WQ_ERR_INVALID_ARG, "NULL batch");
  if (n_items) *n_items = batch->n_items;
  if (nnz_total) *nnz_total = batch->nnz_total;
  if (grid) *grid = batch->grid;
  return WQ_OK;
}

extern "C" wq_status wq_batch_destroy(wq_batch_t batch) {
  free_batch(batch);
  return WQ_OK;
}
