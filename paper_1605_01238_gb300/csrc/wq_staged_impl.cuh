// Staged WQ assembly: the three mode products of Eq. (sumfactorization) as three
// kernels over the whole mesh, with their intermediates in device memory.
//
//   K3  T3[p3][term][q1][q2] = sum_{q3 in Q_i3 n Q_j3} w3^{k3}(i3,q3) B3^{b3}(j3,q3) c_term(q1,q2,q3)
//   K2  G[p3][g][q1][p2]     = sum_{classes of g} sum_{q2 in Q_i2 n Q_j2} B2^{b2}(j2,q2)
//                               sum_{terms of the class} w2^{k2}(i2,q2) T3[p3][term][q1][q2]
//   K1  s(i, j)              = sum_b sum_{q1 in Q_i1 n Q_j1} B1^{b}(j1,q1) sum_a w1^{(a,b)}(i1,q1) G[p3][(a,b)][q1][p2]
//
// with p3 = (i3, j3) and p2 = (i2, j2) running over the 1D band pairs |i - j| <= p
// (prefix sums of the band widths index them). Every output of every stage is
// computed exactly once, so the FP64 work is the halo-free count of the
// factorisation; the price is writing and reading T3 and G once (a few GB at
// p = 4, 64^3), cheap against the FP64 rate. Each stage has a path for regular
// rows (p+1 <= i <= n-p-2: Q_i = [2i-p, 2i+p], the (point, output) pattern known
// at compile time) and a general path for the rows next to the boundary.
//
// Layouts keep every access coalesced: K3 reads a transposed coefficient copy
// cT[slot][q3][q1][q2] and writes T3 with q2 fastest (threads run over q2); K2
// runs over i2 and writes G with the pair index p2 fastest; K1 runs over p2, so
// neighbouring threads write neighbouring j2 blocks of the same CSR row.
//
// Arithmetic (template parameters Real for K3/K2, R1 for K1):
//   FP64        double everywhere;
//   F32X2       f2 (double-float, ~48 bits on the FP32 pipe) everywhere;
//   MIXED       f2 in K3; K2 in f2 for the first and last P+1 rows of direction 2 and
//               for the points q1 that the first and last P+1 rows of direction 1 read,
//               float for the rest; float in K1, whose first and last P+1 rows of
//               direction 1 run in f2 from a double-float copy of G that K2 writes for
//               their points. Near the boundary the WQ weights are large and alternate
//               in sign, so rounding is amplified only in the stages that contract
//               over such rows;
//   FP32        float everywhere.
#pragma once

#include <algorithm>
#include <type_traits>
#include <vector>

#include "wq_internal.h"

namespace wq {

namespace {

__constant__ int sTermL[9] = {0, 0, 0, 1, 1, 1, 2, 2, 2};
__constant__ int sTermM[9] = {0, 1, 2, 0, 1, 2, 0, 1, 2};
// coefficient slot of each term: c_11 c_12 c_13 c_22 c_23 c_33 (c_lm = c_ml)
__constant__ int sSlot[9] = {0, 1, 2, 1, 3, 4, 2, 4, 5};
__constant__ int sSlotTerms[6][2] = {{0, -1}, {1, 3}, {2, 6}, {4, -1}, {5, 7}, {8, -1}};  // terms of each slot

// Stage-2 classes of equal (group, b2), terms ordered as sTerm*:
// class 0: (0,0) g3 b0; 1: (0,1) g2 b1; 2: (0,2) g2 b0; 3: (1,0),(2,0) g1 b0;
// 4: (1,1),(2,1) g0 b1; 5: (1,2),(2,2) g0 b0. Classes come grouped by G group
// (g3 | g2 g2 | g1 | g0 g0): one group's accumulators are live at a time, zeroed
// at its first class and stored after its last.
struct ClassInfo {
  int term[2], g, b2;
  bool first, last;
};
__constant__ ClassInfo sClass[6] = {{{0, -1}, 3, 0, true, true},  {{1, -1}, 2, 1, true, false},
                                    {{2, -1}, 2, 0, false, true}, {{3, 6}, 1, 0, true, true},
                                    {{4, 7}, 0, 1, true, false},  {{5, 8}, 0, 0, false, true}};

// Class c: from compile-time tables when the class loop is unrolled (c folds to a
// constant), from constant memory when it is rolled (double-float, whose ~15
// instructions per multiply-add would otherwise overflow the instruction cache).
template <bool ROLL>
__device__ __forceinline__ ClassInfo class_info(int c) {
  if (ROLL) return sClass[c];
  constexpr int terms[6][2] = {{0, -1}, {1, -1}, {2, -1}, {3, 6}, {4, 7}, {5, 8}};
  constexpr int group[6] = {3, 2, 2, 1, 0, 0};
  constexpr int b2[6] = {0, 1, 0, 0, 1, 0};
  constexpr bool first[6] = {true, true, false, true, true, false};
  constexpr bool last[6] = {true, false, true, true, false, true};
  return ClassInfo{{terms[c][0], terms[c][1]}, group[c], b2[c], first[c], last[c]};
}

// Double-float numbers (WQ_PREC_F32X2): value = hi + lo with |lo| <= ulp(hi)/2,
// about 48 significant bits carried on the FP32 pipe, which GB300 runs at ~60x
// its FP64 rate. Arithmetic by the error-free transformations of Knuth (two-sum)
// and Dekker (two-product, here in its FMA form), renormalised by the fast
// two-sum; the _rn intrinsics keep the compiler from contracting them.
struct f2 {
  float hi, lo;
};

__device__ __forceinline__ f2 f2_renorm(float s, float t) {  // fast two-sum, |s| >= |t|
  const float hi = __fadd_rn(s, t);
  return f2{hi, __fsub_rn(t, __fsub_rn(hi, s))};
}

// a * b + c
__device__ __forceinline__ f2 f2_fma(f2 a, f2 b, f2 c) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);                         // a.hi b.hi = p + e exactly
  e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));         // cross terms (a.lo b.lo < 2^-46 |ab|)
  const float s = __fadd_rn(p, c.hi);                          // two-sum of p and c.hi
  const float v = __fsub_rn(s, p);
  float t = __fadd_rn(__fsub_rn(p, __fsub_rn(s, v)), __fsub_rn(c.hi, v));
  t = __fadd_rn(t, __fadd_rn(e, c.lo));
  return f2_renorm(s, t);
}

__device__ __forceinline__ f2 f2_mul(f2 a, f2 b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
  return f2_renorm(p, e);
}

__device__ __forceinline__ f2 f2_from(double x) {
  const float hi = __double2float_rn(x);
  return f2{hi, __double2float_rn(x - (double)hi)};
}

// Arithmetic of the contractions: Real = double, float or f2.
template <typename T>
__device__ __forceinline__ T fmaR(T a, T b, T c);
template <>
__device__ __forceinline__ double fmaR<double>(double a, double b, double c) { return fma(a, b, c); }
template <>
__device__ __forceinline__ float fmaR<float>(float a, float b, float c) { return fmaf(a, b, c); }
template <>
__device__ __forceinline__ f2 fmaR<f2>(f2 a, f2 b, f2 c) { return f2_fma(a, b, c); }

template <typename T>
__device__ __forceinline__ T mulR(T a, T b) { return a * b; }
template <>
__device__ __forceinline__ f2 mulR<f2>(f2 a, f2 b) { return f2_mul(a, b); }

template <typename T>
__device__ __forceinline__ T zeroR() { return (T)0; }
template <>
__device__ __forceinline__ f2 zeroR<f2>() { return f2{0.0f, 0.0f}; }

template <typename T>
__device__ __forceinline__ T fromD(double x) { return (T)x; }
template <>
__device__ __forceinline__ f2 fromD<f2>(double x) { return f2_from(x); }

// float -> double by re-packing the IEEE-754 fields (exact; integer instructions
// instead of a conversion on the FP64 pipe). Float subnormals (below 1.2e-38)
// become zero, far below the values' rounding.
__device__ __forceinline__ double f2d_exact(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xffu, sign = u & 0x80000000u, m = u & 0x7fffffu;
  if (e == 0u) return __hiloint2double((int)sign, 0);
  const unsigned de = e == 0xffu ? 0x7ffu : e + 896u;
  return __hiloint2double((int)(sign | (de << 20) | (m >> 3)), (int)(m << 29));
}

template <typename T>
__device__ __forceinline__ double toD(T x) { return (double)x; }
template <>
__device__ __forceinline__ double toD<f2>(f2 x) { return f2d_exact(x.hi) + f2d_exact(x.lo); }

// value in an output / intermediate type O
template <typename O, typename T>
__device__ __forceinline__ O toOut(T x) { return (O)x; }
template <>
__device__ __forceinline__ double toOut<double, f2>(f2 x) { return toD(x); }
template <>
__device__ __forceinline__ float toOut<float, f2>(f2 x) { return __fadd_rn(x.hi, x.lo); }
template <>
__device__ __forceinline__ f2 toOut<f2, f2>(f2 x) { return x; }
template <>
__device__ __forceinline__ f2 toOut<f2, float>(float x) { return f2{x, 0.0f}; }
template <>
__device__ __forceinline__ f2 toOut<f2, double>(double x) { return f2_from(x); }

// an intermediate stored as S, read into arithmetic type T (double-float T3 read by
// the FP32 part of stage 2 is rounded to the nearest float)
template <typename T, typename S>
__device__ __forceinline__ T fromStore(S x) { return (T)x; }
template <>
__device__ __forceinline__ float fromStore<float, f2>(f2 x) { return __fadd_rn(x.hi, x.lo); }
template <>
__device__ __forceinline__ f2 fromStore<f2, f2>(f2 x) { return x; }

// read of a volatile shared-memory value
template <typename T>
__device__ __forceinline__ T vld(const volatile T* p) { return *p; }
template <>
__device__ __forceinline__ f2 vld<f2>(const volatile f2* p) { return f2{p->hi, p->lo}; }

__device__ __forceinline__ int blo(int i, int p) { return i - p > 0 ? i - p : 0; }
__device__ __forceinline__ int bw(int i, int p, int n) { return min(n - 1, i + p) - blo(i, p) + 1; }

// Tables and coefficients come in the arithmetic type of the contractions (the
// FP32 path reads float copies made once per call), so no conversion sits in
// the inner loops.
struct Dir {
  int n, nqp;
  const int* q0;
  const int* nq;
  const void* w;          // Real [4][n][NQ]
  const void* bt;         // Real [2][n][NQ]
  const int64_t* prefix;  // [n+1]
  const int* pair_row;    // [nnz1]: i of each band pair
};

struct StagedArgs {
  Dir d[3];
  int NQ;
  int64_t nnz1[3];
  const void* cT;         // Real [7][nqp3][nqp1][nqp2]
  const void* kappaT;     // NULL or Real [nqp3][nqp1][nqp2]
  void* T3;               // Real [nnz1_3][NT][nqp1][t3w]: rows of nqp2 values padded to even t3w
  int t3w;
  void* G;                // Real [nnz1_3][NG][nqp1][nnz1_2]
  void* vals;
  // Mixed precision only: a copy of G in the edge-row type GE (double-float) at the
  // q1 points that the first and last P+1 rows of direction 1 read (q1 < nbl and
  // q1 >= hstart), and the direction-1 tables in that type, so that stage 1 runs
  // those rows in it.
  void* Gb;               // NULL or [nnz1_3][NG][nbq][nnz1_2] in the edge-row type GE
  const void* w1e;        // [4][n1][NQ]: direction-1 rules in the edge-row type
  const void* bt1e;       // [2][n1][NQ]
  int nbl, hstart, nbq;
  // the same point ranges of direction 2 (the q2 that its first and last P+1 rows read)
  int nbl2, hstart2;
  // Slab of direction 3: rows i3 in [i3_off, i3_off + n3 of the launch), band pairs
  // p3 in [p3_off, ...); T3, G and Gb hold the slab only (index p3 - p3_off).
  int64_t p3_off;
  int i3_off;
};

// position of point q1 in the edge copy of G (in range for every q1 that a
// first or last P+1 row of direction 1 reads; clamped for any other q1)
__device__ __forceinline__ int edge_row(int q1, int nbl, int hstart, int nbq) {
  return q1 < nbl ? q1 : min(nbq - 1, max(nbl, q1 - hstart + nbl));
}

template <typename Real>
__device__ __forceinline__ const Real* tab(const void* p) { return reinterpret_cast<const Real*>(p); }

// two consecutive values of an array (p at an even index of a 16-byte aligned
// array), in one vector load
template <typename T>
__device__ __forceinline__ void ld2(const T* p, T& a, T& b);
template <>
__device__ __forceinline__ void ld2<float>(const float* p, float& a, float& b) {
  const float2 v = __ldg(reinterpret_cast<const float2*>(p));
  a = v.x;
  b = v.y;
}
template <>
__device__ __forceinline__ void ld2<double>(const double* p, double& a, double& b) {
  const double2 v = __ldg(reinterpret_cast<const double2*>(p));
  a = v.x;
  b = v.y;
}

// Loads of data that no kernel of the launch writes (tables, T3 in stage 2, G in
// stage 1) go through the read-only path, so the compiler may move them across
// the kernel's own stores.
template <typename T>
__device__ __forceinline__ T ro(const T* p) { return __ldg(p); }
template <>
__device__ __forceinline__ f2 ro<f2>(const f2* p) {
  const float2 v = __ldg(reinterpret_cast<const float2*>(p));
  return f2{v.x, v.y};
}
template <>
__device__ __forceinline__ void ld2<f2>(const f2* p, f2& a, f2& b) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(p));
  a = f2{v.x, v.y};
  b = f2{v.z, v.w};
}

__global__ void k_to_float(const double* __restrict__ in, float* __restrict__ out, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = (float)in[i];
}

__global__ void k_to_f2(const double* __restrict__ in, f2* __restrict__ out, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = f2_from(in[i]);
}

// (q1, q2, q3) -> (q3, q1, q2) copy of the coefficient planes (and kappa)
template <typename Real>
__global__ void k_transpose_coef(const double* __restrict__ c, const double* __restrict__ kappa,
                                 Real* __restrict__ cT, Real* __restrict__ kT, int nq1, int nq2, int nq3,
                                 int nplanes) {
  __shared__ Real tile[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;  // q1, q2 tile
  const int plane = blockIdx.z;                          // slot * nq3 + q3
  const int slot = plane / nq3;
  const double* src = slot < nplanes ? c + (int64_t)plane * nq1 * nq2 : kappa + (int64_t)(plane - nplanes * nq3) * nq1 * nq2;
  Real* dst = slot < nplanes ? cT + (int64_t)plane * nq1 * nq2 : kT + (int64_t)(plane - nplanes * nq3) * nq1 * nq2;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int q2 = by + k, q1 = bx + threadIdx.x;
    if (q1 < nq1 && q2 < nq2) tile[k][threadIdx.x] = fromD<Real>(src[(int64_t)q2 * nq1 + q1]);
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int q1 = bx + k, q2 = by + threadIdx.x;
    if (q1 < nq1 && q2 < nq2) dst[(int64_t)q1 * nq2 + q2] = tile[threadIdx.x][k];
  }
}

// K3 on a regular row i3 (Q_i3 holds 2P+1 points; the overlap with Q_j3, jj = j3 -
// i3 + P, is t in [2 jj - 2P, 2 jj], known at compile time, so c stays in registers),
// in arithmetic T on tables and coefficients stored as Real.
template <int P, bool MASS, typename T, typename Real>
__device__ __forceinline__ void stage3_regular(const StagedArgs& A, const Real* a3, Real* T3, int i3, int q1, int q2,
                                               int64_t p3base) {
  constexpr int MAXQ = 4 * P + 1;
  constexpr int NT = MASS ? 1 : 9;
  constexpr int BW = 2 * P + 1;
  const Dir& D3 = A.d[2];
  const int nq1 = A.d[0].nqp, nq2 = A.d[1].nqp;
  const int qi3 = D3.q0[i3];
  const int64_t plane = (int64_t)nq1 * nq2;
  const int64_t pt = (int64_t)q1 * nq2 + q2;
  const int64_t tplane = (int64_t)nq1 * A.t3w;
  const int nslots = MASS ? 1 : 6;
#pragma unroll 1
  for (int s = 0; s < nslots; ++s) {
    const int slot = MASS ? 6 : s;
    const Real* cs = tab<Real>(A.cT) + ((int64_t)slot * D3.nqp + qi3) * plane + pt;
    const Real* ks = A.kappaT ? tab<Real>(A.kappaT) + (int64_t)qi3 * plane + pt : nullptr;
    T c[BW];
#pragma unroll
    for (int t = 0; t < BW; ++t)
      c[t] = ks ? mulR(fromStore<T>(ro(cs + t * plane)), fromStore<T>(ro(ks + t * plane))) : fromStore<T>(ro(cs + t * plane));
    for (int k = 0; k < (MASS ? 1 : 2); ++k) {
      const int term = MASS ? 0 : sSlotTerms[s][k];
      if (term < 0) break;
      const int l = MASS ? 0 : sTermL[term], m = MASS ? 0 : sTermM[term];
      const int k3 = MASS ? 0 : 2 * (l == 2) + (m == 2);
      Real* dst = T3 + ((p3base * NT + term) * nq1 + q1) * (int64_t)A.t3w + q2;
#pragma unroll
      for (int jj = 0; jj < BW; ++jj) {
        const Real* a = a3 + (k3 * BW + jj) * MAXQ;
        T acc = zeroR<T>();
#pragma unroll
        for (int t = (2 * jj - 2 * P > 0 ? 2 * jj - 2 * P : 0); t <= (2 * jj < 2 * P ? 2 * jj : 2 * P); ++t)
          acc = fmaR<T>(fromStore<T>(a[t]), c[t], acc);
        dst[(int64_t)jj * NT * tplane] = toOut<Real>(acc);
      }
    }
  }
}

// K3: one thread per (q2, q1, i3); all terms and all j3 of the band. Blocks with
// consecutive i3 (blockIdx.x) read overlapping coefficient planes back to back.
template <int P, bool MASS, typename Real, bool SEL = false>
__global__ void __launch_bounds__(128) k_stage3(StagedArgs A) {
  constexpr int MAXQ = 4 * P + 1;
  constexpr int NT = MASS ? 1 : 9;
  constexpr int BW = 2 * P + 1;
  const Dir& D3 = A.d[2];
  const int nq1 = A.d[0].nqp, nq2 = A.d[1].nqp;
  const int i3 = A.i3_off + blockIdx.x;
  const int64_t e = blockIdx.y * (int64_t)blockDim.x + threadIdx.x;  // point index q1 * nq2 + q2
  const int q1 = (int)(e / nq2), q2 = (int)(e % nq2);
  const int NQ = A.NQ;
  const int qi3 = D3.q0[i3], ni3 = D3.nq[i3];
  const int jlo = blo(i3, P), jhi = min(D3.n - 1, i3 + P);
  // a3[k][jj][t] = w3^{k}(i3, qi3 + t) B3^{k & 1}(j3, qi3 + t) on the overlap [lo, hi) of Q_i3 and Q_j3
  __shared__ Real a3[4][BW][MAXQ];
  __shared__ int olo[BW], ohi[BW];
  for (int e = threadIdx.x; e < 4 * BW * MAXQ; e += blockDim.x) {
    const int t = e % MAXQ, jj = (e / MAXQ) % BW, k = e / (MAXQ * BW);
    const int j3 = jlo + jj;
    double v = 0.0;
    if (j3 <= jhi && t < ni3) {
      const int loc = qi3 + t - D3.q0[j3];
      if (loc >= 0 && loc < D3.nq[j3])
        v = toD(tab<Real>(D3.w)[((size_t)k * D3.n + i3) * NQ + t]) *
            toD(tab<Real>(D3.bt)[((size_t)(k & 1) * D3.n + j3) * NQ + loc]);
    }
    a3[k][jj][t] = fromD<Real>(v);
  }
  for (int jj = threadIdx.x; jj < BW; jj += blockDim.x) {
    const int j3 = jlo + jj;
    if (j3 <= jhi) {
      const int qj = D3.q0[j3];
      olo[jj] = max(qi3, qj) - qi3;
      ohi[jj] = min(qi3 + ni3, qj + D3.nq[j3]) - qi3;
    }
  }
  __syncthreads();
  if (q1 >= nq1) return;
  const int64_t plane = (int64_t)nq1 * nq2;
  const int64_t pt = (int64_t)q1 * nq2 + q2;
  const int64_t p3base = D3.prefix[i3] - A.p3_off;  // slab-relative
  Real* T3 = reinterpret_cast<Real*>(A.T3);
  const int nslots = MASS ? 1 : 6;
  if (!std::is_same<Real, double>::value && i3 >= P + 1 && i3 <= D3.n - P - 2) {
    // regular row (FP64 stays on the loop below: the FP64 pipe bounds it either way,
    // and it measured 10% faster at p = 8). SEL (the mixed modes): double-float only
    // at the points whose T3 value a first or last P+1 row of direction 1 or 2 reads
    // later (there the large boundary weights amplify its rounding), FP32 elsewhere
    if (SEL && !(q1 < A.nbl || q1 >= A.hstart || q2 < A.nbl2 || q2 >= A.hstart2))
      stage3_regular<P, MASS, float, Real>(A, &a3[0][0][0], T3, i3, q1, q2, p3base);
    else
      stage3_regular<P, MASS, Real, Real>(A, &a3[0][0][0], T3, i3, q1, q2, p3base);
    return;
  }
  for (int s = 0; s < nslots; ++s) {
    const int slot = MASS ? 6 : s;
    Real c[MAXQ];
    const Real* cs = tab<Real>(A.cT) + ((int64_t)slot * D3.nqp + qi3) * plane + pt;
    const Real* ks = A.kappaT ? tab<Real>(A.kappaT) + (int64_t)qi3 * plane + pt : nullptr;
    for (int t = 0; t < ni3; ++t) c[t] = ks ? mulR(cs[t * plane], ks[t * plane]) : cs[t * plane];
    for (int term = 0; term < NT; ++term) {
      if (!MASS && sSlot[term] != s) continue;
      const int l = MASS ? 0 : sTermL[term], m = MASS ? 0 : sTermM[term];
      const int k3 = MASS ? 0 : 2 * (l == 2) + (m == 2);
      for (int jj = 0; jj <= jhi - jlo; ++jj) {
        const Real* a = a3[k3][jj];
        Real acc = zeroR<Real>();
        for (int t = olo[jj]; t < ohi[jj]; ++t) acc = fmaR<Real>(a[t], c[t], acc);
        T3[(((p3base + jj) * NT + term) * nq1 + q1) * (int64_t)A.t3w + q2] = acc;
      }
    }
  }
}

// K2: one thread per (i2, q1, p3). Regular rows of direction 2 use a compile-time
// (t, j2) pattern; rows next to the boundary loop over the support overlaps.
// Regular rows: threads run over (i2 in [r_lo, r_hi), then q1), neighbouring
// threads sharing q2 points. Boundary rows [0, r_lo) and [r_hi, n2): threads run
// over (the row, then q1), so every lane has work and the rows of one side read
// neighbouring q2 and write neighbouring band pairs.
template <int P, bool MASS, typename Real, bool REG, typename GOut, typename GE = Real>
__global__ void __launch_bounds__(128) k_stage2(StagedArgs A, int r_lo, int r_hi) {
  constexpr int BW = 2 * P + 1;
  constexpr int NT = MASS ? 1 : 9;
  constexpr int NG = MASS ? 1 : 4;
  constexpr int NC = MASS ? 1 : 6;
  constexpr int MAXQ = 4 * P + 1;
  constexpr bool ROLL = std::is_same<Real, f2>::value;
  constexpr int CU = ROLL ? 1 : NC;
  const Dir& D2 = A.d[1];
  const int nq1 = A.d[0].nqp, NQ = A.NQ;
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t p3 = blockIdx.y;
  int i2, q1;
  if (REG) {
    const int nreg = r_hi - r_lo;
    if (e >= (int64_t)nreg * nq1) return;
    i2 = r_lo + (int)(e % nreg);
    q1 = (int)(e / nreg);
  } else {
    const int nb = r_lo + (D2.n - r_hi);
    if (e >= (int64_t)nb * nq1) return;
    const int b = (int)(e % nb);
    q1 = (int)(e / nb);
    i2 = b < r_lo ? b : r_hi + (b - r_lo);
  }
  const int64_t nnz2 = A.nnz1[1];
  const Real* T3 = reinterpret_cast<const Real*>(A.T3) + ((p3 * NT) * nq1 + q1) * (int64_t)A.t3w;
  const int64_t tstride = (int64_t)nq1 * A.t3w;
  const int qi = D2.q0[i2], ni = REG ? BW : D2.nq[i2];
  const int jlo = blo(i2, P), jhi = min(D2.n - 1, i2 + P);
  const int64_t pbase = D2.prefix[i2];
  // classes come grouped by G group (g3 | g2 g2 | g1 | g0 g0): one group's
  // accumulators are live at a time, zeroed at its first class, stored after its last
  Real acc[BW];
#pragma unroll(CU)
  for (int c = 0; c < NC; ++c) {
    const ClassInfo ci = class_info<ROLL>(c);
    if (MASS || ci.first)
#pragma unroll
      for (int tt = 0; tt < BW; ++tt) acc[tt] = zeroR<Real>();
    Real h[REG ? BW : MAXQ];
#pragma unroll
    for (int t = 0; t < (REG ? BW : MAXQ); ++t) h[t] = zeroR<Real>();
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int term = MASS ? 0 : ci.term[k];
      if (term < 0 || (MASS && k > 0)) continue;
      const int l = MASS ? 0 : term / 3, m = MASS ? 0 : term % 3;
      const int k2 = MASS ? 0 : 2 * (l == 1) + (m == 1);
      const Real* wrow = tab<Real>(D2.w) + ((size_t)k2 * D2.n + i2) * NQ;
      const Real* trow = T3 + term * tstride + qi;
      if (REG) {
#pragma unroll
        for (int t = 0; t < BW; ++t) h[t] = fmaR<Real>(ro(wrow + t), ro(trow + t), h[t]);
      } else {
        for (int t = 0; t < ni; ++t) h[t] = fmaR<Real>(ro(wrow + t), ro(trow + t), h[t]);
      }
    }
    const int g = MASS ? 0 : ci.g;
    const int b2 = MASS ? 0 : ci.b2;
    if (REG) {
#pragma unroll
      for (int tt = 0; tt < BW; ++tt) {
        const int j2 = i2 - P + tt;
        const Real* brow = tab<Real>(D2.bt) + ((size_t)b2 * D2.n + j2) * NQ + (qi - D2.q0[j2]);
#pragma unroll
        for (int t = 0; t < BW; ++t)
          if (t >= 2 * tt - 2 * P && t <= 2 * tt) acc[tt] = fmaR<Real>(ro(brow + t), h[t], acc[tt]);
      }
    } else {
#pragma unroll
      for (int tt = 0; tt < BW; ++tt) {
        const int j2 = i2 - P + tt;
        if (j2 < jlo || j2 > jhi) continue;
        const int qj = D2.q0[j2];
        const int lo = max(qi, qj), hi = min(qi + ni, qj + D2.nq[j2]);
        const Real* brow = tab<Real>(D2.bt) + ((size_t)b2 * D2.n + j2) * NQ;
        for (int q = lo; q < hi; ++q) acc[tt] = fmaR<Real>(ro(brow + (q - qj)), h[q - qi], acc[tt]);
      }
    }
    if (MASS || ci.last) {
      GOut* dst = reinterpret_cast<GOut*>(A.G) + ((p3 * NG + g) * nq1 + q1) * nnz2 + pbase;
#pragma unroll
      for (int tt = 0; tt < BW; ++tt) {
        const int j2 = i2 - P + tt;
        if (REG || (j2 >= jlo && j2 <= jhi)) dst[j2 - jlo] = toOut<GOut>(acc[tt]);
      }
      if (sizeof(GOut) < sizeof(Real) && A.Gb && (q1 < A.nbl || q1 >= A.hstart)) {
        GE* dd = reinterpret_cast<GE*>(A.Gb) + ((p3 * NG + g) * A.nbq + edge_row(q1, A.nbl, A.hstart, A.nbq)) * nnz2 + pbase;
#pragma unroll
        for (int tt = 0; tt < BW; ++tt) {
          const int j2 = i2 - P + tt;
          if (REG || (j2 >= jlo && j2 <= jhi)) dd[j2 - jlo] = toOut<GE>(acc[tt]);
        }
      }
    }
  }
}

// Stage 1 for a first or last P+1 row of direction 1: Q_i1 is not the regular
// 2P+1 window and the band is clipped. G points at (p3, group 0, row 0, p2);
// MAPQ maps q1 into the edge copy. out + base + j1 is the value of column j1.
template <int P, bool MASS, typename T, typename OutT, bool MAPQ>
__device__ __forceinline__ void stage1_edge(const T* G, int64_t gstride, int64_t nnz2, const T* w, int64_t wk,
                                            const T* bt1, int64_t bder, const Dir& D1, int i1, int n1, int NQ,
                                            int nbl, int hstart, int nbq, OutT* out, int64_t base) {
  constexpr int BW = 2 * P + 1;
  constexpr int MAXQ = 4 * P + 1;
  const int qi1 = D1.q0[i1], ni1 = D1.nq[i1];
  T h0[MAXQ], h1[MAXQ];
  for (int t = 0; t < ni1; ++t) {
    const int qr = MAPQ ? edge_row(qi1 + t, nbl, hstart, nbq) : qi1 + t;
    const T* gq = G + (int64_t)qr * nnz2;
    if (MASS) {
      h0[t] = mulR(w[t], gq[0]);
    } else {
      h0[t] = fmaR<T>(w[t], gq[0], mulR(w[t + 2 * wk], gq[2 * gstride]));
      h1[t] = fmaR<T>(w[t + wk], gq[gstride], mulR(w[t + 3 * wk], gq[3 * gstride]));
    }
  }
#pragma unroll
  for (int tt = 0; tt < BW; ++tt) {
    const int j1 = i1 - P + tt;
    if (j1 < 0 || j1 >= n1) continue;
    const int qj = D1.q0[j1];
    const int lo = max(qi1, qj), hi = min(qi1 + ni1, qj + D1.nq[j1]);
    const int64_t brow = (int64_t)j1 * NQ - qj;
    T v = zeroR<T>();
    for (int q = lo; q < hi; ++q) {
      if (MASS)
        v = fmaR<T>(bt1[brow + q], h0[q - qi1], v);
      else
        v = fmaR<T>(bt1[brow + q + bder], h1[q - qi1], fmaR<T>(bt1[brow + q], h0[q - qi1], v));
    }
    out[base + j1] = toOut<OutT>(v);
  }
}

// K2 on the regular rows of direction 2 (Q_i2 = [2 i2 - P, 2 i2 + P]), with the
// rule and B-spline tables of the block's rows in shared memory: lanes run over
// 32 consecutive rows i2 (so the T3 reads of a warp are contiguous), the four
// warps over pairs of q1 in [q_lo, q_hi), and the tables are read from shared memory
// instead of one cache line per lane. Bs holds B_j2 of the trial rows i0-P .. i0+31+P
// aligned to the regular pattern: Bs[b][j2 - i0 + P][u] is B^(b)_j2 at point 2 j2 - P + u.
// TIn is the stored type of T3 (the mixed mode runs this kernel in FP32 on double-float
// T3 for the points q1 that no first or last P+1 row of direction 1 reads).
// Double-float up to P = 6 is held to 128 registers (4 blocks per SM; a few dozen bytes
// of spills): 168 registers gave 3 (p = 5, 128^3: mixed 22.04 -> 21.92 ms, f32x2 81.6 ->
// 79.6 ms); at P = 8 the cap spilled ~0.5 KB per thread.
template <int P, bool MASS, typename Real, typename GOut, typename TIn = Real, typename GE = Real>
__global__ void __launch_bounds__(128, std::is_same<Real, f2>::value && P <= 6 ? 4 : 0)
    k_stage2_reg(StagedArgs A, int r_lo, int r_hi, int q_lo, int q_hi) {
  constexpr int BW = 2 * P + 1;
  constexpr int NT = MASS ? 1 : 9;
  constexpr int NG = MASS ? 1 : 4;
  constexpr int NC = MASS ? 1 : 6;
  constexpr int NK = MASS ? 1 : 4;   // rule kinds
  constexpr int NB = MASS ? 1 : 2;   // trial kinds
  constexpr int RW = 32;             // rows per block
  constexpr int NJS = RW + 2 * P;    // trial rows per block
  constexpr bool ROLL = std::is_same<Real, f2>::value;
  constexpr int CU = ROLL ? 1 : NC;
  __shared__ Real Ws[NK][RW][BW];
  __shared__ Real Bs[NB][NJS][BW];
  __shared__ GOut stg[4][RW * BW];   // per warp: its 32 rows x BW values of one G row
  const Dir& D2 = A.d[1];
  const int nq1 = A.d[0].nqp, NQ = A.NQ, n2 = D2.n;
  const int i0 = r_lo + blockIdx.x * RW;
  const int64_t p3 = blockIdx.y;
  const int lane = threadIdx.x, warp = threadIdx.y, tid = warp * 32 + lane;
  for (int e = tid; e < NK * RW * BW; e += 128) {
    const int t = e % BW, r = (e / BW) % RW, k = e / (BW * RW);
    const int i2 = i0 + r;
    Ws[k][r][t] = i2 < r_hi ? ro(tab<Real>(D2.w) + ((size_t)k * n2 + i2) * NQ + t) : zeroR<Real>();
  }
  for (int e = tid; e < NB * NJS * BW; e += 128) {
    const int u = e % BW, jr = (e / BW) % NJS, b = e / (BW * NJS);
    const int j2 = i0 - P + jr;
    Real v = zeroR<Real>();
    if (j2 >= 0 && j2 < n2) {
      const int idx = u + 2 * j2 - P - D2.q0[j2];
      if (idx >= 0 && idx < D2.nq[j2]) v = ro(tab<Real>(D2.bt) + ((size_t)b * n2 + j2) * NQ + idx);
    }
    Bs[b][jr][u] = v;
  }
  __syncthreads();
  // lanes past r_hi compute on row r_hi - 1 and store nothing
  const bool act = i0 + lane < r_hi;
  const int i2 = act ? i0 + lane : r_hi - 1;
  const int nval = min(RW, r_hi - i0) * BW;  // values of the warp's rows in one G row
  const int64_t nnz2 = A.nnz1[1];
  const int64_t pbase = D2.prefix[i2];
  const int64_t pbase0 = D2.prefix[i0];     // regular rows: pbase = pbase0 + lane * BW
  const int64_t tstride = (int64_t)nq1 * A.t3w;
  // the row's window q2 in [2 i2 - P, 2 i2 + P] is read as NV pairs from the even
  // index 2 i2 - P - O (rows of T3 have even length): value t is entry t + O
  constexpr int O = P & 1, NV = (BW + O + 1) / 2;
  const TIn* T3p = reinterpret_cast<const TIn*>(A.T3) + (p3 * NT) * tstride + (2 * i2 - P - O);
  GOut* sb = stg[warp];
  // volatile views: the compiler would otherwise hoist all of the row's table
  // values out of the q1 loop into registers and spill
  const volatile Real* Wv = &Ws[0][lane][0];
  const volatile Real* Bv = &Bs[0][lane][0];
  // NQB q1 points per iteration: every shared-memory value feeds NQB FMA chains (4
  // measured no faster in FP32: the registers it takes cost occupancy)
  constexpr int NQB = 2;
#pragma unroll 1
  for (int qa = q_lo + NQB * warp; qa < q_hi; qa += 4 * NQB) {
    const TIn* Tq[NQB];
#pragma unroll
    for (int v = 0; v < NQB; ++v) Tq[v] = T3p + (int64_t)min(qa + v, q_hi - 1) * A.t3w;  // the last may repeat
    Real acc[NQB][BW];
#pragma unroll(CU)
    for (int c = 0; c < NC; ++c) {
      const ClassInfo ci = class_info<ROLL>(c);
      if (MASS || ci.first)
#pragma unroll
        for (int tt = 0; tt < BW; ++tt)
#pragma unroll
          for (int v = 0; v < NQB; ++v) acc[v][tt] = zeroR<Real>();
      Real h[NQB][BW];
#pragma unroll
      for (int t = 0; t < BW; ++t)
#pragma unroll
        for (int v = 0; v < NQB; ++v) h[v][t] = zeroR<Real>();
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const int term = MASS ? 0 : ci.term[k];
        if (term < 0 || (MASS && k > 0)) continue;
        const int l = MASS ? 0 : term / 3, m = MASS ? 0 : term % 3;
        const int k2 = MASS ? 0 : 2 * (l == 1) + (m == 1);
#pragma unroll
        for (int pv = 0; pv < NV; ++pv) {
          TIn a[NQB][2];
#pragma unroll
          for (int v = 0; v < NQB; ++v) ld2(Tq[v] + term * tstride + 2 * pv, a[v][0], a[v][1]);
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const int t = 2 * pv + u - O;
            if (t >= 0 && t < BW) {
              const Real wv = vld(Wv + k2 * RW * BW + t);
#pragma unroll
              for (int v = 0; v < NQB; ++v) h[v][t] = fmaR<Real>(wv, fromStore<Real>(a[v][u]), h[v][t]);
            }
          }
        }
      }
      const int g = MASS ? 0 : ci.g;
      const int b2 = MASS ? 0 : ci.b2;
#pragma unroll
      for (int tt = 0; tt < BW; ++tt)
#pragma unroll
        for (int t = 0; t < BW; ++t)
          if (t >= 2 * tt - 2 * P && t <= 2 * tt) {
            const Real bv = vld(Bv + (b2 * NJS + tt) * BW + t - 2 * tt + 2 * P);
#pragma unroll
            for (int v = 0; v < NQB; ++v) acc[v][tt] = fmaR<Real>(bv, h[v][t], acc[v][tt]);
          }
      if (MASS || ci.last) {
#pragma unroll
        for (int v = 0; v < NQB; ++v) {
          const int q1 = qa + v;
          if (q1 >= q_hi) break;
          // the warp's values of this G row are contiguous (pbase0 + lane * BW + tt):
          // through shared memory, so that each store of the warp is 32 consecutive values
          __syncwarp();
#pragma unroll
          for (int tt = 0; tt < BW; ++tt) sb[lane * BW + tt] = toOut<GOut>(acc[v][tt]);
          __syncwarp();
          GOut* dst = reinterpret_cast<GOut*>(A.G) + ((p3 * NG + g) * nq1 + q1) * nnz2 + pbase0;
#pragma unroll
          for (int k = 0; k < BW; ++k)
            if (lane + 32 * k < nval) dst[lane + 32 * k] = sb[lane + 32 * k];
          if (sizeof(GOut) < sizeof(Real) && A.Gb && act && (q1 < A.nbl || q1 >= A.hstart)) {
            GE* dd = reinterpret_cast<GE*>(A.Gb) + ((p3 * NG + g) * A.nbq + edge_row(q1, A.nbl, A.hstart, A.nbq)) * nnz2 + pbase;
#pragma unroll
            for (int tt = 0; tt < BW; ++tt) dd[tt] = toOut<GE>(acc[v][tt]);
          }
        }
      }
    }
  }
}

// Compile-time point patterns of the first and last P+1 rows of a direction
// (valid when the direction has n_el >= 2P+2 spans, so that the two ends do not
// meet). Row R from the low end (H = false) or the high end (H = true) has
// NI = 2R+P+1 points and NJ = R+P+1 band members j = jlo + jj; the overlap of Q_i
// and Q_j is t in [e_tlo, e_thi) relative to the first point of Q_i, and
// B_j at that point is entry t + e_toff of its table row.
__host__ __device__ constexpr int e_ni(int P, int R) { return 2 * R + P + 1; }
__host__ __device__ constexpr int e_nj(int P, int R) { return R + P + 1; }
__host__ __device__ constexpr int e_s(int P, int R, int jj) { return R + P - jj; }
__host__ __device__ constexpr int e_tlo(int P, int R, bool H, int jj) {
  return !H ? (jj <= P ? 0 : 2 * jj - P)
            : (e_ni(P, R) - 2 * e_s(P, R, jj) - P - 1 > 0 ? e_ni(P, R) - 2 * e_s(P, R, jj) - P - 1 : 0);
}
__host__ __device__ constexpr int e_thi(int P, int R, bool H, int jj) {
  return !H ? (2 * jj + P + 1 < e_ni(P, R) ? 2 * jj + P + 1 : e_ni(P, R))
            : e_ni(P, R) - (e_s(P, R, jj) <= P ? 0 : 2 * e_s(P, R, jj) - P);
}
__host__ __device__ constexpr int e_toff(int P, int R, bool H, int jj) {
  return !H ? -(jj <= P ? 0 : 2 * jj - P) : -e_ni(P, R) + 2 * e_s(P, R, jj) + P + 1;
}

// Stage 2 for edge row R of direction 2 (i2 = R or n2-1-R) at point q1 of pair p3.
template <int P, bool MASS, typename Real, typename GOut, int R, bool H, typename GE>
__device__ __forceinline__ void stage2_edge_row(const StagedArgs& A, int q1, int64_t p3) {
  constexpr int NT = MASS ? 1 : 9;
  constexpr int NG = MASS ? 1 : 4;
  constexpr int NC = MASS ? 1 : 6;
  constexpr int NI = e_ni(P, R), NJ = e_nj(P, R);
  constexpr int CU = 1;  // classes rolled: unrolled, the six classes took 255 registers and spilled
  const Dir& D2 = A.d[1];
  const int nq1 = A.d[0].nqp, nq2 = D2.nqp, NQ = A.NQ, n2 = D2.n;
  const int i2 = H ? n2 - 1 - R : R;
  const int qi = H ? nq2 - NI : 0;
  const int jlo = H ? n2 - 1 - R - P : 0;
  const int64_t nnz2 = A.nnz1[1];
  // the row's points are read as NV pairs from the even index qi - O (nq2 is odd, so
  // qi = nq2 - NI has the parity of P at the high end; T3 rows have even length)
  constexpr int O = H ? (P & 1) : 0, NV = (NI + O + 1) / 2;
  const Real* T3 = reinterpret_cast<const Real*>(A.T3) + ((p3 * NT) * nq1 + q1) * (int64_t)A.t3w + qi - O;
  const int64_t tstride = (int64_t)nq1 * A.t3w;
  const int64_t pbase = D2.prefix[i2];
  Real acc[NJ];  // one G group at a time (classes come grouped)
#pragma unroll(CU)
  for (int c = 0; c < NC; ++c) {
    const ClassInfo ci = class_info<true>(c);  // rolled: from constant memory
    if (MASS || ci.first)
#pragma unroll
      for (int jj = 0; jj < NJ; ++jj) acc[jj] = zeroR<Real>();
    Real h[NI];
#pragma unroll
    for (int t = 0; t < NI; ++t) h[t] = zeroR<Real>();
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int term = MASS ? 0 : ci.term[k];
      if (term < 0 || (MASS && k > 0)) continue;
      const int l = MASS ? 0 : term / 3, m = MASS ? 0 : term % 3;
      const int k2 = MASS ? 0 : 2 * (l == 1) + (m == 1);
      const Real* wrow = tab<Real>(D2.w) + ((size_t)k2 * n2 + i2) * NQ;
      const Real* trow = T3 + term * tstride;
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        Real a[2];
        ld2(trow + 2 * v, a[0], a[1]);
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int t = 2 * v + u - O;
          if (t >= 0 && t < NI) h[t] = fmaR<Real>(ro(wrow + t), a[u], h[t]);
        }
      }
    }
    const int g = MASS ? 0 : ci.g;
    const int b2 = MASS ? 0 : ci.b2;
#pragma unroll
    for (int jj = 0; jj < NJ; ++jj) {
      const Real* brow = tab<Real>(D2.bt) + ((size_t)b2 * n2 + jlo + jj) * NQ + e_toff(P, R, H, jj);
#pragma unroll
      for (int t = e_tlo(P, R, H, jj); t < e_thi(P, R, H, jj); ++t)
        acc[jj] = fmaR<Real>(ro(brow + t), h[t], acc[jj]);
    }
    if (MASS || ci.last) {
      GOut* dst = reinterpret_cast<GOut*>(A.G) + ((p3 * NG + g) * nq1 + q1) * nnz2 + pbase;
#pragma unroll
      for (int jj = 0; jj < NJ; ++jj) dst[jj] = toOut<GOut>(acc[jj]);
      if (sizeof(GOut) < sizeof(Real) && A.Gb && (q1 < A.nbl || q1 >= A.hstart)) {
        GE* dd = reinterpret_cast<GE*>(A.Gb) + ((p3 * NG + g) * A.nbq + edge_row(q1, A.nbl, A.hstart, A.nbq)) * nnz2 + pbase;
#pragma unroll
        for (int jj = 0; jj < NJ; ++jj) dd[jj] = toOut<GE>(acc[jj]);
      }
    }
  }
}

// K2 on one edge row of direction 2 (R from the low or the high end) with its
// compile-time point pattern; threads over (p3, q1), so a warp shares one pattern
// and every lane has work. One instantiation per edge row keeps each row's
// registers to itself.
template <int P, bool MASS, typename Real, typename GOut, int R, bool H, typename GE>
__global__ void __launch_bounds__(128) k_stage2_edge(StagedArgs A, int64_t np3) {
  const int nq1 = A.d[0].nqp;
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;  // p3 * nq1 + q1
  if (e >= np3 * nq1) return;
  stage2_edge_row<P, MASS, Real, GOut, R, H, GE>(A, (int)(e % nq1), e / nq1);
}

// The P+1 edge rows of one side in one launch (FP32, FP64): blockIdx.x = tile * (P+1)
// + R, so the blocks of the rows that read the same T3 points of a tile run together
// and share them through L2 (as separate launches each row read them from DRAM again;
// FP32 2.38 -> 1.34 ms at p = 5, 128^3, FP64 243.96 -> 242.68 ms per step at p = 8,
// 93^3). The double-float form keeps one launch per row: merged it measured 3.17 ->
// 3.58 ms (bound by arithmetic, and the largest row's registers set every row's
// occupancy).
template <int P, bool MASS, typename Real, typename GOut, bool H, typename GE, int R = 0>
__device__ __forceinline__ void stage2_edge_any(const StagedArgs& A, int r, int q1, int64_t p3) {
  if (r == R) {
    stage2_edge_row<P, MASS, Real, GOut, R, H, GE>(A, q1, p3);
    return;
  }
  if constexpr (R < P) stage2_edge_any<P, MASS, Real, GOut, H, GE, R + 1>(A, r, q1, p3);
}

template <int P, bool MASS, typename Real, typename GOut, bool H, typename GE>
__global__ void __launch_bounds__(128) k_stage2_edge_side(StagedArgs A, int64_t np3) {
  const int nq1 = A.d[0].nqp;
  const int r = blockIdx.x % (P + 1);
  const int64_t e = (blockIdx.x / (P + 1)) * (int64_t)blockDim.x + threadIdx.x;  // p3 * nq1 + q1
  if (e >= np3 * nq1) return;
  stage2_edge_any<P, MASS, Real, GOut, H, GE>(A, r, (int)(e % nq1), e / nq1);
}

template <int P, bool MASS, typename Real, typename GOut, typename GE, int B = 0>
static void launch_stage2_edge(const StagedArgs& A, int nq1, int64_t np3, cudaStream_t s) {
  if constexpr (!std::is_same<Real, f2>::value) {
    // FP32, FP64: one launch per side
    const unsigned tiles = (unsigned)((np3 * nq1 + 127) / 128);
    k_stage2_edge_side<P, MASS, Real, GOut, false, GE><<<tiles * (P + 1), 128, 0, s>>>(A, np3);
    k_stage2_edge_side<P, MASS, Real, GOut, true, GE><<<tiles * (P + 1), 128, 0, s>>>(A, np3);
  } else {
    k_stage2_edge<P, MASS, Real, GOut, (B <= P ? B : B - P - 1), (B > P), GE>
        <<<(unsigned)((np3 * nq1 + 127) / 128), 128, 0, s>>>(A, np3);
    if constexpr (B + 1 < 2 * P + 2) launch_stage2_edge<P, MASS, Real, GOut, GE, B + 1>(A, nq1, np3, s);
  }
}

template <int P, typename Real>
constexpr int stage2_edge_launches() { return std::is_same<Real, f2>::value ? 2 * P + 2 : 2; }

// Stage 1 of one (p2, i1, p3) for the HOST form of k_stage1: the same arithmetic as
// k_stage1, the values into the warp's slice sl (lane-major, bw1 per lane), then the
// warp's stores. Lanes with p2 >= nnz2 compute nothing and store nothing.
template <int P, bool MASS, typename Real, typename OutT, bool EDGE64, typename RE>
__device__ __forceinline__ void k_stage1_host(const StagedArgs& A, int64_t p2, int i1, int64_t p3l, int64_t p3, OutT* sl,
                                              int64_t* hb) {
  constexpr int BW = 2 * P + 1;
  constexpr int NG = MASS ? 1 : 4;
  const Dir& D1 = A.d[0];
  const Dir& D2 = A.d[1];
  const Dir& D3 = A.d[2];
  const int64_t nnz2 = A.nnz1[1];
  const int n1 = D1.n, n2 = D2.n, n3 = D3.n, nq1 = D1.nqp, NQ = A.NQ;
  const int lane = threadIdx.x;
  const bool act = p2 < nnz2;
  const int bw1 = bw(i1, P, n1), jlo1 = blo(i1, P);
  if (act) {
    const int i2 = D2.pair_row[p2], j2 = blo(i2, P) + (int)(p2 - D2.prefix[i2]);
    const int i3 = D3.pair_row[p3], j3 = blo(i3, P) + (int)(p3 - D3.prefix[i3]);
    const int qi1 = D1.q0[i1];
    const bool reg = i1 >= P + 1 && i1 <= n1 - P - 2;
    const Real* G = reinterpret_cast<const Real*>(A.G) + ((p3l * NG) * nq1) * nnz2 + p2;
    const int64_t gstride = (int64_t)nq1 * nnz2;
    const int64_t N1 = D1.prefix[n1], N2 = D2.prefix[n2];
    const int bw2 = bw(i2, P, n2), bw3 = bw(i3, P, n3);
    const int64_t row = D3.prefix[i3] * N2 * N1 + (int64_t)bw3 * (D2.prefix[i2] * N1 + (int64_t)bw2 * D1.prefix[i1]);
    hb[lane] = row + ((int64_t)(j3 - blo(i3, P)) * bw2 + (j2 - blo(i2, P))) * bw1;
    const Real* w = tab<Real>(D1.w) + (size_t)i1 * NQ;
    const Real* bt1 = tab<Real>(D1.bt);
    const int64_t wk = (int64_t)n1 * NQ, bder = (int64_t)n1 * NQ;
    if (reg) {
      Real s[BW];
#pragma unroll
      for (int tt = 0; tt < BW; ++tt) s[tt] = zeroR<Real>();
#pragma unroll
      for (int t = 0; t <= 2 * P; ++t) {
        const Real* gq = G + (int64_t)(qi1 + t) * nnz2;
        Real h0, h1 = zeroR<Real>();
        if (MASS) {
          h0 = mulR(w[t], gq[0]);
        } else {
          h0 = fmaR<Real>(w[t], gq[0], mulR(w[t + 2 * wk], gq[2 * gstride]));
          h1 = fmaR<Real>(w[t + wk], gq[gstride], mulR(w[t + 3 * wk], gq[3 * gstride]));
        }
#pragma unroll
        for (int tt = 0; tt < BW; ++tt) {
          if (t >= 2 * tt - 2 * P && t <= 2 * tt) {
            const int j1 = i1 - P + tt;
            const int64_t idx = (int64_t)j1 * NQ + (qi1 + t - D1.q0[j1]);
            if (MASS)
              s[tt] = fmaR<Real>(bt1[idx], h0, s[tt]);
            else
              s[tt] = fmaR<Real>(bt1[idx + bder], h1, fmaR<Real>(bt1[idx], h0, s[tt]));
          }
        }
      }
#pragma unroll
      for (int tt = 0; tt < BW; ++tt) sl[lane * BW + tt] = toOut<OutT>(s[tt]);  // bw1 = BW here
    } else if (EDGE64 && A.Gb) {
      const RE* Gd = reinterpret_cast<const RE*>(A.Gb) + ((p3l * NG) * A.nbq) * nnz2 + p2;
      stage1_edge<P, MASS, RE, OutT, true>(Gd, (int64_t)A.nbq * nnz2, nnz2, tab<RE>(A.w1e) + (size_t)i1 * NQ, wk,
                                           tab<RE>(A.bt1e), bder, D1, i1, n1, NQ, A.nbl, A.hstart, A.nbq, sl,
                                           (int64_t)lane * bw1 - jlo1);
    } else {
      stage1_edge<P, MASS, Real, OutT, false>(G, gstride, nnz2, w, wk, bt1, bder, D1, i1, n1, NQ, 0, 0, 0, sl,
                                              (int64_t)lane * bw1 - jlo1);
    }
  }
  __syncwarp();
  OutT* out = reinterpret_cast<OutT*>(A.vals);
  const int64_t left = nnz2 - (p2 - lane);
  const int nact = left < 32 ? (int)left : 32;  // active lanes of the warp
  if (bw1 == BW) {
#pragma unroll
    for (int k = 0; k < BW; ++k) {
      const int e = lane + 32 * k, r = e / BW;
      if (r < nact) out[hb[r] + (e - r * BW)] = sl[e];
    }
  } else {
    for (int e = lane; e < nact * bw1; e += 32) {
      const int r = e / bw1;
      out[hb[r] + (e - r * bw1)] = sl[e];
    }
  }
}

// K1: one thread per (p2, i1, p3): the 2P+1 values of row (i1, i2, i3) in the
// column block (j2, j3). A block covers 32 consecutive p2 and 4 consecutive i1, so
// the G rows of overlapping supports are read from L1.
// EDGE64: the first and last P+1 rows of direction 1 run in type RE (double-float)
// from the edge copy of G, where the large, sign-alternating WQ weights near the
// boundary amplify FP32 rounding. Rows [gap_lo, gap_lo + gap_len) of direction 1 are
// skipped (the FFMA or tensor-core kernel assembles them); gap_len = 0 assembles
// every row.
// HOST: out is page-locked host memory; each warp (one row i1, 32 consecutive p2)
// puts its values in a shared-memory slice and stores them as runs of consecutive
// addresses (lane l's bw1 values are contiguous, and neighbouring p2 of one row i2
// are neighbouring blocks), so the values cross the host link as whole lines.
template <int P, bool MASS, typename Real, typename OutT, bool EDGE64, typename RE = double, bool HOST = false>
__global__ void __launch_bounds__(128) k_stage1(StagedArgs A, int gap_lo, int gap_len) {
  constexpr int BW = 2 * P + 1;
  constexpr int NG = MASS ? 1 : 4;
  __shared__ OutT hs[HOST ? 4 : 1][HOST ? 32 * BW : 1];   // per warp: 32 x bw1 values
  __shared__ int64_t hb[HOST ? 4 : 1][32];                // per warp: each lane's first address
  const Dir& D1 = A.d[0];
  const Dir& D2 = A.d[1];
  const Dir& D3 = A.d[2];
  const int64_t p2 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int i1k = blockIdx.y * blockDim.y + threadIdx.y;
  const int i1 = i1k < gap_lo ? i1k : i1k + gap_len;
  const int64_t p3l = blockIdx.z, p3 = A.p3_off + p3l;  // slab-relative and absolute band pair
  const int64_t nnz2 = A.nnz1[1];
  const int n1 = D1.n, n2 = D2.n, n3 = D3.n, nq1 = D1.nqp, NQ = A.NQ;
  if (i1 >= n1) return;                                  // whole warps
  if (!HOST && p2 >= nnz2) return;
  if (HOST) {
    k_stage1_host<P, MASS, Real, OutT, EDGE64, RE>(A, p2, i1, p3l, p3, hs[threadIdx.y], hb[threadIdx.y]);
    return;
  }
  const int i2 = D2.pair_row[p2], j2 = blo(i2, P) + (int)(p2 - D2.prefix[i2]);
  const int i3 = D3.pair_row[p3], j3 = blo(i3, P) + (int)(p3 - D3.prefix[i3]);
  const int qi1 = D1.q0[i1];
  const bool reg = i1 >= P + 1 && i1 <= n1 - P - 2;
  const Real* G = reinterpret_cast<const Real*>(A.G) + ((p3l * NG) * nq1) * nnz2 + p2;
  const int64_t gstride = (int64_t)nq1 * nnz2;  // next group
  const int64_t N1 = D1.prefix[n1], N2 = D2.prefix[n2];
  const int bw1 = bw(i1, P, n1), bw2 = bw(i2, P, n2), bw3 = bw(i3, P, n3);
  const int jlo1 = blo(i1, P);
  const int64_t row = D3.prefix[i3] * N2 * N1 + (int64_t)bw3 * (D2.prefix[i2] * N1 + (int64_t)bw2 * D1.prefix[i1]);
  const int64_t base = row + ((int64_t)(j3 - blo(i3, P)) * bw2 + (j2 - blo(i2, P))) * bw1;  // + (j1 - jlo1)
  OutT* out = reinterpret_cast<OutT*>(A.vals);
  const Real* w = tab<Real>(D1.w) + (size_t)i1 * NQ;   // kind k at + k * n1 * NQ
  const Real* bt1 = tab<Real>(D1.bt);
  const int64_t wk = (int64_t)n1 * NQ;
  const int64_t bder = (int64_t)n1 * NQ;          // B' table after B
  Real s[BW];
#pragma unroll
  for (int tt = 0; tt < BW; ++tt) s[tt] = zeroR<Real>();
  if (reg) {
#pragma unroll
    for (int t = 0; t <= 2 * P; ++t) {
      const Real* gq = G + (int64_t)(qi1 + t) * nnz2;
      Real h0, h1 = zeroR<Real>();
      if (MASS) {
        h0 = mulR(w[t], gq[0]);
      } else {
        h0 = fmaR<Real>(w[t], gq[0], mulR(w[t + 2 * wk], gq[2 * gstride]));
        h1 = fmaR<Real>(w[t + wk], gq[gstride], mulR(w[t + 3 * wk], gq[3 * gstride]));
      }
#pragma unroll
      for (int tt = 0; tt < BW; ++tt) {
        if (t >= 2 * tt - 2 * P && t <= 2 * tt) {
          const int j1 = i1 - P + tt;
          const int64_t idx = (int64_t)j1 * NQ + (qi1 + t - D1.q0[j1]);
          if (MASS)
            s[tt] = fmaR<Real>(bt1[idx], h0, s[tt]);
          else
            s[tt] = fmaR<Real>(bt1[idx + bder], h1, fmaR<Real>(bt1[idx], h0, s[tt]));
        }
      }
    }
#pragma unroll
    for (int tt = 0; tt < BW; ++tt) out[base + tt] = toOut<OutT>(s[tt]);  // j1 - jlo1 = tt for regular rows
  } else if (EDGE64 && A.Gb) {
    const RE* Gd = reinterpret_cast<const RE*>(A.Gb) + ((p3l * NG) * A.nbq) * nnz2 + p2;
    stage1_edge<P, MASS, RE, OutT, true>(Gd, (int64_t)A.nbq * nnz2, nnz2, tab<RE>(A.w1e) + (size_t)i1 * NQ, wk,
                                         tab<RE>(A.bt1e),
                                             bder, D1, i1, n1, NQ, A.nbl, A.hstart, A.nbq, out, base - jlo1);
  } else {
    stage1_edge<P, MASS, Real, OutT, false>(G, gstride, nnz2, w, wk, bt1, bder, D1, i1, n1, NQ, 0, 0, 0, out,
                                            base - jlo1);
  }
}

// ---------------------------------------------------------------------------
// Stage 1 on the tensor cores (WQ_PREC_TF32X3), regular rows of direction 1.
//
// For a regular row i1 (Q_i1 = [q0, q0 + 2P]) the last mode product is a small
// dense contraction, the same for every band pair (p2, p3):
//   s(i1; p2, p3)[tt] = sum_k G[p3][g][q0 + t][p2] W_i1[k][tt],   k = NG t + g,
//   W_i1[k][tt] = w1^{g}(i1, q0 + t) B1^{g & 1}(i1 - P + tt, q0 + t)
// (zero outside the support overlap). With M = 16 band pairs p2 per warp, K = k and
// N = tt it runs as mma.sync m16n8k8 on TF32 operands, each operand split into a
// TF32 head and a TF32 tail (a = a_h + a_t) and the product taken as
// a_t b_h + a_h b_t + a_h b_h with FP32 accumulation: about FP32 accuracy, against
// TF32's 2^-11. For stiffness (NG = 4) one k-step of 8 holds 2 points x 4 groups,
// so row i1 + 1 (window shifted by 2 points) reuses the A fragments of row i1
// shifted by one k-step: G is read once per CTA. The outputs go through shared
// memory and leave as contiguous runs of the CSR rows (coalesced stores).
namespace tc {

__device__ __forceinline__ unsigned tf32_rna(float x) {
  unsigned r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

template <int P, bool MASS>
struct Shape {
  static constexpr int BW = 2 * P + 1;
  static constexpr int NG = MASS ? 1 : 4;
  static constexpr int KT = NG * BW;       // K extent
  static constexpr int KS = (KT + 7) / 8;  // k-steps of 8
  static constexpr int NT = (BW + 7) / 8;  // n-tiles of 8
  static constexpr int WARPS = 8;
  static constexpr int MT = 16 * WARPS;    // band pairs p2 per CTA
  static constexpr int CHUNK = 32;         // rows i1 per CTA
};

// W_i1 in the B-fragment layout of mma.m16n8k8 (.col): for k-step s, n-tile nt and
// lane l, {b0_head, b1_head, b0_tail, b1_tail} with b0 = W[8s + l%4][8nt + l/4] and
// b1 = W[8s + 4 + l%4][8nt + l/4]. One thread per (row, s, nt, lane).
template <int P, bool MASS>
__global__ void k_bfrag(const double* __restrict__ w, const double* __restrict__ bt, const int* __restrict__ q0,
                        const int* __restrict__ nq, int n1, int NQ, int i1_lo, int nrows, float4* __restrict__ out) {
  using S = Shape<P, MASS>;
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)nrows * S::KS * S::NT * 32) return;
  const int lane = (int)(e % 32);
  const int nt = (int)((e / 32) % S::NT);
  const int st = (int)((e / (32 * S::NT)) % S::KS);
  const int i1 = i1_lo + (int)(e / (32 * S::NT * S::KS));
  const int tt = 8 * nt + lane / 4;
  const int qi = q0[i1];
  float hv[2], tv[2];
  for (int h = 0; h < 2; ++h) {
    const int k = 8 * st + 4 * h + lane % 4;
    double v = 0.0;
    if (k < S::KT && tt < S::BW) {
      const int t = MASS ? k : k / 4, g = MASS ? 0 : k % 4;
      const int j1 = i1 - P + tt, q = qi + t;
      const int loc = q - q0[j1];
      if (j1 >= 0 && j1 < n1 && loc >= 0 && loc < nq[j1])
        v = w[((size_t)g * n1 + i1) * NQ + t] * bt[((size_t)(g & 1) * n1 + j1) * NQ + loc];
    }
    const float f = (float)v;
    const float head = __uint_as_float(tf32_rna(f));
    hv[h] = head;
    tv[h] = __uint_as_float(tf32_rna(f - head));
  }
  out[e] = make_float4(hv[0], hv[1], tv[0], tv[1]);
}

template <int P, bool MASS>
__device__ __forceinline__ float a_elem(const float* __restrict__ G, int64_t gstride, int64_t nnz2, int nq1, int qi,
                                        int k, int64_t p2, bool ok) {
  const int t = MASS ? k : k >> 2, g = MASS ? 0 : k & 3;
  const int q = qi + t;
  return (ok && q < nq1) ? __ldg(G + g * gstride + (int64_t)q * nnz2 + p2) : 0.0f;
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ void split4(const float (&v)[4], unsigned (&ah)[4], unsigned (&at)[4]) {
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    ah[r] = tf32_rna(v[r]);
    at[r] = tf32_rna(v[r] - __uint_as_float(ah[r]));
  }
}

template <int P, bool MASS>
__device__ __forceinline__ void fetch_a(const float* G, int64_t gstride, int64_t nnz2, int nq1, int qi, int st,
                                        int64_t p2a, bool oka, int64_t p2b, bool okb, int lane, float (&v)[4]) {
  const int k0 = 8 * st + lane % 4;
  v[0] = a_elem<P, MASS>(G, gstride, nnz2, nq1, qi, k0, p2a, oka);
  v[1] = a_elem<P, MASS>(G, gstride, nnz2, nq1, qi, k0, p2b, okb);
  v[2] = a_elem<P, MASS>(G, gstride, nnz2, nq1, qi, k0 + 4, p2a, oka);
  v[3] = a_elem<P, MASS>(G, gstride, nnz2, nq1, qi, k0 + 4, p2b, okb);
}

// The W fragments of row i1 (shared by the CTA's warps) stream into a double
// buffer in shared memory with cp.async one row ahead; the A k-step that row i1 + 1
// adds is fetched into registers before the products of row i1.
template <int P, bool MASS, typename OutT>
__global__ void __launch_bounds__(256) k_stage1_mma(StagedArgs A, const float4* __restrict__ bfrag, int i1_lo,
                                                    int i1_hi) {
  using S = Shape<P, MASS>;
  constexpr int BW = S::BW, KS = S::KS, NT = S::NT, MT = S::MT, NG = S::NG;
  constexpr int NF = KS * NT * 32;  // float4 fragments per row i1
  __shared__ float stage[2][MT * BW];
  __shared__ float4 wsm[2][NF];
  __shared__ int64_t xb[MT];
  __shared__ int yb[MT];
  const Dir& D1 = A.d[0];
  const Dir& D2 = A.d[1];
  const Dir& D3 = A.d[2];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t nnz2 = A.nnz1[1];
  const int64_t p2_0 = (int64_t)blockIdx.x * MT;
  const int64_t p3l = blockIdx.y, p3 = A.p3_off + p3l;  // slab-relative and absolute band pair
  const int ia = i1_lo + blockIdx.z * S::CHUNK, ib = min(i1_hi, ia + S::CHUNK);
  const int n1 = D1.n, n2 = D2.n, n3 = D3.n, nq1 = D1.nqp;
  // W fragments of the first row
  for (int f = threadIdx.x; f < NF; f += blockDim.x) cp_async16(&wsm[0][f], bfrag + (size_t)(ia - i1_lo) * NF + f);
  // output base of each band pair of the tile: value (i1, p2, p3, tt) sits at
  // xb + yb * prefix1(i1) + tt for a regular row i1 (Kronecker order, Section 3)
  {
    const int i3 = D3.pair_row[p3], j3 = blo(i3, P) + (int)(p3 - D3.prefix[i3]);
    const int bw3 = bw(i3, P, n3);
    const int64_t N1 = D1.prefix[n1], N2 = D2.prefix[n2];
    for (int r = threadIdx.x; r < MT; r += blockDim.x) {
      const int64_t p2 = p2_0 + r;
      if (p2 < nnz2) {
        const int i2 = D2.pair_row[p2], j2 = blo(i2, P) + (int)(p2 - D2.prefix[i2]);
        const int bw2 = bw(i2, P, n2);
        xb[r] = D3.prefix[i3] * N2 * N1 + (int64_t)bw3 * D2.prefix[i2] * N1 +
                ((int64_t)(j3 - blo(i3, P)) * bw2 + (j2 - blo(i2, P))) * BW;
        yb[r] = bw3 * bw2;
      }
    }
  }
  const float* G = reinterpret_cast<const float*>(A.G) + (p3l * NG) * (int64_t)nq1 * nnz2;
  const int64_t gstride = (int64_t)nq1 * nnz2;
  const int64_t p2a = p2_0 + 16 * warp + (lane >> 2), p2b = p2a + 8;
  const bool oka = p2a < nnz2, okb = p2b < nnz2;
  float av[KS][4];  // A fragments as FP32; split into TF32 head and tail at each use
  {
    const int qi = D1.q0[ia];
#pragma unroll
    for (int st = 0; st < KS; ++st) fetch_a<P, MASS>(G, gstride, nnz2, nq1, qi, st, p2a, oka, p2b, okb, lane, av[st]);
  }
  cp_async_wait_all();
  __syncthreads();
  OutT* out = reinterpret_cast<OutT*>(A.vals);
  const int nflush = MT * BW;
  for (int i1 = ia; i1 < ib; ++i1) {
    const int cur = (i1 - ia) & 1;
    const bool more = i1 + 1 < ib;
    // prefetch: W of row i1 + 1 into the other buffer, the k-step that row i1 + 1 adds
    if (more)
      for (int f = threadIdx.x; f < NF; f += blockDim.x)
        cp_async16(&wsm[cur ^ 1][f], bfrag + (size_t)(i1 + 1 - i1_lo) * NF + f);
    float nv[4];
    if (!MASS && more) fetch_a<P, MASS>(G, gstride, nnz2, nq1, D1.q0[i1 + 1], KS - 1, p2a, oka, p2b, okb, lane, nv);
    // two accumulator sets: head x head, and the two correction products, so that
    // 2 NT independent MMA chains are in flight
    float acc[NT][4], cor[NT][4];
#pragma unroll
    for (int nt = 0; nt < NT; ++nt)
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[nt][r] = cor[nt][r] = 0.0f;
    const float4* wf = wsm[cur] + lane;
#pragma unroll
    for (int st = 0; st < KS; ++st) {
      unsigned ah[4], at[4];
      split4(av[st], ah, at);
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) {
        const float4 b = wf[(st * NT + nt) * 32];
        mma_tf32(cor[nt], at, __float_as_uint(b.x), __float_as_uint(b.y));   // tail x head
        mma_tf32(acc[nt], ah, __float_as_uint(b.x), __float_as_uint(b.y));   // head x head
        mma_tf32(cor[nt], ah, __float_as_uint(b.z), __float_as_uint(b.w));   // head x tail
      }
    }
    // accumulators: rows lane/4 (+8), columns 8 nt + 2 (lane % 4) (+1)
    float* sb = stage[cur];
    const int r0 = 16 * warp + (lane >> 2);
#pragma unroll
    for (int nt = 0; nt < NT; ++nt)
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int tt = 8 * nt + 2 * (lane & 3) + c;
        if (tt < BW) {
          sb[r0 * BW + tt] = acc[nt][c] + cor[nt][c];
          sb[(r0 + 8) * BW + tt] = acc[nt][2 + c] + cor[nt][2 + c];
        }
      }
    if (more) {
      if (MASS) {
        const int qn = D1.q0[i1 + 1];
#pragma unroll
        for (int st = 0; st < KS; ++st) fetch_a<P, MASS>(G, gstride, nnz2, nq1, qn, st, p2a, oka, p2b, okb, lane, av[st]);
      } else {
        // the window moves by two points = one k-step
#pragma unroll
        for (int st = 0; st + 1 < KS; ++st)
#pragma unroll
          for (int r = 0; r < 4; ++r) av[st][r] = av[st + 1][r];
#pragma unroll
        for (int r = 0; r < 4; ++r) av[KS - 1][r] = nv[r];
      }
    }
    cp_async_wait_all();
    __syncthreads();
    const int64_t pre = D1.prefix[i1];
    for (int e = threadIdx.x; e < nflush; e += blockDim.x) {
      const int r = e / BW;
      if (p2_0 + r < nnz2) out[xb[r] + (int64_t)yb[r] * pre + (e - r * BW)] = toOut<OutT>(sb[e]);
    }
  }
}

}  // namespace tc

// ---------------------------------------------------------------------------
// Stage 1 for the regular rows of direction 1 with FP32 G (WQ_PREC_MIXED, WQ_PREC_FP32):
// one band pair p2 per thread, a CTA of 256 consecutive band pairs for one p3 and
// a chunk of rows i1. For a regular row the q1 window is [2 i1 - P, 2 i1 + P], so
// row i1 + 1 reuses the window of row i1 shifted by two points: each thread keeps
// the window of its G column in registers and loads every value once. The row's
// rule weights and trial values sit in shared memory (built one row ahead, read as
// broadcasts), the contraction folds the test weights into h_b per point and adds
// B^{(b)}(j1) h_b over the support overlaps only, and the values leave through
// shared memory as contiguous runs of the CSR rows.
// Tables of the FFMA stage 1 for regular rows [i1_lo, i1_lo + nrows) of direction 1,
// as float4: the four rule weights of point t, then for point t the (B, B') values of
// its band tt = (t + 1)/2 .. (t + 1)/2 + P (P + 1 - (t & 1) of them, the rest zero),
// SL float4 per point. One thread per (row, float4).
template <int P, bool MASS>
__global__ void k_s1_tables(const float* __restrict__ w1, const float* __restrict__ b1, const int* __restrict__ q0,
                            const int* __restrict__ nq, int n1, int NQ, int i1_lo, int nrows, float4* __restrict__ out) {
  constexpr int BW = 2 * P + 1, SL = (P + 2) / 2, TF4 = BW + BW * SL;
  const int64_t e0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e0 >= (int64_t)nrows * TF4) return;
  const int i1 = i1_lo + (int)(e0 / TF4), e = (int)(e0 % TF4);
  const int qi = q0[i1];
  auto bval = [&](int b, int t, int tt) {
    const int j1 = i1 - P + tt, loc = qi + t - q0[j1];
    return (tt < BW && loc >= 0 && loc < nq[j1]) ? b1[((size_t)b * n1 + j1) * NQ + loc] : 0.0f;
  };
  float4 v;
  if (e < BW) {
    const size_t o = (size_t)i1 * NQ + e, k = (size_t)n1 * NQ;
    v = MASS ? make_float4(w1[o], 0.0f, 0.0f, 0.0f) : make_float4(w1[o], w1[o + k], w1[o + 2 * k], w1[o + 3 * k]);
  } else {
    const int f = e - BW, t = f / SL, k = 2 * (f % SL), tt = (t + 1) / 2 + k;
    const int cnt = P + 1 - (t & 1);
    v = make_float4(k < cnt ? bval(0, t, tt) : 0.0f, (!MASS && k < cnt) ? bval(1, t, tt) : 0.0f,
                    k + 1 < cnt ? bval(0, t, tt + 1) : 0.0f, (!MASS && k + 1 < cnt) ? bval(1, t, tt + 1) : 0.0f);
  }
  out[e0] = v;
}

// Regular rows [i1_lo, i1_hi) of direction 1 in chunks of 32 rows (blockIdx.x = tile
// of 256 band pairs * n_chunks + chunk, blockIdx.y = p3 of the slab). The first and last
// P+1 rows run in k_stage1 (gap = these rows) beside this kernel on another stream.
// Each warp hands its 32 x BW values to the CSR through a shared-memory slice: lane l
// puts its BW values at l * BW + tt (BW odd: no bank conflicts), then the warp stores
// element e = l + 32 k to out[base + off(e)], where off(e) = X(r) - X(0) + tt +
// (yb(r) - yb(0)) * prefix1(i1) for r = e / BW, tt = e - r BW, X(r) the row-independent
// part of lane r's CSR offset and yb(r) = bw3 bw2(r). The relative offsets are fixed
// for the block, so a store costs a shared load, an integer multiply-add and the store
// itself; consecutive lanes write consecutive addresses inside each row i2.
template <int P, bool MASS, typename OutT>
__global__ void __launch_bounds__(256, P <= 6 ? 2 : 1) k_stage1_ffma(StagedArgs A, const float4* __restrict__ tabs, int i1_lo,
                                                        int i1_hi, int n_chunks) {
  constexpr int BW = 2 * P + 1, NG = MASS ? 1 : 4, MT = 256, CHUNK = 32, WARPS = MT / 32;
  // Tables of a row, read as float4 broadcasts: the four rule weights of point t,
  // then for point t the (B, B') values of its band tt = (t + 1)/2 .. (t + 1)/2 + P
  // (P + 1 - (t & 1) of them; the rest zero), in a slot of SL float4.
  constexpr int SL = (P + 2) / 2;  // float4 per point: 2 (B, B') pairs each
  constexpr int TF4 = BW + BW * SL;
  // dynamic shared memory (ffma_smem<P>() bytes): the tables of the chunk's rows,
  // loaded once, so the warps run through the rows without block barriers; the
  // per-warp store slices; the store offsets
  extern __shared__ float4 dsm[];
  float4* tbl = dsm;                                                 // [CHUNK][TF4]
  float* stage = reinterpret_cast<float*>(dsm + CHUNK * TF4);        // [WARPS][32 BW]
  int* soff = reinterpret_cast<int*>(stage + WARPS * 32 * BW);       // [BW][MT]: relative offset of
                                                                     // element e = lane + 32 k (INT_MIN: none)
  short* syd = reinterpret_cast<short*>(soff + BW * MT);             // [BW][MT]: yb(r) - yb(0)
  const int role = blockIdx.x % n_chunks;
  const int64_t p2_0 = (int64_t)(blockIdx.x / n_chunks) * MT;
  const Dir& D1 = A.d[0];
  const Dir& D2 = A.d[1];
  const Dir& D3 = A.d[2];
  const int64_t nnz2 = A.nnz1[1];
  const int64_t p3l = blockIdx.y, p3 = A.p3_off + p3l;
  const int ia = i1_lo + role * CHUNK, ib = min(i1_hi, ia + CHUNK);
  const int n1 = D1.n, n2 = D2.n, n3 = D3.n, nq1 = D1.nqp;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // tables of the chunk's rows (precomputed by k_s1_tables), through cp.async
  for (int e = threadIdx.x; e < (ib - ia) * TF4; e += blockDim.x)
    tc::cp_async16(tbl + e, tabs + (size_t)(ia - i1_lo) * TF4 + e);
  const int i3 = D3.pair_row[p3], j3 = blo(i3, P) + (int)(p3 - D3.prefix[i3]);
  const int bw3 = bw(i3, P, n3);
  const int64_t N1 = D1.prefix[n1], N2 = D2.prefix[n2];
  const int64_t p2 = p2_0 + threadIdx.x;
  const bool ok = p2 < nnz2;
  // this lane's X and yb (the CSR offset of its block of row i1 is X + yb * prefix1(i1))
  int64_t X = 0;
  int yb = 0;
  if (ok) {
    const int i2 = D2.pair_row[p2], j2 = blo(i2, P) + (int)(p2 - D2.prefix[i2]);
    const int bw2 = bw(i2, P, n2);
    X = D3.prefix[i3] * N2 * N1 + (int64_t)bw3 * D2.prefix[i2] * N1 +
        ((int64_t)(j3 - blo(i3, P)) * bw2 + (j2 - blo(i2, P))) * BW;
    yb = bw3 * bw2;
  }
  const int64_t X0 = __shfl_sync(0xffffffffu, X, 0);
  const int yb0 = __shfl_sync(0xffffffffu, yb, 0);
#pragma unroll
  for (int k = 0; k < BW; ++k) {
    const int e = lane + 32 * k, r = e / BW;
    const int64_t Xr = __shfl_sync(0xffffffffu, X, r);
    const int ybr = __shfl_sync(0xffffffffu, yb, r);
    const bool okr = p2_0 + warp * 32 + r < nnz2;
    soff[k * MT + threadIdx.x] = okr ? (int)(Xr - X0) + (e - r * BW) : INT_MIN;
    syd[k * MT + threadIdx.x] = (short)(ybr - yb0);
  }
  // the thread's G column (lanes past nnz2 read column 0 and store nothing); regular
  // rows' windows [2 i1 - P, 2 i1 + P] lie inside [0, nq1)
  const float* G = reinterpret_cast<const float*>(A.G) + (p3l * NG) * (int64_t)nq1 * nnz2 + (ok ? p2 : 0);
  const int64_t gstride = (int64_t)nq1 * nnz2;
  float gw[NG][BW];  // the q1 window of this thread's G column
  const float* gq = G + (int64_t)D1.q0[ia] * nnz2;
#pragma unroll
  for (int g = 0; g < NG; ++g)
#pragma unroll
    for (int t = 0; t < BW; ++t) gw[g][t] = __ldg(gq + g * gstride + (int64_t)t * nnz2);
  gq += (int64_t)BW * nnz2;  // the window's next two points (the window moves by two per row)
  // warps whose band pairs all have yb = yb0 store without the per-element yb term
  const bool yu = __all_sync(0xffffffffu, !ok || yb == yb0);
  tc::cp_async_wait_all();
  __syncthreads();
  OutT* out = reinterpret_cast<OutT*>(A.vals);
  float* sb = stage + warp * 32 * BW;
  for (int i1 = ia; i1 < ib; ++i1) {
    const bool more = i1 + 1 < ib;
    const float4* tw = tbl + (i1 - ia) * TF4;
    const float4* tb = tw + BW;
    float sacc[BW];
#pragma unroll
    for (int tt = 0; tt < BW; ++tt) sacc[tt] = 0.0f;
#pragma unroll
    for (int t = 0; t < BW; ++t) {
      const float4 wv = tw[t];
      float h0, h1 = 0.0f;
      if (MASS) {
        h0 = wv.x * gw[0][t];
      } else {
        h0 = fmaf(wv.x, gw[0][t], wv.z * gw[2][t]);
        h1 = fmaf(wv.y, gw[1][t], wv.w * gw[3][t]);
      }
      const int tt0 = (t + 1) / 2, cnt = P + 1 - (t & 1);
#pragma unroll
      for (int m = 0; m < SL; ++m) {
        const float4 bv = tb[t * SL + m];
        if (2 * m < cnt) sacc[tt0 + 2 * m] = MASS ? fmaf(bv.x, h0, sacc[tt0 + 2 * m])
                                                   : fmaf(bv.y, h1, fmaf(bv.x, h0, sacc[tt0 + 2 * m]));
        if (2 * m + 1 < cnt) sacc[tt0 + 2 * m + 1] = MASS ? fmaf(bv.z, h0, sacc[tt0 + 2 * m + 1])
                                                           : fmaf(bv.w, h1, fmaf(bv.z, h0, sacc[tt0 + 2 * m + 1]));
      }
    }
    if (more) {  // the window moves by two points
#pragma unroll
      for (int g = 0; g < NG; ++g) {
#pragma unroll
        for (int t = 0; t + 2 < BW; ++t) gw[g][t] = gw[g][t + 2];
        gw[g][BW - 2] = __ldg(gq + g * gstride);
        gw[g][BW - 1] = __ldg(gq + g * gstride + nnz2);
      }
      gq += 2 * nnz2;
    }
    __syncwarp();
#pragma unroll
    for (int tt = 0; tt < BW; ++tt) sb[lane * BW + tt] = sacc[tt];
    __syncwarp();
    const int pre = (int)D1.prefix[i1];
    OutT* ob = out + (X0 + (int64_t)yb0 * pre);
    if (yu) {
#pragma unroll
      for (int k = 0; k < BW; ++k) {
        const int o = soff[k * MT + threadIdx.x];
        if (o != INT_MIN) ob[o] = toOut<OutT>(sb[lane + 32 * k]);
      }
    } else {
#pragma unroll
      for (int k = 0; k < BW; ++k) {
        const int o = soff[k * MT + threadIdx.x];
        if (o != INT_MIN) ob[o + (int)syd[k * MT + threadIdx.x] * pre] = toOut<OutT>(sb[lane + 32 * k]);
      }
    }
  }
}

template <int P>
constexpr size_t ffma_smem() {
  return sizeof(float4) * 32 * ((2 * P + 1) * (1 + (P + 2) / 2)) + sizeof(float) * 256 * (2 * P + 1) +
         (sizeof(int) + sizeof(short)) * 256 * (2 * P + 1);
}

// Stage 1 on edge row R of direction 1 (i1 = R or n1-1-R) with its compile-time
// point pattern (n_el >= 2P+2 in direction 1, as for the stage-2 edge kernels): one
// thread per band pair p2, a block row per p3. The row's rule weights and trial
// values (zero outside the support overlap) sit in shared memory; the loop runs over
// the row's NI points, folds the test weights into h_0, h_1 at the point and adds
// B h_0 + B' h_1 to the band members whose support holds the point, so no per-point
// array is kept. RE is the arithmetic: double-float from the edge copy of G (GB, the
// mixed modes), or FP32 from G itself.
template <int P, bool MASS, typename RE, typename OutT, bool GB, int R, bool H>
__device__ __forceinline__ void stage1_edge_row(const StagedArgs& A, int64_t tile) {
  constexpr int NI = e_ni(P, R), NJ = e_nj(P, R);
  constexpr int NG = MASS ? 1 : 4, NB = MASS ? 1 : 2;
  __shared__ RE ws[NG][NI];
  __shared__ RE bs[NB][NJ][NI];
  const Dir& D1 = A.d[0];
  const Dir& D2 = A.d[1];
  const Dir& D3 = A.d[2];
  const int n1 = D1.n, n2 = D2.n, n3 = D3.n, nq1 = D1.nqp, NQ = A.NQ;
  const int i1 = H ? n1 - 1 - R : R, jlo = H ? n1 - 1 - R - P : 0, qi = H ? nq1 - NI : 0;
  const RE* w1 = tab<RE>(GB ? A.w1e : D1.w);
  const RE* b1 = tab<RE>(GB ? A.bt1e : D1.bt);
  for (int e = threadIdx.x; e < NG * NI; e += blockDim.x) {
    const int g = e / NI, t = e - g * NI;
    ws[g][t] = w1[((size_t)g * n1 + i1) * NQ + t];
  }
  for (int e = threadIdx.x; e < NB * NJ * NI; e += blockDim.x) {
    const int b = e / (NJ * NI), jj = (e / NI) % NJ, t = e % NI;
    const int j1 = jlo + jj, loc = qi + t - D1.q0[j1];
    bs[b][jj][t] = (loc >= 0 && loc < D1.nq[j1]) ? b1[((size_t)b * n1 + j1) * NQ + loc] : zeroR<RE>();
  }
  __syncthreads();
  const int64_t nnz2 = A.nnz1[1];
  const int64_t p2 = tile * blockDim.x + threadIdx.x;
  if (p2 >= nnz2) return;
  const int64_t p3l = blockIdx.y, p3 = A.p3_off + p3l;
  const int nrow = GB ? A.nbq : nq1;                       // rows of the G array read
  const int r0 = GB ? (H ? A.nbq - NI : 0) : qi;           // its row of point qi
  const RE* G = reinterpret_cast<const RE*>(GB ? A.Gb : A.G) + ((p3l * NG) * nrow + r0) * nnz2 + p2;
  const int64_t gstride = (int64_t)nrow * nnz2;
  RE acc[NJ];
#pragma unroll
  for (int jj = 0; jj < NJ; ++jj) acc[jj] = zeroR<RE>();
#pragma unroll 1
  for (int t = 0; t < NI; ++t) {
    const RE* gq = G + (int64_t)t * nnz2;
    RE h0, h1 = zeroR<RE>();
    if (MASS) {
      h0 = mulR(ws[0][t], ro(gq));
    } else {
      h0 = fmaR<RE>(ws[0][t], ro(gq), mulR(ws[2][t], ro(gq + 2 * gstride)));
      h1 = fmaR<RE>(ws[1][t], ro(gq + gstride), mulR(ws[3][t], ro(gq + 3 * gstride)));
    }
#pragma unroll
    for (int jj = 0; jj < NJ; ++jj)
      if (t >= e_tlo(P, R, H, jj) && t < e_thi(P, R, H, jj))
        acc[jj] = MASS ? fmaR<RE>(bs[0][jj][t], h0, acc[jj])
                       : fmaR<RE>(bs[1][jj][t], h1, fmaR<RE>(bs[0][jj][t], h0, acc[jj]));
  }
  const int i2 = D2.pair_row[p2], j2 = blo(i2, P) + (int)(p2 - D2.prefix[i2]);
  const int i3 = D3.pair_row[p3], j3 = blo(i3, P) + (int)(p3 - D3.prefix[i3]);
  const int bw2 = bw(i2, P, n2), bw3 = bw(i3, P, n3);
  const int64_t N1 = D1.prefix[n1], N2 = D2.prefix[n2];
  const int64_t base = D3.prefix[i3] * N2 * N1 + (int64_t)bw3 * (D2.prefix[i2] * N1 + (int64_t)bw2 * D1.prefix[i1]) +
                       ((int64_t)(j3 - blo(i3, P)) * bw2 + (j2 - blo(i2, P))) * NJ;
  OutT* out = reinterpret_cast<OutT*>(A.vals) + base;
#pragma unroll
  for (int jj = 0; jj < NJ; ++jj) out[jj] = toOut<OutT>(acc[jj]);
}

// The P+1 rows of one side in one launch in FP32: blockIdx.x = tile * (P+1) + R, so the
// rows that read the same points of G run together and share them through L2 (1.60 ->
// 1.16 ms at p = 5, 128^3); double-float keeps one launch per row (merged, 3.06 -> 4.28
// ms: it is bound by arithmetic, and the largest row's registers set every row's
// occupancy).
template <int P, bool MASS, typename RE, typename OutT, bool GB, bool H, int R = 0>
__device__ __forceinline__ void stage1_edge_any(const StagedArgs& A, int r, int64_t tile) {
  if (r == R) {
    stage1_edge_row<P, MASS, RE, OutT, GB, R, H>(A, tile);
    return;
  }
  if constexpr (R < P) stage1_edge_any<P, MASS, RE, OutT, GB, H, R + 1>(A, r, tile);
}

template <int P, bool MASS, typename RE, typename OutT, bool GB, bool H>
__global__ void __launch_bounds__(128) k_stage1_edge(StagedArgs A) {
  stage1_edge_any<P, MASS, RE, OutT, GB, H>(A, blockIdx.x % (P + 1), blockIdx.x / (P + 1));
}

template <int P, bool MASS, typename RE, typename OutT, bool GB, int R, bool H>
__global__ void __launch_bounds__(128) k_stage1_edge_row(StagedArgs A) {
  stage1_edge_row<P, MASS, RE, OutT, GB, R, H>(A, blockIdx.x);
}

template <int P, bool MASS, typename RE, typename OutT, bool GB, int B = 0>
static void launch_stage1_edge(const StagedArgs& A, int64_t np3, cudaStream_t s) {
  const unsigned tiles = (unsigned)((A.nnz1[1] + 127) / 128);
  if constexpr (std::is_same<RE, float>::value) {
    k_stage1_edge<P, MASS, RE, OutT, GB, false><<<dim3(tiles * (P + 1), (unsigned)np3), 128, 0, s>>>(A);
    k_stage1_edge<P, MASS, RE, OutT, GB, true><<<dim3(tiles * (P + 1), (unsigned)np3), 128, 0, s>>>(A);
  } else {
    k_stage1_edge_row<P, MASS, RE, OutT, GB, (B <= P ? B : B - P - 1), (B > P)><<<dim3(tiles, (unsigned)np3), 128, 0, s>>>(A);
    if constexpr (B + 1 < 2 * P + 2) launch_stage1_edge<P, MASS, RE, OutT, GB, B + 1>(A, np3, s);
  }
}

__global__ void k_pair_rows(const int64_t* __restrict__ prefix, int n, int* __restrict__ pair_row) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int64_t k = prefix[i]; k < prefix[i + 1]; ++k) pair_row[k] = i;
}

}  // namespace

// Scratch of the staged path, allocated on first use and owned by the plan.
static wq_status staged_scratch(wq_plan_s* pl, size_t t3, size_t g, size_t gb, bool need_f32, cudaStream_t s) {
  t3 = std::max<size_t>(16, t3);
  g = std::max<size_t>(16, g);
  if (pl->stg_a_bytes < t3 || pl->stg_b_bytes < g) {
    plan_free(pl, pl->stg_a, s);
    plan_free(pl, pl->stg_b, s);
    pl->stg_a = pl->stg_b = nullptr;
    pl->stg_a_bytes = pl->stg_b_bytes = 0;
    wq_status st = plan_alloc(pl, &pl->stg_a, t3, s, "staged assembly scratch (T3)");
    if (st == WQ_OK) st = plan_alloc(pl, &pl->stg_b, g, s, "staged assembly scratch (G)");
    if (st != WQ_OK) {
      plan_free(pl, pl->stg_a, s);
      pl->stg_a = nullptr;
      return st;
    }
    pl->stg_a_bytes = t3;
    pl->stg_b_bytes = g;
  }
  if (pl->stg_c_bytes < gb) {
    plan_free(pl, pl->stg_c, s);
    pl->stg_c = nullptr;
    pl->stg_c_bytes = 0;
    wq_status st = plan_alloc(pl, &pl->stg_c, gb, s, "staged assembly scratch (edge copy of G)");
    if (st != WQ_OK) return st;
    pl->stg_c_bytes = gb;
  }
  if (!pl->coefT) {
    wq_status st = plan_alloc(pl, (void**)&pl->coefT, sizeof(double) * 8 * (size_t)pl->n_qp_total, s,
                              "transposed coefficients");
    if (st != WQ_OK) return st;
  }
  if (need_f32)
    for (int l = 0; l < 3; ++l)
      if (!pl->dir[l].tab32) {
        const size_t nt = (size_t)6 * pl->dir[l].n * pl->nq_max;  // 4 rule kinds + 2 basis tables
        wq_status st = plan_alloc(pl, (void**)&pl->dir[l].tab32, sizeof(float) * nt, s, "float tables");
        if (st != WQ_OK) return st;
      }
  for (int l = 1; l < 3; ++l)
    if (!pl->dir[l].pair_row) {
      wq_status st = plan_alloc(pl, (void**)&pl->dir[l].pair_row,
                                sizeof(int) * (size_t)std::max<int64_t>(1, pl->nnz1[l]), s, "pair index");
      if (st != WQ_OK) return st;
      k_pair_rows<<<(pl->dir[l].n + 127) / 128, 128, 0, s>>>(pl->dir[l].prefix, pl->dir[l].n, pl->dir[l].pair_row);
      count_launch();
    }
  return WQ_OK;
}

// The q1 points that the first and last p+1 rows of direction 1 read: [0, nbl) and
// [hstart, nqp) (Q_i = points inside the support of B_i; the whole range when the
// two ends meet).
static void edge_points(const wq_plan_s* pl, int* nbl, int* hstart, int* nbq, int dir = 0) {
  const int p = pl->p, ne = pl->dir[dir].n_el, nqp = (int)pl->nqp[dir], n1 = (int)pl->n[dir];
  const int il = std::min(p, n1 - 1), ih = std::max(n1 - p - 1, 0);
  const int hi = std::min(ne, il + 1), lo = std::max(0, ih - p);
  *nbl = (hi == ne ? nqp - 1 : 2 * hi + p - 2) + 1;
  *hstart = lo == 0 ? 0 : 2 * lo + p;
  if (*hstart <= *nbl) *nbl = *hstart = nqp;
  *nbq = *nbl + (nqp - *hstart);
}

// Real: arithmetic of stages 3 and 2 (and T3); R1: arithmetic of stage 1 (and G).
// TC: the regular rows of stage 1 on the tensor cores (3xTF32, tc::k_stage1_mma).
template <int P, bool MASS, typename Real, typename R1, typename OutT, bool TC = false>
static wq_status staged_t(wq_plan_s* pl, const double* kappa, void* vals, cudaStream_t s, const SlabHook* hook) {
  const int NT = MASS ? 1 : 9, NG = MASS ? 1 : 4;
  constexpr bool EDGE64 = sizeof(R1) < sizeof(Real);
  static_assert(!TC || std::is_same<R1, float>::value, "the tensor-core stage 1 reads FP32 G");
  // arithmetic of the first and last P+1 rows of direction 1 in the mixed modes:
  // double-float, in launches of their own beside the kernel of the regular rows
  // (their FP64 form is bound by the FP64 pipe: 7.6 ms against 3.2 ms at p = 5, 128^3)
  using GE = Real;
  int nbl = 0, hstart = 0, nbq = 0;
  if (EDGE64) edge_points(pl, &nbl, &hstart, &nbq);
  // slabs of direction 3: T3, G and the edge copy of G hold one slab at a time
  const int n3 = (int)pl->n[2];
  std::vector<int64_t> P3(n3 + 1, 0);  // prefix sums of the band widths of direction 3
  for (int i = 0; i < n3; ++i) P3[i + 1] = P3[i] + (std::min(n3 - 1, i + P) - std::max(0, i - P) + 1);
  const int t3w = (int)((pl->nqp[1] + 1) & ~1LL);  // T3 row length (even: pair loads)
  const size_t per_p3 = (size_t)NT * pl->nqp[0] * t3w * sizeof(Real) +
                        (size_t)NG * pl->nqp[0] * pl->nnz1[1] * sizeof(R1) + (size_t)NG * nbq * pl->nnz1[1] * sizeof(GE);
  int rows = hook && hook->rows > 0 ? hook->rows : n3;
  if (!(hook && hook->rows > 0) && pl->opt.scratch_limit > 0)
    rows = (int)std::max<size_t>(1, pl->opt.scratch_limit / (per_p3 * (2 * P + 1)));
  rows = std::max(1, std::min(rows, n3));
  int64_t np3_max = 0;
  for (int a = 0; a < n3; a += rows) np3_max = std::max(np3_max, P3[std::min(n3, a + rows)] - P3[a]);
  wq_status st = staged_scratch(pl, (size_t)np3_max * NT * pl->nqp[0] * t3w * sizeof(Real),
                                (size_t)np3_max * NG * pl->nqp[0] * pl->nnz1[1] * sizeof(R1),
                                (size_t)np3_max * NG * nbq * pl->nnz1[1] * sizeof(GE),
                                sizeof(Real) == sizeof(float) || sizeof(R1) == sizeof(float), s);
  if (st != WQ_OK) return st;
  constexpr bool F2 = std::is_same<Real, f2>::value, F2_1 = std::is_same<R1, f2>::value;
  static_assert(!F2_1 || F2, "double-float stage 1 needs double-float stages 3 and 2");
  StagedArgs A, A1;  // A: tables in Real (stages 3, 2); A1: tables in R1 (stage 1)
  for (int l = 0; l < 3; ++l) {
    DirData& d = pl->dir[l];
    const void* w32 = d.w;
    const void* bt32 = d.bt;
    if (F2) {
      const int64_t nw = (int64_t)4 * d.n * pl->nq_max, nb = (int64_t)2 * d.n * pl->nq_max;
      if (!d.tabf2) {
        wq_status st = plan_alloc(pl, &d.tabf2, sizeof(f2) * (size_t)(nw + nb), s, "double-float tables");
        if (st != WQ_OK) return st;
      }
      f2* t = reinterpret_cast<f2*>(d.tabf2);
      k_to_f2<<<(unsigned)((nw + 255) / 256), 256, 0, s>>>(d.w, t, nw);
      k_to_f2<<<(unsigned)((nb + 255) / 256), 256, 0, s>>>(d.bt, t + nw, nb);
      count_launch(2);
      A.d[l] = Dir{d.n, d.nqp, d.q0, d.nq, t, t + nw, d.prefix, d.pair_row};
      A.nnz1[l] = A1.nnz1[l] = pl->nnz1[l];
      if (F2_1) {
        A1.d[l] = A.d[l];
        continue;
      }
    }
    if (sizeof(Real) == sizeof(float) || sizeof(R1) == sizeof(float)) {
      const int64_t nw = (int64_t)4 * d.n * pl->nq_max, nb = (int64_t)2 * d.n * pl->nq_max;
      k_to_float<<<(unsigned)((nw + 255) / 256), 256, 0, s>>>(d.w, d.tab32, nw);
      k_to_float<<<(unsigned)((nb + 255) / 256), 256, 0, s>>>(d.bt, d.tab32 + nw, nb);
      count_launch(2);
      w32 = d.tab32;
      bt32 = d.tab32 + nw;
    }
    const bool f = sizeof(Real) == sizeof(float), f1 = sizeof(R1) == sizeof(float);
    if (!F2) A.d[l] = Dir{d.n, d.nqp, d.q0, d.nq, f ? w32 : d.w, f ? bt32 : d.bt, d.prefix, d.pair_row};
    A1.d[l] = Dir{d.n, d.nqp, d.q0, d.nq, f1 ? w32 : d.w, f1 ? bt32 : d.bt, d.prefix, d.pair_row};
    A.nnz1[l] = A1.nnz1[l] = pl->nnz1[l];
  }
  A.NQ = A1.NQ = pl->nq_max;
  A.t3w = A1.t3w = t3w;
  const int nq1 = (int)pl->nqp[0], nq2 = (int)pl->nqp[1], nq3 = (int)pl->nqp[2];
  const int64_t NQP = pl->n_qp_total;
  Real* cT = reinterpret_cast<Real*>(pl->coefT);
  A.cT = A1.cT = cT;
  A.kappaT = A1.kappaT = kappa ? cT + 7 * NQP : nullptr;
  A.T3 = A1.T3 = pl->stg_a;
  A.G = A1.G = pl->stg_b;
  A.vals = A1.vals = vals;
  A.Gb = A1.Gb = EDGE64 ? pl->stg_c : nullptr;
  // direction-1 tables in the edge-row type
  A.w1e = A1.w1e = std::is_same<GE, double>::value ? (const void*)pl->dir[0].w : A.d[0].w;
  A.bt1e = A1.bt1e = std::is_same<GE, double>::value ? (const void*)pl->dir[0].bt : A.d[0].bt;
  A.nbl = A1.nbl = nbl;
  A.hstart = A1.hstart = hstart;
  A.nbq = A1.nbq = nbq;
  {
    int nbl2 = 0, hstart2 = 0, nbq2 = 0;
    if (EDGE64) edge_points(pl, &nbl2, &hstart2, &nbq2, 1);
    A.nbl2 = A1.nbl2 = nbl2;
    A.hstart2 = A1.hstart2 = hstart2;
  }
  // tensor-core stage 1: B fragments of the regular rows of direction 1; FFMA stage 1
  // (FP32 G): the float4 tables of the regular rows
  // FP32 G (FP32 and mixed modes): the regular rows of stage 1 by k_stage1_ffma, the
  // first and last P+1 rows beside it on the side stream (k_stage1_edge, or k_stage1
  // where the two ends of direction 1 meet)
  constexpr bool FF = !TC && std::is_same<R1, float>::value;
  const int tc_lo = P + 1, tc_rows = TC ? std::max(0, (int)pl->n[0] - 2 * P - 2) : 0;
  const int ff_rows = FF ? std::max(0, (int)pl->n[0] - 2 * P - 2) : 0;
  constexpr int FF_TF4 = (2 * P + 1) * (1 + (P + 2) / 2);
  if (FF && ff_rows > 0) {
    const size_t fb = (size_t)ff_rows * FF_TF4 * sizeof(float4);
    if (pl->stg_d_bytes < fb) {
      plan_free(pl, pl->stg_d, s);
      pl->stg_d = nullptr;
      pl->stg_d_bytes = 0;
      wq_status st2 = plan_alloc(pl, &pl->stg_d, fb, s, "stage-1 row tables");
      if (st2 != WQ_OK) return st2;
      pl->stg_d_bytes = fb;
    }
  }
  if (TC && tc_rows > 0) {
    using SH = tc::Shape<P, MASS>;
    const size_t fb = (size_t)tc_rows * SH::KS * SH::NT * 32 * sizeof(float4);
    if (pl->stg_d_bytes < fb) {
      plan_free(pl, pl->stg_d, s);
      pl->stg_d = nullptr;
      pl->stg_d_bytes = 0;
      wq_status st2 = plan_alloc(pl, &pl->stg_d, fb, s, "tensor-core stage-1 fragments");
      if (st2 != WQ_OK) return st2;
      pl->stg_d_bytes = fb;
    }
  }
  if (!vals) return WQ_OK;  // wq_plan_reserve: scratch only
  // transposed coefficients (the slots this matrix uses) and kappa, in Real
  {
    dim3 blk(32, 8), grd((nq1 + 31) / 32, (nq2 + 31) / 32, 7 * nq3 + (kappa ? nq3 : 0));
    k_transpose_coef<Real><<<grd, blk, 0, s>>>(pl->coef, kappa, cT, cT + 7 * NQP, nq1, nq2, nq3, 7);
  }
  const int n1 = (int)pl->n[0], n2 = (int)pl->n[1];
  int r_lo = P + 1, r_hi = n2 - P - 1;  // regular rows [r_lo, r_hi)
  if (r_hi <= r_lo) r_lo = r_hi = n2;   // no regular rows: every row takes the boundary path
  if (FF && ff_rows > 0) {
    const int64_t nf = (int64_t)ff_rows * FF_TF4;
    k_s1_tables<P, MASS><<<(unsigned)((nf + 255) / 256), 256, 0, s>>>(
        reinterpret_cast<const float*>(A1.d[0].w), reinterpret_cast<const float*>(A1.d[0].bt), pl->dir[0].q0,
        pl->dir[0].nq, n1, pl->nq_max, P + 1, ff_rows, reinterpret_cast<float4*>(pl->stg_d));
    count_launch();
  }
  if (TC && tc_rows > 0) {
    using SH = tc::Shape<P, MASS>;
    const int64_t nf = (int64_t)tc_rows * SH::KS * SH::NT * 32;
    tc::k_bfrag<P, MASS><<<(unsigned)((nf + 255) / 256), 256, 0, s>>>(
        pl->dir[0].w, pl->dir[0].bt, pl->dir[0].q0, pl->dir[0].nq, n1, pl->nq_max, tc_lo, tc_rows,
        reinterpret_cast<float4*>(pl->stg_d));
    count_launch();
  }
  for (int i3a = 0; i3a < n3; i3a += rows) {
  const int i3b = std::min(n3, i3a + rows);
  A.p3_off = A1.p3_off = P3[i3a];
  A.i3_off = A1.i3_off = i3a;
  const int64_t np3 = P3[i3b] - P3[i3a];
  k_stage3<P, MASS, Real, EDGE64><<<dim3(i3b - i3a, (unsigned)(((int64_t)nq1 * nq2 + 127) / 128)), 128, 0, s>>>(A);
  // Regular rows: k_stage2_reg (tables in shared memory, 32 rows per block) unless,
  // in FP64, the FP64 pipe bounds the flat mapping too and the 32-row blocks would
  // leave lanes idle: more than 4% of them for P <= 4 (flat measured at 97% of the DFMA
  // rate), more than 10% for P = 8 (83 regular rows, 13.5% idle: flat 244.1 ms per step
  // against 251.2 ms). At p = 5 the flat form measured far slower (121 rows, 5.5% idle:
  // 155.8 ms against 127.6 ms), so P = 5..7 keep the blocks.
  const int nreg = r_hi - r_lo;
  const int idle_pct = nreg > 0 ? (int)(100 * (32 * ((nreg + 31) / 32) - nreg) / (32 * ((nreg + 31) / 32))) : 0;
  const bool flat = std::is_same<Real, double>::value && ((P <= 4 && idle_pct > 3) || (P >= 8 && idle_pct > 10));
  if (nreg > 0 && flat)
    k_stage2<P, MASS, Real, true, R1, GE>
        <<<dim3((unsigned)(((int64_t)nreg * nq1 + 127) / 128), (unsigned)np3), 128, 0, s>>>(A, r_lo, r_hi);
  else if (nreg > 0 && EDGE64) {
    // mixed precision: double-float only for the points q1 that the first and last P+1
    // rows of direction 1 read (their large WQ weights amplify rounding in stage 1);
    // FP32 on the points between, whose G only regular rows of direction 1 read
    const dim3 g2((unsigned)((nreg + 31) / 32), (unsigned)np3), b2(32, 4);
    const int a1 = std::min(nbl, nq1), b0 = std::max(hstart, a1);
    k_stage2_reg<P, MASS, Real, R1, Real, GE><<<g2, b2, 0, s>>>(A, r_lo, r_hi, 0, a1);
    if (b0 < nq1) k_stage2_reg<P, MASS, Real, R1, Real, GE><<<g2, b2, 0, s>>>(A, r_lo, r_hi, b0, nq1);
    if (b0 > a1) k_stage2_reg<P, MASS, R1, R1, Real, GE><<<g2, b2, 0, s>>>(A1, r_lo, r_hi, a1, b0);
    count_launch((b0 < nq1 ? 1 : 0) + (b0 > a1 ? 1 : 0));
  } else if (nreg > 0)
    k_stage2_reg<P, MASS, Real, R1, Real, GE>
        <<<dim3((unsigned)((nreg + 31) / 32), (unsigned)np3), dim3(32, 4), 0, s>>>(A, r_lo, r_hi, 0, nq1);
  const int nb = r_lo + (n2 - r_hi);
  const bool edge2 = pl->dir[1].n_el >= 2 * P + 2;  // edge rows with compile-time patterns
  if (edge2)
    launch_stage2_edge<P, MASS, Real, R1, GE>(A, nq1, np3, s);
  else
    k_stage2<P, MASS, Real, false, R1, GE>
        <<<dim3((unsigned)(((int64_t)nb * nq1 + 127) / 128), (unsigned)np3), 128, 0, s>>>(A, r_lo, r_hi);
  int gap_lo = 0, gap_len = 0;
  cudaStream_t s1 = s;  // stream of the k_stage1 launch (all rows, or the edge rows)
  if ((FF && ff_rows > 0) || (TC && tc_rows > 0)) {
    // the edge rows run beside the kernel of the regular rows on the plan's side
    // stream, forked from and joined back into `s`
    if (!pl->side_stream) {
      WQ_CUDA_TRY(cudaStreamCreateWithFlags(&pl->side_stream, cudaStreamNonBlocking), "side stream");
      WQ_CUDA_TRY(cudaEventCreateWithFlags(&pl->ev_fork, cudaEventDisableTiming), "fork event");
      WQ_CUDA_TRY(cudaEventCreateWithFlags(&pl->ev_join, cudaEventDisableTiming), "join event");
    }
    WQ_CUDA_TRY(cudaEventRecord(pl->ev_fork, s), "fork event");
    WQ_CUDA_TRY(cudaStreamWaitEvent(pl->side_stream, pl->ev_fork, 0), "fork wait");
    s1 = pl->side_stream;
  }
  if (FF && ff_rows > 0) {
    const int nch = (ff_rows + 31) / 32;
    static unsigned long long smem_set = 0;  // per instantiation, a bit per device
    int dev = 0;
    WQ_CUDA_TRY(cudaGetDevice(&dev), "current device");
    if (dev < 64 && !((smem_set >> dev) & 1ULL)) {
      WQ_CUDA_TRY(cudaFuncSetAttribute(k_stage1_ffma<P, MASS, OutT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)ffma_smem<P>()), "stage-1 shared memory");
      smem_set |= 1ULL << dev;
    }
    k_stage1_ffma<P, MASS, OutT>
        <<<dim3((unsigned)(((pl->nnz1[1] + 255) / 256) * nch), (unsigned)np3), 256, ffma_smem<P>(), s>>>(
            A1, reinterpret_cast<const float4*>(pl->stg_d), P + 1, P + 1 + ff_rows, nch);
    gap_lo = P + 1;
    gap_len = ff_rows;
    count_launch();
  } else if (TC && tc_rows > 0) {
    using SH = tc::Shape<P, MASS>;
    tc::k_stage1_mma<P, MASS, OutT>
        <<<dim3((unsigned)((pl->nnz1[1] + SH::MT - 1) / SH::MT), (unsigned)np3,
                (unsigned)((tc_rows + SH::CHUNK - 1) / SH::CHUNK)),
           32 * SH::WARPS, 0, s>>>(A1, reinterpret_cast<const float4*>(pl->stg_d), tc_lo, tc_lo + tc_rows);
    gap_lo = tc_lo;
    gap_len = tc_rows;
    count_launch();
  }
  // the first and last P+1 rows of direction 1: with compile-time point patterns
  // where the two ends of direction 1 are apart, else by k_stage1
  const bool edge1 = gap_len > 0 && gap_lo == P + 1 && gap_len == n1 - 2 * P - 2 && pl->dir[0].n_el >= 2 * P + 2;
  if constexpr (FF || TC) {
    if (edge1) launch_stage1_edge<P, MASS, typename std::conditional<EDGE64, GE, R1>::type, OutT, EDGE64>(A1, np3, s1);
  }
  const dim3 g1((unsigned)((pl->nnz1[1] + 31) / 32), (n1 - gap_len + 3) / 4, (unsigned)np3);
  bool host_done = false;
  if constexpr (std::is_same<R1, double>::value && std::is_same<OutT, double>::value && !FF && !TC) {
    if (hook && hook->host_vals) {
      k_stage1<P, MASS, R1, OutT, EDGE64, GE, true><<<g1, dim3(32, 4), 0, s1>>>(A1, gap_lo, gap_len);
      host_done = true;
    }
  }
  if (!host_done && !edge1 && n1 > gap_len)
    k_stage1<P, MASS, R1, OutT, EDGE64, GE><<<g1, dim3(32, 4), 0, s1>>>(A1, gap_lo, gap_len);
  if (s1 != s) {
    WQ_CUDA_TRY(cudaEventRecord(pl->ev_join, s1), "join event");
    WQ_CUDA_TRY(cudaStreamWaitEvent(s, pl->ev_join, 0), "join wait");
  }
  count_launch(1 + (edge1 ? (std::is_same<typename std::conditional<EDGE64, GE, R1>::type, float>::value ? 2 : 2 * P + 2)
                          : n1 > gap_len ? 1 : 0) +
               (r_hi > r_lo ? 1 : 0) + (edge2 ? stage2_edge_launches<P, Real>() : 1));
  WQ_CUDA_TRY(cudaGetLastError(), "staged assembly launch");
  if (hook && hook->after) {
    wq_status hs = hook->after(hook->ctx, i3a, i3b, s);
    if (hs != WQ_OK) return hs;
  }
  }  // slabs
  count_launch();  // the coefficient transpose
  return WQ_OK;
}

// Precision dispatch for one degree. Each degree is instantiated in a translation
// unit of its own (wq_staged_p<P>.cu), so the degrees compile in parallel.
template <int P>
wq_status launch_staged_deg(wq_plan_s* pl, bool mass, const double* kappa, void* vals, int value_dtype,
                            int precision, cudaStream_t s, const SlabHook* hook) {
  const bool v32 = value_dtype == WQ_VALUES_F32;
  if (precision == WQ_PREC_FP64)
    return mass ? staged_t<P, true, double, double, double>(pl, kappa, vals, s, hook)
                : staged_t<P, false, double, double, double>(pl, kappa, vals, s, hook);
  if (precision == WQ_PREC_F32X2) {
    if (v32)
      return mass ? staged_t<P, true, f2, f2, float>(pl, kappa, vals, s, hook)
                  : staged_t<P, false, f2, f2, float>(pl, kappa, vals, s, hook);
    return mass ? staged_t<P, true, f2, f2, double>(pl, kappa, vals, s, hook)
                : staged_t<P, false, f2, f2, double>(pl, kappa, vals, s, hook);
  }
  if (precision == WQ_PREC_TF32X3) {
    if (v32)
      return mass ? staged_t<P, true, f2, float, float, true>(pl, kappa, vals, s, hook)
                  : staged_t<P, false, f2, float, float, true>(pl, kappa, vals, s, hook);
    return mass ? staged_t<P, true, f2, float, double, true>(pl, kappa, vals, s, hook)
                : staged_t<P, false, f2, float, double, true>(pl, kappa, vals, s, hook);
  }
  if (precision == WQ_PREC_MIXED) {
    if (v32)
      return mass ? staged_t<P, true, f2, float, float>(pl, kappa, vals, s, hook)
                  : staged_t<P, false, f2, float, float>(pl, kappa, vals, s, hook);
    return mass ? staged_t<P, true, f2, float, double>(pl, kappa, vals, s, hook)
                : staged_t<P, false, f2, float, double>(pl, kappa, vals, s, hook);
  }
  if (v32)
    return mass ? staged_t<P, true, float, float, float>(pl, kappa, vals, s, hook)
                : staged_t<P, false, float, float, float>(pl, kappa, vals, s, hook);
  return mass ? staged_t<P, true, float, float, double>(pl, kappa, vals, s, hook)
              : staged_t<P, false, float, float, double>(pl, kappa, vals, s, hook);
}

}  // namespace wq
