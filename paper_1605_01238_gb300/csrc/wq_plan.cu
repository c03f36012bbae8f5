// Plan set-up: everything of the WQ method that depends only on the mesh and the
// geometry, computed on the GPU.
//
//   k_gauss          Gauss-Legendre rule with p+1 points (double-double)
//   k_points         quadrature points (Remark on the choice of quadrature points)
//   k_qranges        Q_{l,i}: points inside the open support of B_i (Eq. (support))
//   k_basis_points   B and B' at the points (Algorithm 1, first loop)
//   k_gauss_basis    B and B' at the Gauss points of every span
//   k_integrals      exact integrals I^{(a,b)}_{l,i,j} (Eq. (integrals), Algorithm 1)
//   k_rules          minimum-norm WQ rules of four kinds (Eq. (exact), Algorithm 2)
//   k_prefix / k_row_ptr / k_cols   Kronecker-structured CSR pattern (Section 3)
//   k_coef           DF, det DF and c_lm = det DF (DF^{-1} DF^{-T})_lm (Eq. (coef_stiff))
//
// The univariate steps run in double-double arithmetic: the rule systems near
// the boundary are ill-conditioned at high degree (row-scaled condition numbers
// ~1e7 at p = 8), and float64 data alone would put errors of ~1e-9 into the
// weights. With double-double points, basis values, integrals and solves, every
// weight is rounded to float64 once, at the end.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "wq_internal.h"

namespace wq {

// ---------------------------------------------------------------------------
// Cox-de Boor recursion on one span, in double-double.
// s is the knot-vector index of the span start (xi_s <= x < xi_{s+1} for points
// of that span); the p+1 functions B_{s-p+t}, t = 0..p, are returned with their
// first derivatives, as the span's polynomial pieces evaluated at x.
__device__ void basis_dd(const double* xi, const dd* rc, int ld, int p, int s, dd x, dd* val, dd* der) {
  // rc[k * ld + j] = 1 / (xi_{j+k} - xi_j) (zero for a repeated knot), see k_recips
  dd cur[kMaxP + 1], nxt[kMaxP + 1], low[kMaxP + 1];
  cur[0] = dd_make(1.0);
  for (int k = 1; k <= p; ++k) {
    for (int t = 0; t <= k; ++t) {
      int j = s - k + t;
      dd v = dd_make(0.0);
      if (t >= 1)  // (x - xi_j)/(xi_{j+k} - xi_j) B_{j,k-1}
        v = dd_add(v, dd_mul(dd_mul(dd_sub(x, dd_make(xi[j])), rc[k * ld + j]), cur[t - 1]));
      if (t <= k - 1)  // (xi_{j+k+1} - x)/(xi_{j+k+1} - xi_{j+1}) B_{j+1,k-1}
        v = dd_add(v, dd_mul(dd_mul(dd_sub(dd_make(xi[j + k + 1]), x), rc[k * ld + j + 1]), cur[t]));
      nxt[t] = v;
    }
    if (k == p)
      for (int t = 0; t < p; ++t) low[t] = cur[t];
    for (int t = 0; t <= k; ++t) cur[t] = nxt[t];
  }
  for (int t = 0; t <= p; ++t) {
    val[t] = cur[t];
    int j = s - p + t;
    dd d = dd_make(0.0);
    if (t >= 1) d = dd_add(d, dd_mul_d(dd_mul(low[t - 1], rc[p * ld + j]), (double)p));
    if (t <= p - 1) d = dd_sub(d, dd_mul_d(dd_mul(low[t], rc[p * ld + j + 1]), (double)p));
    der[t] = d;
  }
}

// Reciprocals of the knot differences: rc[k * ld + j] = 1/(xi_{j+k} - xi_j),
// k = 1..p, j = 0..n+p-k, in double-double (zero where the knots coincide).
__global__ void k_recips(const double* __restrict__ xi, int n, int p, int ld, dd* __restrict__ rc) {
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  const int len = n + p + 1;
  if (id >= p * ld) return;
  const int k = 1 + id / ld, j = id % ld;
  dd v = dd_make(0.0);
  if (j + k < len) {
    dd d = two_sum(xi[j + k], -xi[j]);
    if (d.hi != 0.0) v = dd_div(dd_make(1.0), d);
  }
  rc[k * ld + j] = v;
}

// Legendre P_m and P_{m-1} at x by the three-term recurrence, double-double.
__device__ void legendre_dd(int m, dd x, dd* pm, dd* pm1) {
  dd a = dd_make(1.0), b = x;
  for (int j = 1; j < m; ++j) {
    dd c = dd_sub(dd_mul_d(dd_mul(x, b), (double)(2 * j + 1)), dd_mul_d(a, (double)j));
    c = dd_div(c, dd_make((double)(j + 1)));
    a = b;
    b = c;
  }
  *pm = b;
  *pm1 = a;
}

// m-point Gauss-Legendre nodes g[k] and weights g[m+k] on [-1, 1].
__global__ void k_gauss(dd* g, int m) {
  int k = threadIdx.x;
  if (k >= m) return;
  double x = cos(M_PI * (k + 0.75) / (m + 0.5));
  for (int it = 0; it < 8; ++it) {  // Newton in double from the asymptotic guess
    double a = 1.0, b = x;
    for (int j = 1; j < m; ++j) {
      double c = ((2 * j + 1) * x * b - j * a) / (j + 1);
      a = b;
      b = c;
    }
    double dp = m * (x * b - a) / (x * x - 1.0);
    x -= b / dp;
  }
  dd X = dd_make(x), pm, pm1, dp;
  for (int it = 0; it < 3; ++it) {  // Newton in double-double
    legendre_dd(m, X, &pm, &pm1);
    dd x2m1 = dd_sub(dd_mul(X, X), dd_make(1.0));
    dp = dd_div(dd_mul_d(dd_sub(dd_mul(X, pm), pm1), (double)m), x2m1);
    X = dd_sub(X, dd_div(pm, dp));
  }
  legendre_dd(m, X, &pm, &pm1);
  dd x2m1 = dd_sub(dd_mul(X, X), dd_make(1.0));
  dp = dd_div(dd_mul_d(dd_sub(dd_mul(X, pm), pm1), (double)m), x2m1);
  // w = 2 / ((1 - x^2) P'_m(x)^2)
  dd den = dd_mul(dd_neg(x2m1), dd_mul(dp, dp));
  g[k] = X;
  g[m + k] = dd_div(dd_make(2.0), den);
}

struct DirArgs {
  int p, n, n_el, nqp, nq_stride;
  const double* knots;
  double* x;
  dd* x_dd;
  int* first;
  int* q0;
  int* nq;
  dd* bt_dd;
  double* bt;
  double* bp;
  dd* gb;
  dd* integ;
  double* w;
  int64_t* prefix;
  dd* greville;
  const dd* gauss;
  const dd* recip;  // [p+1][n+p+1] knot-difference reciprocals
  int* err;
};

// The three directions of a plan, one launch for all of them (blockIdx.y, or
// blockIdx.z for k_rules, selects the direction; gridDim covers the largest).
struct DirArgs3 {
  DirArgs d[3];
};

static DirArgs dir_args(wq_plan_s* pl, int l) {
  DirData& d = pl->dir[l];
  DirArgs a;
  a.p = pl->p;
  a.n = d.n;
  a.n_el = d.n_el;
  a.nqp = d.nqp;
  a.nq_stride = pl->nq_max;
  a.knots = d.knots;
  a.x = d.x;
  a.x_dd = d.x_dd;
  a.first = d.first;
  a.q0 = d.q0;
  a.nq = d.nq;
  a.bt_dd = d.bt_dd;
  a.bt = d.bt;
  a.bp = d.bp;
  a.gb = d.gb;
  a.integ = d.integ;
  a.w = d.w;
  a.prefix = d.prefix;
  a.greville = d.greville;
  a.recip = d.recip;
  a.gauss = pl->gauss;
  a.err = pl->err;
  return a;
}

// Points: p+1 equally spaced points strictly inside each boundary span,
// x = a + k (b - a)/(p + 2), k = 1..p+1; knots and midpoints elsewhere.
__global__ void k_points(DirArgs3 A) {
  const DirArgs& a = A.d[blockIdx.y];
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= a.nqp) return;
  const double* chi = a.knots + a.p;  // distinct knots chi_0..chi_{n_el}
  const int p = a.p, ne = a.n_el;
  dd x;
  int first;
  if (q <= p || q >= 2 * ne + p - 2) {
    int span = q <= p ? 0 : ne - 1;
    int k = q <= p ? q + 1 : q - (2 * ne + p - 2) + 1;
    dd h = two_sum(chi[span + 1], -chi[span]);
    x = dd_add(dd_make(chi[span]), dd_div(dd_mul_d(h, (double)k), dd_make((double)(p + 2))));
    first = span;
  } else {
    int t = q - p - 1;
    int k = 1 + t / 2;
    if ((t & 1) == 0) {
      x = dd_make(chi[k]);
    } else {
      dd s = two_sum(chi[k], chi[k + 1]);
      x = dd{0.5 * s.hi, 0.5 * s.lo};
    }
    first = k;
  }
  a.x_dd[q] = x;
  a.x[q] = dd_to_d(x);
  a.first[q] = first;
}

// Q_i = points strictly inside (chi_{max(0,i-p)}, chi_{min(n_el,i+1)}).
__global__ void k_qranges(DirArgs3 A) {
  const DirArgs& a = A.d[blockIdx.y];
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  int lo = max(0, i - a.p), hi = min(a.n_el, i + 1);
  int qs = lo == 0 ? 0 : 2 * lo + a.p;
  int qe = hi == a.n_el ? a.nqp - 1 : 2 * hi + a.p - 2;
  a.q0[i] = qs;
  a.nq[i] = qe - qs + 1;
}

__global__ void k_basis_points(DirArgs3 A) {
  const DirArgs& a = A.d[blockIdx.y];
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= a.nqp) return;
  const int p = a.p;
  int f = a.first[q];
  dd val[kMaxP + 1], der[kMaxP + 1];
  basis_dd(a.knots, a.recip, a.n + p + 1, p, f + p, a.x_dd[q], val, der);
  for (int t = 0; t <= p; ++t) {
    a.bp[(0 * a.nqp + q) * (p + 1) + t] = dd_to_d(val[t]);
    a.bp[(1 * a.nqp + q) * (p + 1) + t] = dd_to_d(der[t]);
    int j = f + t;
    int loc = q - a.q0[j];
    if (loc >= 0 && loc < a.nq[j]) {
      size_t i0 = ((size_t)0 * a.n + j) * a.nq_stride + loc;
      size_t i1 = ((size_t)1 * a.n + j) * a.nq_stride + loc;
      a.bt_dd[i0] = val[t];
      a.bt_dd[i1] = der[t];
      a.bt[i0] = dd_to_d(val[t]);
      a.bt[i1] = dd_to_d(der[t]);
    }
  }
}

// Basis at the p+1 Gauss points of every span: gb[span][g][b][t].
__global__ void k_gauss_basis(DirArgs3 A) {
  const DirArgs& a = A.d[blockIdx.y];
  int id = blockIdx.x * blockDim.x + threadIdx.x;
  const int p = a.p, m = p + 1;
  if (id >= a.n_el * m) return;
  int span = id / m, g = id % m;
  const double* chi = a.knots + p;
  dd mid = two_sum(chi[span], chi[span + 1]);
  mid = dd{0.5 * mid.hi, 0.5 * mid.lo};
  dd half = two_sum(chi[span + 1], -chi[span]);
  half = dd{0.5 * half.hi, 0.5 * half.lo};
  dd x = dd_add(mid, dd_mul(half, a.gauss[g]));
  dd val[kMaxP + 1], der[kMaxP + 1];
  basis_dd(a.knots, a.recip, a.n + p + 1, p, span + p, x, val, der);
  dd* out = a.gb + ((size_t)span * m + g) * 2 * m;
  for (int t = 0; t <= p; ++t) {
    out[t] = val[t];
    out[m + t] = der[t];
  }
}

// I^{(a,b)}_{i,j} for j = i - p + t by Gauss on the common spans, one thread per
// (i, t, kind = 2a + b): the double-double chains are short and spread over many SMs.
__global__ void k_integrals(DirArgs3 A) {
  const DirArgs& a = A.d[blockIdx.y];
  int id = blockIdx.x * blockDim.x + threadIdx.x;
  const int p = a.p, m = p + 1, bw = 2 * p + 1;
  if (id >= a.n * bw * 4) return;
  const int kind = id & 3;
  id >>= 2;
  const int i = id / bw, t = id % bw;
  const int j = i - p + t;
  const int ta = kind >> 1, tb = kind & 1;
  dd acc = dd_make(0.0);
  if (j >= 0 && j < a.n) {
    const double* chi = a.knots + p;
    int k0 = max(max(i, j) - p, 0), k1 = min(min(i, j), a.n_el - 1);
    for (int k = k0; k <= k1; ++k) {
      dd half = two_sum(chi[k + 1], -chi[k]);
      half = dd{0.5 * half.hi, 0.5 * half.lo};
      const dd* gbk = a.gb + (size_t)k * m * 2 * m;
      for (int g = 0; g < m; ++g) {
        const dd* row = gbk + (size_t)g * 2 * m;
        dd wi = dd_mul(dd_mul(a.gauss[m + g], half), row[ta * m + i - k]);
        acc = dd_add(acc, dd_mul(wi, row[tb * m + j - k]));
      }
    }
  }
  a.integ[((size_t)kind * a.n + i) * bw + t] = acc;
}

// Minimum-norm rule of kind (a,b) for test function i: one warp per system.
// Rows (j in I_i) are scaled by powers of two (exact, solution set unchanged);
// the normal equations (M M^T) y = r are solved by LDL^T and w = M^T y. For
// b = 1 the rows of M sum to zero and r is consistent; the rank-one term
// sigma u u^T with u = D^{-1} 1 (the left null vector of the scaled matrix)
// makes the system definite without changing w.
__global__ void k_rules(DirArgs3 A) {
  const DirArgs& a = A.d[blockIdx.z];
  const int i = blockIdx.x, kind = blockIdx.y;
  if (i >= a.n) return;
  const int ka = kind >> 1, kb = kind & 1;
  const int lane = threadIdx.x;
  const int p = a.p, bw = 2 * p + 1;
  __shared__ dd M[kMaxI][kMaxQ];
  __shared__ dd G[kMaxI][kMaxI];
  __shared__ dd r[kMaxI], y[kMaxI], Dg[kMaxI];
  __shared__ double scale[kMaxI];
  __shared__ int bad;
  const int jlo = max(0, i - p), jhi = min(a.n - 1, i + p);
  const int m = jhi - jlo + 1;
  const int q0i = a.q0[i], nqi = a.nq[i];
  if (lane == 0) bad = 0;
  for (int e = lane; e < m * nqi; e += 32) {
    int rr = e / nqi, c = e % nqi;
    int j = jlo + rr, q = q0i + c;
    int loc = q - a.q0[j];
    dd v = dd_make(0.0);
    if (loc >= 0 && loc < a.nq[j]) v = a.bt_dd[((size_t)kb * a.n + j) * a.nq_stride + loc];
    M[rr][c] = v;
  }
  for (int rr = lane; rr < m; rr += 32) r[rr] = a.integ[((size_t)kind * a.n + i) * bw + (jlo + rr - i + p)];
  __syncwarp();
  for (int rr = lane; rr < m; rr += 32) {
    double mx = 0.0;
    for (int c = 0; c < nqi; ++c) mx = fmax(mx, fabs(M[rr][c].hi));
    double s = mx > 0.0 ? ldexp(1.0, -ilogb(mx)) : 0.0;
    if (!(mx > 0.0)) atomicOr(a.err, kErrSingularRule);
    scale[rr] = s;
    for (int c = 0; c < nqi; ++c) M[rr][c] = dd{M[rr][c].hi * s, M[rr][c].lo * s};
    r[rr] = dd{r[rr].hi * s, r[rr].lo * s};
  }
  __syncwarp();
  for (int e = lane; e < m * m; e += 32) {
    int rr = e / m, ss = e % m;
    if (ss > rr) continue;
    dd acc = dd_make(0.0);
    for (int c = 0; c < nqi; ++c) acc = dd_add(acc, dd_mul(M[rr][c], M[ss][c]));
    G[rr][ss] = acc;
    G[ss][rr] = acc;
  }
  __syncwarp();
  if (kb == 1) {  // G += sigma u u^T, u = D^{-1} 1 (the left null vector of the scaled system)
    __shared__ dd sig_s;
    if (lane == 0) {
      dd tr = dd_make(0.0), un = dd_make(0.0);
      for (int rr = 0; rr < m; ++rr) {
        tr = dd_add(tr, G[rr][rr]);
        double u = 1.0 / scale[rr];  // exact: scale is a power of two
        un = dd_add(un, dd_mul_d(dd_make(u), u));
      }
      sig_s = dd_div(tr, dd_mul_d(un, (double)m));
    }
    __syncwarp();
    const dd sig = sig_s;
    for (int e = lane; e < m * m; e += 32) {
      const int rr = e / m, ss = e % m;
      G[rr][ss] = dd_add(G[rr][ss], dd_mul_d(dd_mul_d(sig, 1.0 / scale[rr]), 1.0 / scale[ss]));
    }
  }
  __syncwarp();
  // Right-looking LDL^T: at column c every lane updates part of the trailing block.
  // L is stored in the strict lower triangle of G, D in Dg.
  double gmax = 0.0;
  for (int rr = 0; rr < m; ++rr) gmax = fmax(gmax, G[rr][rr].hi);
  __shared__ dd col[kMaxI];
  for (int c = 0; c < m; ++c) {
    const dd d = G[c][c];
    if (lane == 0) {
      Dg[c] = d;
      if (!(d.hi > 1e-28 * gmax)) bad = 1;
    }
    for (int rr = c + 1 + lane; rr < m; rr += 32) col[rr] = G[rr][c];
    __syncwarp();
    for (int rr = c + 1 + lane; rr < m; rr += 32) G[rr][c] = dd_div(col[rr], d);
    __syncwarp();
    const int t = m - c - 1;  // trailing block (c, m) x (c, m), lower triangle
    for (int e = lane; e < t * t; e += 32) {
      const int rr = c + 1 + e / t, ss = c + 1 + e % t;
      if (ss <= rr) G[rr][ss] = dd_sub(G[rr][ss], dd_mul(G[rr][c], col[ss]));
    }
    __syncwarp();
  }
  if (lane == 0 && bad) atomicOr(a.err, kErrSingularRule);
  // L z = r, z /= D, L^T y = z: column by column, rows in parallel
  for (int rr = lane; rr < m; rr += 32) y[rr] = r[rr];
  __syncwarp();
  for (int k = 0; k < m; ++k) {
    const dd yk = y[k];
    for (int rr = k + 1 + lane; rr < m; rr += 32) y[rr] = dd_sub(y[rr], dd_mul(G[rr][k], yk));
    __syncwarp();
  }
  for (int rr = lane; rr < m; rr += 32) y[rr] = dd_div(y[rr], Dg[rr]);
  __syncwarp();
  for (int k = m - 1; k > 0; --k) {
    const dd yk = y[k];
    for (int rr = lane; rr < k; rr += 32) y[rr] = dd_sub(y[rr], dd_mul(G[k][rr], yk));
    __syncwarp();
  }
  __syncwarp();
  double* wout = a.w + ((size_t)kind * a.n + i) * a.nq_stride;
  for (int c = lane; c < a.nq_stride; c += 32) {
    if (c < nqi) {
      dd acc = dd_make(0.0);
      for (int rr = 0; rr < m; ++rr) acc = dd_add(acc, dd_mul(M[rr][c], y[rr]));
      wout[c] = dd_to_d(acc);
    } else {
      wout[c] = 0.0;
    }
  }
  (void)ka;
}

// Prefix sums of the band widths |I_i| = min(n-1, i+p) - max(0, i-p) + 1.
__global__ void k_prefix(DirArgs3 A) {
  const DirArgs& a = A.d[blockIdx.y];
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int64_t s = 0;
  for (int i = 0; i < a.n; ++i) {
    a.prefix[i] = s;
    s += min(a.n - 1, i + a.p) - max(0, i - a.p) + 1;
  }
  a.prefix[a.n] = s;
}

// Greville abscissae g_i = (xi_{i+1} + ... + xi_{i+p}) / p, double-double.
__global__ void k_greville(DirArgs3 A) {
  const DirArgs& a = A.d[blockIdx.y];
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  dd s = dd_make(0.0);
  for (int k = 1; k <= a.p; ++k) s = dd_add(s, dd_make(a.knots[i + k]));
  a.greville[i] = dd_div(s, dd_make((double)a.p));
}

struct PatternArgs {
  int p;
  int n1, n2, n3;
  const int64_t *P1, *P2, *P3;
  int64_t* row_ptr;
  int32_t* col;
};

__device__ inline int band_lo(int i, int p) { return max(0, i - p); }
__device__ inline int band_w(int i, int p, int n) { return min(n - 1, i + p) - max(0, i - p) + 1; }

// row_ptr(i1,i2,i3) = P3(i3) N2 N1 + bw3(i3) (P2(i2) N1 + bw2(i2) P1(i1)).
__global__ void k_row_ptr(PatternArgs a) {
  int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t N = (int64_t)a.n1 * a.n2 * a.n3;
  if (r > N) return;
  int64_t N1 = a.P1[a.n1], N2 = a.P2[a.n2];
  if (r == N) {
    a.row_ptr[N] = a.P3[a.n3] * N2 * N1;
    return;
  }
  int i1 = (int)(r % a.n1);
  int i2 = (int)((r / a.n1) % a.n2);
  int i3 = (int)(r / ((int64_t)a.n1 * a.n2));
  a.row_ptr[r] = a.P3[i3] * N2 * N1 +
                 (int64_t)band_w(i3, a.p, a.n3) * (a.P2[i2] * N1 + (int64_t)band_w(i2, a.p, a.n2) * a.P1[i1]);
}

// Column indices: one warp per row, ascending j1 + n1 (j2 + n2 j3). Each lane
// walks its entries e = lane, lane + 32, ... keeping (t1, t2, t3) up to date by
// carries; N_DOF < 2^31, so the column arithmetic stays in 32 bits.
// Rows whose band is full in all three directions (every row away from the
// boundary) share one pattern of column offsets, t1 + n1 t2 + n1 n2 t3 in
// lexicographic order of (t3, t2, t1): it sits in shared memory (dynamic, (2p+1)^3
// ints), so such a row costs a load, an add and a store per column.
__global__ void k_cols(PatternArgs a) {
  extern __shared__ int tmpl[];
  const int64_t N = (int64_t)a.n1 * a.n2 * a.n3;
  const int lane = threadIdx.x & 31;
  int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int n12 = a.n1 * a.n2;
  const int BW = 2 * a.p + 1, full = BW * BW * BW;
  for (int e = threadIdx.x; e < full; e += blockDim.x)
    tmpl[e] = e % BW + a.n1 * ((e / BW) % BW) + n12 * (e / (BW * BW));
  __syncthreads();
  for (int64_t r = warp; r < N; r += nwarps) {
    const int rr = (int)r;
    const int i1 = rr % a.n1, i2 = (rr / a.n1) % a.n2, i3 = rr / n12;
    const int w1 = band_w(i1, a.p, a.n1), w2 = band_w(i2, a.p, a.n2), w3 = band_w(i3, a.p, a.n3);
    const int c0 = band_lo(i1, a.p) + a.n1 * band_lo(i2, a.p) + n12 * band_lo(i3, a.p);
    int32_t* out = a.col + a.row_ptr[r];
    const int cnt = w1 * w2 * w3;
    if (cnt == full) {
      for (int e = lane; e < full; e += 32) out[e] = c0 + tmpl[e];
      continue;
    }
    int t1 = lane % w1, rest = lane / w1;
    int t2 = rest % w2, t3 = rest / w2;
    const int s1 = 32 % w1, c1 = 32 / w1;        // step of 32 entries: +s1 in t1, +c1 carried to t2
    const int s2 = c1 % w2, c2 = c1 / w2;
    for (int e = lane; e < cnt; e += 32) {
      out[e] = c0 + t1 + a.n1 * t2 + n12 * t3;
      t1 += s1;
      int k2 = s2, k3 = c2;
      if (t1 >= w1) { t1 -= w1; ++k2; }
      t2 += k2;
      if (t2 >= w2) { t2 -= w2; ++k3; }
      t3 += k3;
    }
  }
}

// ---------------------------------------------------------------------------
// Coefficients. The tensor-product B-splines reproduce linear functions with
// the Greville points g_i as coefficients (zeta = sum_i g_i B_i(zeta)), so
//   F(zeta) = zeta + sum_i (C_i - g_i) B_i(zeta),  DF = I + sum_i (C_i - g_i) x grad B_i.
// Summing the small differences C_i - g_i instead of C_i keeps the O(1/h) terms
// C_i x grad B_i, which cancel to O(1), out of the rounded sum: DF then carries
// an absolute error of a few ulp of |C - g| instead of ulp(1)/h.
//
// k_delta forms C_i - g_i in double-double and rounds once. k_coef runs one
// block per (q3, tile of TQ2 q2-points, tile of TQ1 q1-points) and
// sum-factorises DF over the tile: contract i3, then i2, then i1.
struct DeltaArgs {
  int n1, n2, n3;
  const double* ctrl;
  const dd *g1, *g2, *g3;
  double* delta;
};

__global__ void k_delta(DeltaArgs a) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t N = (int64_t)a.n1 * a.n2 * a.n3;
  if (i >= N) return;
  int i1 = (int)(i % a.n1), i2 = (int)((i / a.n1) % a.n2), i3 = (int)(i / ((int64_t)a.n1 * a.n2));
  const dd g[3] = {a.g1[i1], a.g2[i2], a.g3[i3]};
  for (int r = 0; r < 3; ++r) a.delta[i * 3 + r] = dd_to_d(dd_sub(dd_make(a.ctrl[i * 3 + r]), g[r]));
}

constexpr int kCoefTQ1 = 32, kCoefTQ2 = 8;

struct CoefArgs {
  int p;
  int n1, n2, n3, nq1, nq2, nq3;
  const double* ctrl;   // C_i - g_i (see k_delta); the control points C_i for a rational map
  const double *bp1, *bp2, *bp3;
  const int *f1, *f2, *f3;
  double* coef;
  double* jac;  // NULL, or [9][N_QP]: DF_{rc} at (3r + c)
  int64_t nqp_total;
  int* err;
  const double* K;        // NULL (identity), or [6][N_QP]: K11 K12 K13 K22 K23 K33 at the points
  const double* weights;  // rational map only: w_i [N_DOF]
  int nurbs_basis;        // rational map only: c = det DF / W^2 (NURBS basis functions)
};

// From DF at point qg: c_lm = det DF (DF^{-1} K DF^{-T})_lm = (adj K adj^T)_lm / det DF
// (Eq. (coef_stiff) with the coefficient tensor K, the identity when a.K is NULL),
// and c = det DF * mass_scale (Eq. (mass2)).
__device__ void write_coefficients(const CoefArgs& a, const double (&F)[3][3], int64_t qg, double mass_scale) {
  if (a.jac)
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) a.jac[(3 * r + c) * a.nqp_total + qg] = F[r][c];
  // adj = det * DF^{-1}: adj[l][k] = cofactor[k][l]
  double adj[3][3];
  adj[0][0] = F[1][1] * F[2][2] - F[1][2] * F[2][1];
  adj[0][1] = F[0][2] * F[2][1] - F[0][1] * F[2][2];
  adj[0][2] = F[0][1] * F[1][2] - F[0][2] * F[1][1];
  adj[1][0] = F[1][2] * F[2][0] - F[1][0] * F[2][2];
  adj[1][1] = F[0][0] * F[2][2] - F[0][2] * F[2][0];
  adj[1][2] = F[0][2] * F[1][0] - F[0][0] * F[1][2];
  adj[2][0] = F[1][0] * F[2][1] - F[1][1] * F[2][0];
  adj[2][1] = F[0][1] * F[2][0] - F[0][0] * F[2][1];
  adj[2][2] = F[0][0] * F[1][1] - F[0][1] * F[1][0];
  double det = F[0][0] * adj[0][0] + F[0][1] * adj[1][0] + F[0][2] * adj[2][0];
  if (!(det > 0.0) || !isfinite(det)) atomicOr(a.err, kErrBadGeometry);
  double inv = 1.0 / det;
  const int L[6] = {0, 0, 0, 1, 1, 2}, Mi[6] = {0, 1, 2, 1, 2, 2};
  if (a.K) {
    double Km[3][3];
    for (int s = 0; s < 6; ++s) Km[L[s]][Mi[s]] = Km[Mi[s]][L[s]] = a.K[(int64_t)s * a.nqp_total + qg];
    double AK[3][3];  // adj K
    for (int l = 0; l < 3; ++l)
      for (int b = 0; b < 3; ++b) AK[l][b] = adj[l][0] * Km[0][b] + adj[l][1] * Km[1][b] + adj[l][2] * Km[2][b];
    for (int s = 0; s < 6; ++s) {
      int l = L[s], mm = Mi[s];
      double v = AK[l][0] * adj[mm][0] + AK[l][1] * adj[mm][1] + AK[l][2] * adj[mm][2];
      a.coef[(int64_t)s * a.nqp_total + qg] = v * inv;
    }
  } else {
    for (int s = 0; s < 6; ++s) {
      int l = L[s], mm = Mi[s];
      double v = adj[l][0] * adj[mm][0] + adj[l][1] * adj[mm][1] + adj[l][2] * adj[mm][2];
      a.coef[(int64_t)s * a.nqp_total + qg] = v * inv;
    }
  }
  a.coef[6 * a.nqp_total + qg] = det * mass_scale;
}

__global__ void k_coef(CoefArgs a) {
  extern __shared__ double sm[];
  const int p = a.p, m = p + 1;
  const int nt1 = (a.nq1 + kCoefTQ1 - 1) / kCoefTQ1;
  int bid = blockIdx.x;
  const int tq1 = bid % nt1;
  bid /= nt1;
  const int nt2 = (a.nq2 + kCoefTQ2 - 1) / kCoefTQ2;
  const int tq2 = bid % nt2;
  const int q3 = bid / nt2;
  const int qa1 = tq1 * kCoefTQ1, qb1 = min(a.nq1, qa1 + kCoefTQ1);
  const int qa2 = tq2 * kCoefTQ2, qb2 = min(a.nq2, qa2 + kCoefTQ2);
  const int ia1 = a.f1[qa1], ib1 = a.f1[qb1 - 1] + p + 1;  // i1 window [ia1, ib1)
  const int ia2 = a.f2[qa2], ib2 = a.f2[qb2 - 1] + p + 1;
  const int W1 = ib1 - ia1, W2 = ib2 - ia2;
  const int f3 = a.f3[q3];
  double* X = sm;                       // [2][W2][W1][3]
  double* Y = X + 2 * W2 * W1 * 3;      // [3][TQ2][W1][3]
  const int nthr = blockDim.x;
  // A: X[d3][i2][i1][r] = sum_t3 B3^{(d3)}(q3, t3) C[i1, i2, f3 + t3][r]
  for (int e = threadIdx.x; e < 2 * W2 * W1 * 3; e += nthr) {
    int rr = e % 3, i1 = (e / 3) % W1, i2 = (e / (3 * W1)) % W2, d3 = e / (3 * W1 * W2);
    double acc = 0.0;
    for (int t = 0; t < m; ++t) {
      int64_t idx = ((int64_t)(f3 + t) * a.n2 + (ia2 + i2)) * a.n1 + (ia1 + i1);
      acc = fma(a.bp3[((int64_t)d3 * a.nq3 + q3) * m + t], a.ctrl[idx * 3 + rr], acc);
    }
    X[e] = acc;
  }
  __syncthreads();
  // B: Y[e][q2][i1][r], e = (d2,d3) in {(0,0), (1,0), (0,1)}
  const int nq2t = qb2 - qa2;
  for (int e = threadIdx.x; e < 3 * nq2t * W1 * 3; e += nthr) {
    int rr = e % 3, i1 = (e / 3) % W1, q2l = (e / (3 * W1)) % nq2t, kind = e / (3 * W1 * nq2t);
    int d2 = kind == 1, d3 = kind == 2;
    int q2 = qa2 + q2l, f2 = a.f2[q2];
    double acc = 0.0;
    for (int t = 0; t < m; ++t)
      acc = fma(a.bp2[((int64_t)d2 * a.nq2 + q2) * m + t], X[((d3 * W2 + (f2 + t - ia2)) * W1 + i1) * 3 + rr], acc);
    Y[((kind * kCoefTQ2 + q2l) * W1 + i1) * 3 + rr] = acc;
  }
  __syncthreads();
  const int nq1t = qb1 - qa1;
  for (int e = threadIdx.x; e < nq2t * nq1t; e += nthr) {
    int q1l = e % nq1t, q2l = e / nq1t;
    int q1 = qa1 + q1l, q2 = qa2 + q2l;
    int f1 = a.f1[q1];
    double F[3][3];
    for (int c = 0; c < 3; ++c) {
      int d1 = c == 0;
      const double* Yk = Y + ((c * kCoefTQ2 + q2l) * W1) * 3;
      for (int rr = 0; rr < 3; ++rr) {
        double acc = 0.0;
        for (int t = 0; t < m; ++t)
          acc = fma(a.bp1[((int64_t)d1 * a.nq1 + q1) * m + t], Yk[(f1 + t - ia1) * 3 + rr], acc);
        F[rr][c] = acc + (rr == c ? 1.0 : 0.0);  // dF_r / dzeta_c
      }
    }
    write_coefficients(a, F, ((int64_t)q3 * a.nq2 + q2) * a.nq1 + q1, 1.0);
  }
}

// Coefficients of a rational (NURBS) map F = sum_i w_i C_i B_i / W, W = sum_i w_i B_i.
// Point by point over the (p+1)^3 functions active there (one block per (q3, tile
// of TQ2 q2, tile of TQ1 q1), the tile's control points and weights in shared
// memory): F first, then DF = sum_i w_i (C_i - F) x grad B_i / W (the quotient rule
// with sum_i w_i grad B_i = grad W), so the O(1/h) gradients multiply the small
// differences C_i - F and do not cancel in the sum. With NURBS basis functions
// (w_i B_i / W) the mass coefficient is det DF / W^2 (the denominator folded into c).
__global__ void k_coef_rational(CoefArgs a) {
  extern __shared__ double sm[];
  const int p = a.p, m = p + 1;
  const int nt1 = (a.nq1 + kCoefTQ1 - 1) / kCoefTQ1;
  int bid = blockIdx.x;
  const int tq1 = bid % nt1;
  bid /= nt1;
  const int nt2 = (a.nq2 + kCoefTQ2 - 1) / kCoefTQ2;
  const int tq2 = bid % nt2;
  const int q3 = bid / nt2;
  const int qa1 = tq1 * kCoefTQ1, qb1 = min(a.nq1, qa1 + kCoefTQ1);
  const int qa2 = tq2 * kCoefTQ2, qb2 = min(a.nq2, qa2 + kCoefTQ2);
  const int ia1 = a.f1[qa1], ib1 = a.f1[qb1 - 1] + p + 1;
  const int ia2 = a.f2[qa2], ib2 = a.f2[qb2 - 1] + p + 1;
  const int W1 = ib1 - ia1, W2 = ib2 - ia2;
  const int f3 = a.f3[q3];
  double* Cs = sm;  // [m][W2][W1][4]: C_x C_y C_z w
  for (int e = threadIdx.x; e < m * W2 * W1; e += blockDim.x) {
    const int i1 = e % W1, i2 = (e / W1) % W2, t3 = e / (W1 * W2);
    const int64_t idx = ((int64_t)(f3 + t3) * a.n2 + (ia2 + i2)) * a.n1 + (ia1 + i1);
    double* c = Cs + (size_t)e * 4;
    c[0] = a.ctrl[idx * 3];
    c[1] = a.ctrl[idx * 3 + 1];
    c[2] = a.ctrl[idx * 3 + 2];
    c[3] = a.weights[idx];
  }
  __syncthreads();
  const int nq1t = qb1 - qa1, nq2t = qb2 - qa2;
  for (int e = threadIdx.x; e < nq2t * nq1t; e += blockDim.x) {
    const int q1 = qa1 + e % nq1t, q2 = qa2 + e / nq1t;
    const int o1 = a.f1[q1] - ia1, o2 = a.f2[q2] - ia2;
    const double* b1 = a.bp1 + (int64_t)q1 * m;
    const double* d1 = a.bp1 + ((int64_t)a.nq1 + q1) * m;
    const double* b2 = a.bp2 + (int64_t)q2 * m;
    const double* d2 = a.bp2 + ((int64_t)a.nq2 + q2) * m;
    const double* b3 = a.bp3 + (int64_t)q3 * m;
    const double* d3 = a.bp3 + ((int64_t)a.nq3 + q3) * m;
    double W = 0.0, N[3] = {0.0, 0.0, 0.0};
    for (int t3 = 0; t3 < m; ++t3)
      for (int t2 = 0; t2 < m; ++t2) {
        const double* row = Cs + ((size_t)(t3 * W2 + o2 + t2) * W1 + o1) * 4;
        const double b23 = b3[t3] * b2[t2];
        for (int t1 = 0; t1 < m; ++t1) {
          const double* c = row + t1 * 4;
          const double wb = c[3] * (b23 * b1[t1]);
          W += wb;
          N[0] = fma(wb, c[0], N[0]);
          N[1] = fma(wb, c[1], N[1]);
          N[2] = fma(wb, c[2], N[2]);
        }
      }
    const double iw = 1.0 / W;
    const double Fx[3] = {N[0] * iw, N[1] * iw, N[2] * iw};
    double J[3][3] = {{0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}};
    for (int t3 = 0; t3 < m; ++t3)
      for (int t2 = 0; t2 < m; ++t2) {
        const double* row = Cs + ((size_t)(t3 * W2 + o2 + t2) * W1 + o1) * 4;
        for (int t1 = 0; t1 < m; ++t1) {
          const double* c = row + t1 * 4;
          const double g[3] = {c[3] * d1[t1] * b2[t2] * b3[t3], c[3] * b1[t1] * d2[t2] * b3[t3],
                               c[3] * b1[t1] * b2[t2] * d3[t3]};
          for (int r = 0; r < 3; ++r) {
            const double dr = c[r] - Fx[r];
            J[r][0] = fma(g[0], dr, J[r][0]);
            J[r][1] = fma(g[1], dr, J[r][1]);
            J[r][2] = fma(g[2], dr, J[r][2]);
          }
        }
      }
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) J[r][c] *= iw;
    if (!(W > 0.0) || !isfinite(W)) atomicOr(a.err, kErrBadGeometry);
    write_coefficients(a, J, ((int64_t)q3 * a.nq2 + q2) * a.nq1 + q1, a.nurbs_basis ? iw * iw : 1.0);
  }
}

static size_t coef_smem(int p) {
  int W1 = kCoefTQ1 / 2 + p + 2, W2 = kCoefTQ2 / 2 + p + 2;
  return sizeof(double) * (size_t)(2 * W2 * W1 * 3 + 3 * kCoefTQ2 * W1 * 3);
}

static size_t coef_rational_smem(int p) {
  int W1 = kCoefTQ1 / 2 + p + 2, W2 = kCoefTQ2 / 2 + p + 2;
  return sizeof(double) * (size_t)(p + 1) * W2 * W1 * 4;
}

wq_status run_coefficients(wq_plan_s* pl, cudaStream_t s, double* jac) {
  if (fault("geometry")) return set_error(WQ_ERR_INJECTED, "injected failure at the coefficient step");
  if (pl->wts) {
    CoefArgs a{};
    a.p = pl->p;
    a.n1 = (int)pl->n[0];
    a.n2 = (int)pl->n[1];
    a.n3 = (int)pl->n[2];
    a.nq1 = (int)pl->nqp[0];
    a.nq2 = (int)pl->nqp[1];
    a.nq3 = (int)pl->nqp[2];
    a.ctrl = pl->ctrl;
    a.bp1 = pl->dir[0].bp;
    a.bp2 = pl->dir[1].bp;
    a.bp3 = pl->dir[2].bp;
    a.f1 = pl->dir[0].first;
    a.f2 = pl->dir[1].first;
    a.f3 = pl->dir[2].first;
    a.coef = pl->coef;
    a.jac = jac;
    a.nqp_total = pl->n_qp_total;
    a.err = pl->err;
    a.K = pl->Kt;
    a.weights = pl->wts;
    a.nurbs_basis = pl->nurbs_basis;
    int64_t blocks = (int64_t)((a.nq1 + kCoefTQ1 - 1) / kCoefTQ1) * ((a.nq2 + kCoefTQ2 - 1) / kCoefTQ2) * a.nq3;
    size_t smem = coef_rational_smem(pl->p);
    WQ_CUDA_TRY(cudaFuncSetAttribute(k_coef_rational, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                "rational coefficient kernel attributes");
    k_coef_rational<<<(unsigned)blocks, 256, smem, s>>>(a);
    count_launch();
    WQ_CUDA_TRY(cudaGetLastError(), "rational coefficient kernel launch");
    return WQ_OK;
  }
  DeltaArgs da;
  da.n1 = (int)pl->n[0];
  da.n2 = (int)pl->n[1];
  da.n3 = (int)pl->n[2];
  da.ctrl = pl->ctrl;
  da.g1 = pl->dir[0].greville;
  da.g2 = pl->dir[1].greville;
  da.g3 = pl->dir[2].greville;
  da.delta = pl->ctrl_delta;
  k_delta<<<(unsigned)((pl->n_rows + 255) / 256), 256, 0, s>>>(da);
  count_launch();
  CoefArgs a{};
  a.p = pl->p;
  a.n1 = (int)pl->n[0];
  a.n2 = (int)pl->n[1];
  a.n3 = (int)pl->n[2];
  a.nq1 = (int)pl->nqp[0];
  a.nq2 = (int)pl->nqp[1];
  a.nq3 = (int)pl->nqp[2];
  a.ctrl = pl->ctrl_delta;
  a.bp1 = pl->dir[0].bp;
  a.bp2 = pl->dir[1].bp;
  a.bp3 = pl->dir[2].bp;
  a.f1 = pl->dir[0].first;
  a.f2 = pl->dir[1].first;
  a.f3 = pl->dir[2].first;
  a.coef = pl->coef;
  a.jac = jac;
  a.nqp_total = pl->n_qp_total;
  a.err = pl->err;
  a.K = pl->Kt;
  a.weights = nullptr;
  a.nurbs_basis = 0;
  int64_t blocks = (int64_t)((a.nq1 + kCoefTQ1 - 1) / kCoefTQ1) * ((a.nq2 + kCoefTQ2 - 1) / kCoefTQ2) * a.nq3;
  size_t smem = coef_smem(pl->p);
  WQ_CUDA_TRY(cudaFuncSetAttribute(k_coef, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
              "coefficient kernel attributes");
  k_coef<<<(unsigned)blocks, 256, smem, s>>>(a);
  count_launch();
  WQ_CUDA_TRY(cudaGetLastError(), "coefficient kernel launch");
  return WQ_OK;
}

wq_status run_setup(wq_plan_s* pl, cudaStream_t s, bool with_pattern) {
  const int p = pl->p;
  DirArgs3 A;
  int max_n = 0, max_qp = 0, max_el = 0;
  for (int l = 0; l < 3; ++l) {
    A.d[l] = dir_args(pl, l);
    DirData& d = pl->dir[l];
    max_n = std::max(max_n, d.n);
    max_qp = std::max(max_qp, d.nqp);
    max_el = std::max(max_el, d.n_el);
    size_t tab = (size_t)2 * d.n * pl->nq_max;
    WQ_CUDA_TRY(cudaMemsetAsync(d.bt, 0, tab * sizeof(double), s), "table reset");
    WQ_CUDA_TRY(cudaMemsetAsync(d.bt_dd, 0, tab * sizeof(dd), s), "table reset");
  }
  const int tb = 128;
  for (int l = 0; l < 3; ++l) {
    const DirData& d = pl->dir[l];
    const int ld = d.n + p + 1;
    k_recips<<<(p * ld + tb - 1) / tb, tb, 0, s>>>(d.knots, d.n, p, ld, d.recip);
  }
  count_launch(3);
  k_points<<<dim3((max_qp + tb - 1) / tb, 3), tb, 0, s>>>(A);
  k_qranges<<<dim3((max_n + tb - 1) / tb, 3), tb, 0, s>>>(A);
  // double-double chains: one warp per block, so the work spreads over the SMs
  k_basis_points<<<dim3((max_qp + 31) / 32, 3), 32, 0, s>>>(A);
  k_gauss_basis<<<dim3((max_el * (p + 1) + 31) / 32, 3), 32, 0, s>>>(A);
  k_integrals<<<dim3((max_n * (2 * p + 1) * 4 + 31) / 32, 3), 32, 0, s>>>(A);
  k_rules<<<dim3(max_n, 4, 3), 32, 0, s>>>(A);
  k_prefix<<<dim3(1, 3), 32, 0, s>>>(A);
  k_greville<<<dim3((max_n + tb - 1) / tb, 3), tb, 0, s>>>(A);
  count_launch(8);
  WQ_CUDA_TRY(cudaGetLastError(), "set-up kernels");
  if (fault("solve")) return set_error(WQ_ERR_INJECTED, "injected failure at the WQ rule step");
  if (with_pattern) {
    PatternArgs pa;
    pa.p = p;
    pa.n1 = (int)pl->n[0];
    pa.n2 = (int)pl->n[1];
    pa.n3 = (int)pl->n[2];
    pa.P1 = pl->dir[0].prefix;
    pa.P2 = pl->dir[1].prefix;
    pa.P3 = pl->dir[2].prefix;
    pa.row_ptr = pl->row_ptr;
    pa.col = pl->col;
    int64_t N = pl->n_rows;
    k_row_ptr<<<(unsigned)((N + 1 + 255) / 256), 256, 0, s>>>(pa);
    int dev_sms = 152;
    cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, pl->device);
    int64_t warps_needed = N;
    int64_t blocks = (warps_needed + 7) / 8;
    int64_t cap = (int64_t)dev_sms * 16;
    if (blocks > cap) blocks = cap;
    const int bw = 2 * pl->p + 1;
    k_cols<<<(unsigned)blocks, 256, sizeof(int) * bw * bw * bw, s>>>(pa);
    count_launch(2);
    WQ_CUDA_TRY(cudaGetLastError(), "pattern kernels");
  }
  return run_coefficients(pl, s);
}

}  // namespace wq

// ---------------------------------------------------------------------------
// Host side of the plan.

using wq::set_error;

static bool knots_ok(const double* xi, int64_t len, int p, std::string* why) {
  if (len < 2 * (p + 1) + 1) {
    *why = "a knot vector needs at least two spans (length >= 2p+3)";
    return false;
  }
  for (int64_t k = 0; k < len; ++k)
    if (!std::isfinite(xi[k])) {
      *why = "knots must be finite";
      return false;
    }
  for (int k = 1; k <= p; ++k)
    if (xi[k] != xi[0] || xi[len - 1 - k] != xi[len - 1]) {
      *why = "end knots must repeat p+1 times (open knot vector)";
      return false;
    }
  for (int64_t k = p; k < len - p - 1; ++k)
    if (!(xi[k + 1] > xi[k])) {
      *why = "interior knots must be simple and strictly increasing";
      return false;
    }
  return true;
}

static void free_plan(wq_plan_s* pl) {
  if (!pl) return;
  // a caller allocator may hand the memory out again at once: let queued work finish
  if (pl->opt.free) cudaDeviceSynchronize();
  for (int l = 0; l < 3; ++l) {
    wq::DirData& d = pl->dir[l];
    void* ptrs[] = {d.knots, d.x, d.x_dd, d.first, d.q0, d.nq, d.bt_dd, d.bt, d.bp, d.gb, d.integ, d.w, d.prefix,
                    d.greville, d.pair_row, d.tab32, d.tabf2, d.recip};
    for (void* q : ptrs) wq::plan_free(pl, q, nullptr);
  }
  void* ptrs[] = {pl->ctrl, pl->ctrl_delta, pl->coef, pl->row_ptr, pl->col, pl->gauss, pl->err, pl->jac,
                  pl->adj_scratch, pl->coefT, pl->stg_a, pl->stg_b, pl->stg_c, pl->stg_d, pl->wts, pl->Kt, pl->load_scratch};
  for (void* q : ptrs) wq::plan_free(pl, q, nullptr);
  if (pl->slab_done) cudaEventDestroy(pl->slab_done);
  if (pl->copy_stream) cudaStreamDestroy(pl->copy_stream);
  if (pl->ev_fork) cudaEventDestroy(pl->ev_fork);
  if (pl->ev_join) cudaEventDestroy(pl->ev_join);
  if (pl->side_stream) cudaStreamDestroy(pl->side_stream);
  delete pl;
}

namespace wq {

bool fault(const char* step) {
  const char* env = std::getenv("WQ_FAULT");
  if (!env || !*env) return false;
  const size_t n = std::strlen(step);
  for (const char* c = env; *c;) {
    const char* e = std::strchr(c, ',');
    const size_t len = e ? (size_t)(e - c) : std::strlen(c);
    if (len == n && std::strncmp(c, step, n) == 0) return true;
    if (!e) break;
    c = e + 1;
  }
  return false;
}

wq_status plan_alloc(wq_plan_s* pl, void** ptr, size_t bytes, cudaStream_t s, const char* what) {
  *ptr = nullptr;
  if (fault("alloc")) return set_error(WQ_ERR_INJECTED, std::string("injected allocation failure: ") + what);
  if (bytes == 0) bytes = 16;
  if (pl->opt.alloc) {
    void* q = pl->opt.alloc(bytes, (void*)s, pl->opt.alloc_ctx);
    if (!q) return set_error(WQ_ERR_OOM, std::string("the caller's allocator returned NULL: ") + what);
    if (reinterpret_cast<uintptr_t>(q) % 256 != 0) {
      pl->opt.free(q, (void*)s, pl->opt.alloc_ctx);
      return set_error(WQ_ERR_INVALID_ARG, std::string("the caller's allocator returned memory not aligned to "
                                                       "256 bytes: ") + what);
    }
    *ptr = q;
    return WQ_OK;
  }
  cudaError_t e = cudaMalloc(ptr, bytes);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    *ptr = nullptr;
    return set_error(WQ_ERR_OOM, std::string("device allocation failed: ") + what);
  }
  if (e != cudaSuccess) {
    *ptr = nullptr;
    return cuda_error(e, what);
  }
  return WQ_OK;
}

void plan_free(wq_plan_s* pl, void* ptr, cudaStream_t s) {
  if (!ptr) return;
  if (pl->opt.free)
    pl->opt.free(ptr, (void*)s, pl->opt.alloc_ctx);
  else
    cudaFree(ptr);
}

// cuMemGetAddressRange through the runtime's driver entry point (no link-time
// dependency on the driver library).
typedef int (*AddressRangeFn)(unsigned long long* base, size_t* size, unsigned long long ptr);

wq_status check_device_range(const wq_plan_s* pl, const void* p, size_t bytes, const char* what) {
  static AddressRangeFn fn = nullptr;
  if (!fn) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuMemGetAddressRange", &f, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !f)
      return set_error(WQ_ERR_UNSUPPORTED, "checked mode: the driver's address-range query is unavailable");
    fn = reinterpret_cast<AddressRangeFn>(f);
  }
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_error(WQ_ERR_INVALID_ARG, std::string("checked mode: not a device pointer: ") + what);
  }
  if (at.type != cudaMemoryTypeDevice || at.device != pl->device)
    return set_error(WQ_ERR_INVALID_ARG, std::string("checked mode: not device memory of the plan's device: ") + what);
  unsigned long long base = 0;
  size_t size = 0;
  if (fn(&base, &size, reinterpret_cast<unsigned long long>(p)) != 0)
    return set_error(WQ_ERR_INVALID_ARG, std::string("checked mode: no device allocation holds ") + what);
  const unsigned long long a = reinterpret_cast<unsigned long long>(p);
  if (a + bytes > base + size)
    return set_error(WQ_ERR_INVALID_ARG, std::string("checked mode: ") + what + " needs " + std::to_string(bytes) +
                                             " bytes but its allocation ends " + std::to_string(base + size - a) +
                                             " bytes after it");
  return WQ_OK;
}

}  // namespace wq

static wq_status dev_alloc(wq_plan_s* pl, void** ptr, size_t bytes, cudaStream_t s, const char* what) {
  return wq::plan_alloc(pl, ptr, bytes, s, what);
}

static wq_status read_error_word(wq_plan_s* pl, cudaStream_t s) {
  int h = 0;
  WQ_CUDA_TRY(cudaMemcpyAsync(&h, pl->err, sizeof(int), cudaMemcpyDeviceToHost, s), "error word read");
  WQ_CUDA_TRY(cudaStreamSynchronize(s), "stream synchronize");
  if (h) WQ_CUDA_TRY(cudaMemsetAsync(pl->err, 0, sizeof(int), s), "error word reset");
  if (h & wq::kErrBadGeometry) return set_error(WQ_ERR_BAD_GEOMETRY, "det DF <= 0 or not finite at a quadrature point");
  if (h & wq::kErrSingularRule) return set_error(WQ_ERR_SINGULAR_RULE, "a WQ rule system broke down");
  if (h & wq::kErrTimeout) return set_error(WQ_ERR_TIMEOUT, "a bounded device wait gave up");
  if (h & wq::kErrNonFinite) return set_error(WQ_ERR_NONFINITE, "an assembled value is NaN or infinite");
  return WQ_OK;
}

extern "C" wq_status wq_options_init(wq_options* opt) {
  if (!opt) return set_error(WQ_ERR_INVALID_ARG, "NULL options");
  *opt = wq_options{};
  opt->size = sizeof(wq_options);
  opt->value_dtype = WQ_VALUES_F64;
  opt->precision = WQ_PREC_FP64;
  opt->algorithm = WQ_ALGO_AUTO;
  return WQ_OK;
}

// Tile extents for degree p from a text cache of "p t1 t2" lines ('#' starts a comment).
static bool read_tune_cache(const char* path, int p, int* t1, int* t2) {
  FILE* f = std::fopen(path, "r");
  if (!f) return false;
  char line[256];
  bool found = false;
  while (std::fgets(line, sizeof line, f)) {
    int q, a, b;
    if (line[0] == '#') continue;
    if (std::sscanf(line, "%d %d %d", &q, &a, &b) == 3 && q == p && a >= 1 && a <= 64 && b >= 1 && b <= 64) {
      *t1 = a;
      *t2 = b;
      found = true;
    }
  }
  std::fclose(f);
  return found;
}

static wq_status validate_options(const wq_options* o) {
  if (o->size != sizeof(wq_options))
    return set_error(WQ_ERR_INVALID_ARG, "wq_options.size does not match this library (call wq_options_init)");
  if (o->value_dtype != WQ_VALUES_F64 && o->value_dtype != WQ_VALUES_F32)
    return set_error(WQ_ERR_INVALID_ARG, "wq_options.value_dtype is not a value type");
  if (o->precision < WQ_PREC_FP64 || o->precision > WQ_PREC_TF32X3)
    return set_error(WQ_ERR_INVALID_ARG, "wq_options.precision is not a precision mode");
  if (o->precision == WQ_PREC_FP64 && o->value_dtype != WQ_VALUES_F64)
    return set_error(WQ_ERR_INVALID_ARG, "FP64 contractions write FP64 values");
  if (o->algorithm != WQ_ALGO_FUSED && o->algorithm != WQ_ALGO_STAGED && o->algorithm != WQ_ALGO_AUTO)
    return set_error(WQ_ERR_INVALID_ARG, "wq_options.algorithm is not an algorithm");
  if (o->tile[0] < 0 || o->tile[1] < 0 || o->tile[0] > 64 || o->tile[1] > 64 || (o->tile[0] == 0) != (o->tile[1] == 0))
    return set_error(WQ_ERR_INVALID_ARG, "wq_options.tile must be {0, 0} or in 1..64");
  if (o->checked != 0 && o->checked != 1) return set_error(WQ_ERR_INVALID_ARG, "wq_options.checked must be 0 or 1");
  if ((o->alloc == nullptr) != (o->free == nullptr))
    return set_error(WQ_ERR_INVALID_ARG, "wq_options.alloc and wq_options.free come together");
  return WQ_OK;
}

extern "C" wq_status wq_plan_create(wq_plan_t* out, int d, int p, const int64_t n_knots[3],
                                    const double* const h_knots[3], const double* h_ctrl, const wq_options* opt,
                                    void* stream) {
  if (!out || !n_knots || !h_knots || !h_ctrl) return set_error(WQ_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  wq_options o;
  wq_options_init(&o);
  if (opt) {
    wq_status vs = validate_options(opt);
    if (vs != WQ_OK) return vs;
    o = *opt;
  }
  if (d != 3) return set_error(WQ_ERR_UNSUPPORTED, "only d = 3 is supported");
  if (p < 2 || p > wq::kMaxP) return set_error(WQ_ERR_INVALID_ARG, "degree must be in 2..8");
  int64_t n[3];
  for (int l = 0; l < 3; ++l) {
    std::string why;
    if (!h_knots[l]) return set_error(WQ_ERR_INVALID_ARG, "NULL knot vector");
    if (!knots_ok(h_knots[l], n_knots[l], p, &why)) return set_error(WQ_ERR_INVALID_ARG, why);
    n[l] = n_knots[l] - p - 1;
  }
  const int64_t N = n[0] * n[1] * n[2];
  if (N > INT32_MAX) return set_error(WQ_ERR_UNSUPPORTED, "N_DOF must fit in int32 column indices");
  for (int64_t k = 0; k < 3 * N; ++k)
    if (!std::isfinite(h_ctrl[k])) return set_error(WQ_ERR_INVALID_ARG, "control points must be finite");
  int dev = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce != cudaSuccess) return wq::cuda_error(ce, "no CUDA device");
  cudaStream_t s = (cudaStream_t)stream;

  wq_plan_s* pl = new wq_plan_s();
  pl->opt = o;
  pl->p = p;
  pl->device = dev;
  pl->algorithm = o.algorithm;
  pl->tile[0] = o.tile[0];
  pl->tile[1] = o.tile[1];
  if (o.tile[0] == 0 && o.tune_cache) read_tune_cache(o.tune_cache, p, &pl->tile[0], &pl->tile[1]);
  pl->opt.tune_cache = nullptr;  // the path is not kept
  pl->n_rows = N;
  int64_t nnz = 1;
  int nqmax = 0;
  for (int l = 0; l < 3; ++l) {
    wq::DirData& dd = pl->dir[l];
    dd.n = (int)n[l];
    dd.n_el = (int)(n[l] - p);
    dd.nqp = 2 * dd.n_el + 2 * p - 1;
    pl->n[l] = n[l];
    pl->nqp[l] = dd.nqp;
    pl->nnz1[l] = 0;  // sum of the band widths |I_i| (= (2p+1) n - p(p+1) when n >= 2p+1)
    for (int i = 0; i < dd.n; ++i) pl->nnz1[l] += std::min(dd.n - 1, i + p) - std::max(0, i - p) + 1;
    nnz *= pl->nnz1[l];
    for (int i = 0; i < dd.n; ++i) {  // |Q_i| from the same closed form as k_qranges
      int lo = std::max(0, i - p), hi = std::min(dd.n_el, i + 1);
      int qs = lo == 0 ? 0 : 2 * lo + p;
      int qe = hi == dd.n_el ? dd.nqp - 1 : 2 * hi + p - 2;
      nqmax = std::max(nqmax, qe - qs + 1);
    }
  }
  pl->nnz = nnz;
  pl->nq_max = nqmax;
  pl->n_qp_total = pl->nqp[0] * pl->nqp[1] * pl->nqp[2];

  wq_status st = WQ_OK;
#define ALLOC(ptr, bytes, what)                                  \
  do {                                                           \
    st = dev_alloc(pl, (void**)&(ptr), (size_t)(bytes), s, what); \
    if (st != WQ_OK) {                                           \
      free_plan(pl);                                             \
      return st;                                                 \
    }                                                            \
  } while (0)
  for (int l = 0; l < 3; ++l) {
    wq::DirData& dd = pl->dir[l];
    const int m = p + 1;
    ALLOC(dd.knots, sizeof(double) * n_knots[l], "knots");
    ALLOC(dd.x, sizeof(double) * dd.nqp, "points");
    ALLOC(dd.x_dd, sizeof(wq::dd) * dd.nqp, "points");
    ALLOC(dd.first, sizeof(int) * dd.nqp, "spans");
    ALLOC(dd.q0, sizeof(int) * dd.n, "Q ranges");
    ALLOC(dd.nq, sizeof(int) * dd.n, "Q ranges");
    ALLOC(dd.bt_dd, sizeof(wq::dd) * 2 * dd.n * nqmax, "basis tables");
    ALLOC(dd.bt, sizeof(double) * 2 * dd.n * nqmax, "basis tables");
    ALLOC(dd.bp, sizeof(double) * 2 * dd.nqp * m, "basis tables");
    ALLOC(dd.gb, sizeof(wq::dd) * dd.n_el * m * 2 * m, "Gauss basis");
    ALLOC(dd.integ, sizeof(wq::dd) * 4 * dd.n * (2 * p + 1), "integrals");
    ALLOC(dd.w, sizeof(double) * 4 * dd.n * nqmax, "rules");
    ALLOC(dd.prefix, sizeof(int64_t) * (dd.n + 1), "band prefix");
    ALLOC(dd.greville, sizeof(wq::dd) * dd.n, "Greville points");
    ALLOC(dd.recip, sizeof(wq::dd) * (p + 1) * (dd.n + p + 1), "knot reciprocals");
  }
  ALLOC(pl->ctrl, sizeof(double) * 3 * N, "control points");
  ALLOC(pl->ctrl_delta, sizeof(double) * 3 * N, "control point offsets");
  ALLOC(pl->coef, sizeof(double) * 7 * pl->n_qp_total, "coefficients");
  ALLOC(pl->row_ptr, sizeof(int64_t) * (N + 1), "row_ptr");
  ALLOC(pl->col, sizeof(int32_t) * nnz, "col");
  ALLOC(pl->gauss, sizeof(wq::dd) * 2 * (p + 1), "Gauss rule");
  ALLOC(pl->err, sizeof(int), "error word");
#undef ALLOC
  auto fail = [&](wq_status code) {
    free_plan(pl);
    return code;
  };
  if (wq::fault("h2d")) return fail(set_error(WQ_ERR_INJECTED, "injected failure of the knot copy"));
  for (int l = 0; l < 3; ++l) {
    cudaError_t e = cudaMemcpyAsync(pl->dir[l].knots, h_knots[l], sizeof(double) * n_knots[l],
                                    cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return fail(wq::cuda_error(e, "knot copy"));
  }
  cudaError_t e = cudaMemcpyAsync(pl->ctrl, h_ctrl, sizeof(double) * 3 * N, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return fail(wq::cuda_error(e, "control point copy"));
  e = cudaMemsetAsync(pl->err, 0, sizeof(int), s);
  if (e != cudaSuccess) return fail(wq::cuda_error(e, "error word reset"));
  // the Gauss-Legendre rule depends on p only: computed once per plan
  wq::k_gauss<<<1, 32, 0, s>>>(pl->gauss, p + 1);
  wq::count_launch();
  st = wq::run_setup(pl, s, true);
  if (st != WQ_OK) return fail(st);
  st = read_error_word(pl, s);
  if (st != WQ_OK) return fail(st);
  *out = pl;
  return WQ_OK;
}

extern "C" wq_status wq_destroy(wq_plan_t plan) {
  free_plan(plan);
  return WQ_OK;
}

extern "C" wq_status wq_plan_destroy(wq_plan_t plan) { return wq_destroy(plan); }

extern "C" wq_status wq_plan_info(wq_plan_t plan, int* p, int64_t n[3], int64_t n_qp[3], int64_t* n_rows,
                                  int64_t* nnz) {
  if (!plan) return set_error(WQ_ERR_INVALID_ARG, "NULL plan");
  if (p) *p = plan->p;
  for (int l = 0; l < 3; ++l) {
    if (n) n[l] = plan->n[l];
    if (n_qp) n_qp[l] = plan->nqp[l];
  }
  if (n_rows) *n_rows = plan->n_rows;
  if (nnz) *nnz = plan->nnz;
  return WQ_OK;
}

extern "C" wq_status wq_plan_pattern(wq_plan_t plan, const int64_t** d_row_ptr, const int32_t** d_col) {
  if (!plan) return set_error(WQ_ERR_INVALID_ARG, "NULL plan");
  if (d_row_ptr) *d_row_ptr = plan->row_ptr;
  if (d_col) *d_col = plan->col;
  return WQ_OK;
}

static wq_status copy_ctrl(wq_plan_t plan, const double* ctrl, int on_device, cudaStream_t s) {
  if (!ctrl) return WQ_OK;
  if (!on_device && wq::fault("h2d")) return set_error(WQ_ERR_INJECTED, "injected failure of the control point copy");
  if (on_device && plan->opt.checked) {
    wq_status st = wq::check_device_range(plan, ctrl, sizeof(double) * 3 * plan->n_rows, "control points");
    if (st != WQ_OK) return st;
  }
  cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  WQ_CUDA_TRY(cudaMemcpyAsync(plan->ctrl, ctrl, sizeof(double) * 3 * plan->n_rows, kind, s), "control point copy");
  return WQ_OK;
}

extern "C" wq_status wq_plan_set_geometry(wq_plan_t plan, const double* ctrl, int ctrl_on_device, void* stream) {
  if (!plan || !ctrl) return set_error(WQ_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  wq_status st = copy_ctrl(plan, ctrl, ctrl_on_device, s);
  if (st != WQ_OK) return st;
  return wq::run_coefficients(plan, s);
}

extern "C" wq_status wq_plan_refresh(wq_plan_t plan, const double* ctrl, int ctrl_on_device, void* stream) {
  if (!plan) return set_error(WQ_ERR_INVALID_ARG, "NULL plan");
  cudaStream_t s = (cudaStream_t)stream;
  wq_status st = copy_ctrl(plan, ctrl, ctrl_on_device, s);
  if (st != WQ_OK) return st;
  return wq::run_setup(plan, s, true);
}

extern "C" wq_status wq_plan_set_weights(wq_plan_t plan, const double* w, int on_device, int nurbs_basis,
                                         void* stream) {
  if (!plan) return set_error(WQ_ERR_INVALID_ARG, "NULL plan");
  if (nurbs_basis != 0 && nurbs_basis != 1) return set_error(WQ_ERR_INVALID_ARG, "nurbs_basis must be 0 or 1");
  if (!w && nurbs_basis) return set_error(WQ_ERR_INVALID_ARG, "NURBS basis functions need weights");
  cudaStream_t s = (cudaStream_t)stream;
  if (!w) {
    wq::plan_free(plan, plan->wts, s);
    plan->wts = nullptr;
    plan->nurbs_basis = 0;
    return wq::run_coefficients(plan, s);
  }
  const size_t bytes = sizeof(double) * (size_t)plan->n_rows;
  if (!on_device) {
    for (int64_t k = 0; k < plan->n_rows; ++k)
      if (!(w[k] > 0.0) || !std::isfinite(w[k])) return set_error(WQ_ERR_INVALID_ARG, "weights must be positive");
    if (wq::fault("h2d")) return set_error(WQ_ERR_INJECTED, "injected failure of the weight copy");
  } else if (plan->opt.checked) {
    wq_status st = wq::check_device_range(plan, w, bytes, "weights");
    if (st != WQ_OK) return st;
  }
  if (!plan->wts) {
    wq_status st = wq::plan_alloc(plan, (void**)&plan->wts, bytes, s, "NURBS weights");
    if (st != WQ_OK) return st;
  }
  WQ_CUDA_TRY(cudaMemcpyAsync(plan->wts, w, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s),
              "weight copy");
  plan->nurbs_basis = nurbs_basis;
  return wq::run_coefficients(plan, s);
}

extern "C" wq_status wq_plan_set_tensor(wq_plan_t plan, const double* d_K, void* stream) {
  if (!plan) return set_error(WQ_ERR_INVALID_ARG, "NULL plan");
  cudaStream_t s = (cudaStream_t)stream;
  if (!d_K) {
    wq::plan_free(plan, plan->Kt, s);
    plan->Kt = nullptr;
    return wq::run_coefficients(plan, s);
  }
  const size_t bytes = sizeof(double) * 6 * (size_t)plan->n_qp_total;
  if (plan->opt.checked) {
    wq_status st = wq::check_device_range(plan, d_K, bytes, "d_K");
    if (st != WQ_OK) return st;
  }
  if (!plan->Kt) {
    wq_status st = wq::plan_alloc(plan, (void**)&plan->Kt, bytes, s, "coefficient tensor");
    if (st != WQ_OK) return st;
  }
  WQ_CUDA_TRY(cudaMemcpyAsync(plan->Kt, d_K, bytes, cudaMemcpyDeviceToDevice, s), "tensor copy");
  return wq::run_coefficients(plan, s);
}

extern "C" wq_status wq_sync_check(wq_plan_t plan, void* stream) {
  if (!plan) return set_error(WQ_ERR_INVALID_ARG, "NULL plan");
  return read_error_word(plan, (cudaStream_t)stream);
}

extern "C" wq_status wq_get_nq_max(wq_plan_t plan, int* nq_max) {
  if (!plan || !nq_max) return set_error(WQ_ERR_INVALID_ARG, "NULL argument");
  *nq_max = plan->nq_max;
  return WQ_OK;
}

extern "C" wq_status wq_get_points(wq_plan_t plan, int dir, double* h_x) {
  if (!plan || !h_x || dir < 0 || dir > 2) return set_error(WQ_ERR_INVALID_ARG, "bad argument");
  WQ_CUDA_TRY(cudaDeviceSynchronize(), "synchronize");
  WQ_CUDA_TRY(cudaMemcpy(h_x, plan->dir[dir].x, sizeof(double) * plan->nqp[dir], cudaMemcpyDeviceToHost),
              "points copy");
  return WQ_OK;
}

extern "C" wq_status wq_get_rules(wq_plan_t plan, int dir, int a, int b, double* h_w, int32_t* h_q0,
                                  int32_t* h_nq) {
  if (!plan || dir < 0 || dir > 2 || a < 0 || a > 1 || b < 0 || b > 1)
    return set_error(WQ_ERR_INVALID_ARG, "bad argument");
  const wq::DirData& d = plan->dir[dir];
  WQ_CUDA_TRY(cudaDeviceSynchronize(), "synchronize");
  if (h_w)
    WQ_CUDA_TRY(cudaMemcpy(h_w, d.w + (size_t)(2 * a + b) * d.n * plan->nq_max,
                           sizeof(double) * d.n * plan->nq_max, cudaMemcpyDeviceToHost),
                "rules copy");
  if (h_q0) WQ_CUDA_TRY(cudaMemcpy(h_q0, d.q0, sizeof(int) * d.n, cudaMemcpyDeviceToHost), "rules copy");
  if (h_nq) WQ_CUDA_TRY(cudaMemcpy(h_nq, d.nq, sizeof(int) * d.n, cudaMemcpyDeviceToHost), "rules copy");
  return WQ_OK;
}

extern "C" wq_status wq_get_coefficients(wq_plan_t plan, double* h_coef) {
  if (!plan || !h_coef) return set_error(WQ_ERR_INVALID_ARG, "NULL argument");
  WQ_CUDA_TRY(cudaDeviceSynchronize(), "synchronize");
  WQ_CUDA_TRY(cudaMemcpy(h_coef, plan->coef, sizeof(double) * 7 * plan->n_qp_total, cudaMemcpyDeviceToHost),
              "coefficient copy");
  return WQ_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free rule construction (wq_rules_noalloc).
//
// Some callers cannot allocate device memory from inside their own code. Examples
// are code that runs under a framework that owns all of GPU memory through its own
// pool, real-time loops where cudaMalloc's implicit device synchronisation is not
// acceptable, and embedded users with a fixed, pre-reserved memory budget. This
// entry point builds the four WQ rules of one direction with the same kernels as
// wq_plan_create, but keeps every intermediate table in one file-scope device
// array of fixed size instead of plan-owned buffers.
namespace wq {

constexpr int kNoAllocMaxN = 1024;                                    // functions per direction
constexpr int kNoAllocMaxKnots = kNoAllocMaxN + kMaxP + 1;
constexpr int kNoAllocMaxElems = kNoAllocMaxN;                        // n_el <= n - p < n
constexpr int kNoAllocMaxQp = 2 * kNoAllocMaxElems + 2 * kMaxP - 1;

constexpr size_t align256(size_t x) { return (x + 255) / 256 * 256; }

struct NoAllocLayout {
  size_t knots, x, x_dd, first, bt_dd, bt, bp, gb, integ, gauss, recip, err, total;
};

constexpr NoAllocLayout noalloc_layout() {
  NoAllocLayout L{};
  size_t o = 0;
  L.knots = o; o += align256(sizeof(double) * kNoAllocMaxKnots);
  L.x = o; o += align256(sizeof(double) * kNoAllocMaxQp);
  L.x_dd = o; o += align256(sizeof(dd) * kNoAllocMaxQp);
  L.first = o; o += align256(sizeof(int) * kNoAllocMaxQp);
  L.bt_dd = o; o += align256(sizeof(dd) * 2 * kNoAllocMaxN * kMaxQ);
  L.bt = o; o += align256(sizeof(double) * 2 * kNoAllocMaxN * kMaxQ);
  L.bp = o; o += align256(sizeof(double) * 2 * kNoAllocMaxQp * (kMaxP + 1));
  L.gb = o; o += align256(sizeof(dd) * kNoAllocMaxElems * (kMaxP + 1) * 2 * (kMaxP + 1));
  L.integ = o; o += align256(sizeof(dd) * 4 * kNoAllocMaxN * (2 * kMaxP + 1));
  L.gauss = o; o += align256(sizeof(dd) * 2 * (kMaxP + 1));
  L.recip = o; o += align256(sizeof(dd) * (kMaxP + 1) * kNoAllocMaxKnots);
  L.err = o; o += align256(sizeof(int));
  L.total = o;
  return L;
}

constexpr NoAllocLayout kNoAlloc = noalloc_layout();
static_assert(kNoAlloc.total == WQ_RULES_NOALLOC_SCRATCH_BYTES, "scratch size and its declared value differ");
static_assert(kNoAllocMaxN == WQ_RULES_NOALLOC_MAX_N, "scratch limit and its declared value differ");

// The scratch array: WQ_RULES_NOALLOC_SCRATCH_BYTES on every device that loads
// the library, held until the process exits. Host code must not take its
// address directly (that is a host-side stand-in); it uses the device address
// obtained by cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_rules_scratch[kNoAlloc.total];

// Device address of g_rules_scratch in the current device's context, looked up
// on every call: a cached address would outlive a cudaDeviceReset, after which
// the module is loaded again and the array may sit elsewhere.
static wq_status scratch_address(unsigned char** out) {
  void* ptr = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&ptr, g_rules_scratch);
  if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress of the rule scratch");
  *out = static_cast<unsigned char*>(ptr);
  return WQ_OK;
}

}  // namespace wq

extern "C" wq_status wq_rules_noalloc(int p, int64_t n_knots, const double* h_knots, double* d_w, int32_t* d_q0,
                                      int32_t* d_nq, int nq_stride, void* stream) {
  if (!h_knots || !d_w || !d_q0 || !d_nq) return set_error(WQ_ERR_INVALID_ARG, "NULL argument");
  if (p < 2 || p > wq::kMaxP) return set_error(WQ_ERR_INVALID_ARG, "degree must be in 2..8");
  std::string why;
  if (!knots_ok(h_knots, n_knots, p, &why)) return set_error(WQ_ERR_INVALID_ARG, why);
  const int64_t n = n_knots - p - 1;
  if (n > wq::kNoAllocMaxN)
    return set_error(WQ_ERR_INVALID_ARG, "wq_rules_noalloc: the knot vector has more basis functions than the "
                                         "1024 (WQ_RULES_NOALLOC_MAX_N) its fixed scratch holds; use "
                                         "wq_plan_create for larger knot vectors");
  const int n_el = (int)(n - p), nqp = 2 * n_el + 2 * p - 1;
  int nqmax = 0;
  for (int i = 0; i < (int)n; ++i) {
    int lo = std::max(0, i - p), hi = std::min(n_el, i + 1);
    int qs = lo == 0 ? 0 : 2 * lo + p;
    int qe = hi == n_el ? nqp - 1 : 2 * hi + p - 2;
    nqmax = std::max(nqmax, qe - qs + 1);
  }
  if (nq_stride < nqmax || nq_stride > 4 * p + 1)
    return set_error(WQ_ERR_INVALID_ARG, "nq_stride must lie between max |Q_i| and 4p+1");
  unsigned char* base = nullptr;
  wq_status st = wq::scratch_address(&base);
  if (st != WQ_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const wq::NoAllocLayout& L = wq::kNoAlloc;
  wq::DirArgs a;
  a.p = p;
  a.n = (int)n;
  a.n_el = n_el;
  a.nqp = nqp;
  a.nq_stride = nq_stride;
  a.knots = reinterpret_cast<const double*>(base + L.knots);
  a.x = reinterpret_cast<double*>(base + L.x);
  a.x_dd = reinterpret_cast<wq::dd*>(base + L.x_dd);
  a.first = reinterpret_cast<int*>(base + L.first);
  a.q0 = reinterpret_cast<int*>(d_q0);
  a.nq = reinterpret_cast<int*>(d_nq);
  a.bt_dd = reinterpret_cast<wq::dd*>(base + L.bt_dd);
  a.bt = reinterpret_cast<double*>(base + L.bt);
  a.bp = reinterpret_cast<double*>(base + L.bp);
  a.gb = reinterpret_cast<wq::dd*>(base + L.gb);
  a.integ = reinterpret_cast<wq::dd*>(base + L.integ);
  a.w = d_w;
  a.prefix = nullptr;
  a.greville = nullptr;
  a.gauss = reinterpret_cast<const wq::dd*>(base + L.gauss);
  a.recip = reinterpret_cast<const wq::dd*>(base + L.recip);
  int* err = reinterpret_cast<int*>(base + L.err);
  a.err = err;
  // the scratch keeps the previous call's contents: clear what is read before written
  size_t tab = (size_t)2 * n * nq_stride;
  WQ_CUDA_TRY(cudaMemcpyAsync(base + L.knots, h_knots, sizeof(double) * n_knots, cudaMemcpyHostToDevice, s),
              "knot copy");
  WQ_CUDA_TRY(cudaMemsetAsync(base + L.bt_dd, 0, tab * sizeof(wq::dd), s), "scratch reset");
  WQ_CUDA_TRY(cudaMemsetAsync(base + L.bt, 0, tab * sizeof(double), s), "scratch reset");
  WQ_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), s), "scratch reset");
  const int tb = 128;
  wq::DirArgs3 A;
  A.d[0] = a;
  wq::k_gauss<<<1, 32, 0, s>>>(reinterpret_cast<wq::dd*>(base + L.gauss), p + 1);
  wq::k_recips<<<(p * (int)n_knots + tb - 1) / tb, tb, 0, s>>>(reinterpret_cast<const double*>(base + L.knots), (int)n,
                                                                p, (int)n_knots, reinterpret_cast<wq::dd*>(base + L.recip));
  wq::k_points<<<(nqp + tb - 1) / tb, tb, 0, s>>>(A);
  wq::k_qranges<<<((int)n + tb - 1) / tb, tb, 0, s>>>(A);
  wq::k_basis_points<<<(nqp + 31) / 32, 32, 0, s>>>(A);
  wq::k_gauss_basis<<<(n_el * (p + 1) + 31) / 32, 32, 0, s>>>(A);
  wq::k_integrals<<<((int)n * (2 * p + 1) * 4 + 31) / 32, 32, 0, s>>>(A);
  wq::k_rules<<<dim3((unsigned)n, 4, 1), 32, 0, s>>>(A);
  wq::count_launch(8);
  WQ_CUDA_TRY(cudaGetLastError(), "rule kernels");
  int h_err = 0;
  WQ_CUDA_TRY(cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, s), "error word read");
  WQ_CUDA_TRY(cudaStreamSynchronize(s), "stream synchronize");
  if (h_err & wq::kErrSingularRule) return set_error(WQ_ERR_SINGULAR_RULE, "a WQ rule system broke down");
  return WQ_OK;
}
