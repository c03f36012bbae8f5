// Adjoint of the WQ bilinear forms: J = lambda^T S u (+ lambda^T M u) and its
// gradients with respect to the coefficient field kappa (at the quadrature
// points) and the control points of the geometry.
//
// With the WQ entries of Eq. (stiff) / Eq. (Mass_approx) written out,
//   J_S = sum_q kappa(q) sum_{l,m} c_lm(q) Lam_lm(q) U_m(q),
//   J_M = sum_q kappa(q) c(q) Lam_0(q) U_0(q),
// where U_m = sum_j u_j d_m B_j (U_0 = sum_j u_j B_j) at the points, and
// Lam_lm(q) = sum_i lambda_i prod_k w^{(delta_kl, delta_km)}_{k,i_k,q_k} (the
// test functions' rules, Lam_0 with the (0,0) rules). Both are tensor-product
// contractions, evaluated by three banded mode products each (Eq.
// (sumfactorization), applied to a field instead of a matrix row). Then
//   dJ/dkappa(q) = sum_{lm} c_lm Lam_lm U_m (+ c Lam_0 U_0),
//   Kb_lm = kappa Lam_lm U_m,  cb = kappa Lam_0 U_0,
//   dJ/dDF = det G [<Kb, P> G^{-T} - G^{-T} (Kb + Kb^T) P] + cb det G G^{-T},
// with G = DF, P = G^{-1} G^{-T} (c_lm = det G P_lm, Eq. (coef_stiff)), and
// dJ/dC_i = sum_q dJ/dDF(q) grad B_i(q) (DF = I + sum_i (C_i - g_i) grad B_i),
// a transposed mode product from the points back to the control points.
#include <algorithm>
#include <vector>

#include "wq_internal.h"

namespace wq {

// out[o] = sum_{t <= p} T[q][t] in[o with coordinate q replaced by first[q] + t]
// along `axis` of a 3D array (axis 0 fastest); q = o_axis in [0, nout).
__global__ void k_to_points(const double* __restrict__ in, double* __restrict__ out, int d0, int d1, int d2,
                            int axis, int nout, const double* __restrict__ T, const int* __restrict__ first, int m) {
  int od[3] = {d0, d1, d2};
  od[axis] = nout;
  const int64_t total = (int64_t)od[0] * od[1] * od[2];
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= total) return;
  int o[3];
  o[0] = (int)(idx % od[0]);
  o[1] = (int)((idx / od[0]) % od[1]);
  o[2] = (int)(idx / ((int64_t)od[0] * od[1]));
  const int q = o[axis];
  const int64_t stride = axis == 0 ? 1 : (axis == 1 ? (int64_t)d0 : (int64_t)d0 * d1);
  o[axis] = first[q];
  const int64_t base = o[0] + (int64_t)d0 * (o[1] + (int64_t)d1 * o[2]);
  double acc = 0.0;
  for (int t = 0; t < m; ++t) acc = fma(T[(int64_t)q * m + t], in[base + t * stride], acc);
  out[idx] = acc;
}

// out[o] = (accumulate ? out : 0) + sum_{t < nq[i]} T[i][t] in[o with coordinate i
// replaced by q0[i] + t], i = o_axis in [0, nout); the output may be strided
// (out[o * out_stride + out_offset]).
__global__ void k_to_functions(const double* __restrict__ in, double* __restrict__ out, int d0, int d1, int d2,
                               int axis, int nout, const double* __restrict__ T, const int* __restrict__ q0,
                               const int* __restrict__ nq, int NQ, int out_stride, int out_offset, int accumulate) {
  int od[3] = {d0, d1, d2};
  od[axis] = nout;
  const int64_t total = (int64_t)od[0] * od[1] * od[2];
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= total) return;
  int o[3];
  o[0] = (int)(idx % od[0]);
  o[1] = (int)((idx / od[0]) % od[1]);
  o[2] = (int)(idx / ((int64_t)od[0] * od[1]));
  const int i = o[axis];
  const int64_t stride = axis == 0 ? 1 : (axis == 1 ? (int64_t)d0 : (int64_t)d0 * d1);
  o[axis] = q0[i];
  const int64_t base = o[0] + (int64_t)d0 * (o[1] + (int64_t)d1 * o[2]);
  double acc = 0.0;
  const int n = nq[i];
  for (int t = 0; t < n; ++t) acc = fma(T[(int64_t)i * NQ + t], in[base + t * stride], acc);
  double* dst = out + idx * out_stride + out_offset;
  *dst = accumulate ? *dst + acc : acc;
}

// Point-major rule tables: Wp[kind][q][t] = w^{kind}_{first(q)+t, q} (0 when q is
// outside the open support of that function).
__global__ void k_point_weights(const double* __restrict__ w, const int* __restrict__ first,
                                const int* __restrict__ q0, const int* __restrict__ nq, int n, int nqp, int p, int NQ,
                                double* __restrict__ Wp) {
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  const int m = p + 1;
  if (id >= 4 * nqp) return;
  const int kind = id / nqp, q = id % nqp;
  for (int t = 0; t < m; ++t) {
    const int i = first[q] + t;
    const int loc = q - q0[i];
    double v = 0.0;
    if (i < n && loc >= 0 && loc < nq[i]) v = w[((int64_t)kind * n + i) * NQ + loc];
    Wp[((int64_t)kind * nqp + q) * m + t] = v;
  }
}

struct PointArgs {
  int64_t nqp;
  const double* coef;
  const double* jac;
  const double* kappa;
  const double* U;       // [4][nqp]: u, d1 u, d2 u, d3 u
  const double* L;       // [10][nqp]: Lam_{lm} (3l+m), Lam_0
  int which;             // bit 0 stiffness, bit 1 mass
  double* grad_kappa;    // NULL or [nqp]
  double* gbar;          // NULL or [9][nqp]: dJ/dDF_{rc}
  double* J;             // one accumulator
};

__global__ void k_adjoint_point(PointArgs a) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double contrib = 0.0;
  if (q < a.nqp) {
    const int64_t N = a.nqp;
    const double kap = a.kappa ? a.kappa[q] : 1.0;
    const int slot[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
    double Kb[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    double cb = 0.0, dk = 0.0;
    if (a.which & 1) {
      for (int l = 0; l < 3; ++l)
        for (int m = 0; m < 3; ++m) {
          const double lu = a.L[(3 * l + m) * N + q] * a.U[(m + 1) * N + q];
          dk = fma(a.coef[slot[l][m] * N + q], lu, dk);
          Kb[l][m] = kap * lu;
        }
    }
    if (a.which & 2) {
      const double lu = a.L[9 * N + q] * a.U[q];
      dk = fma(a.coef[6 * N + q], lu, dk);
      cb = kap * lu;
    }
    contrib = kap * dk;
    if (a.grad_kappa) a.grad_kappa[q] = dk;
    if (a.gbar) {
      double G[3][3];
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) G[r][c] = a.jac[(3 * r + c) * N + q];
      double adj[3][3];  // det * G^{-1}
      adj[0][0] = G[1][1] * G[2][2] - G[1][2] * G[2][1];
      adj[0][1] = G[0][2] * G[2][1] - G[0][1] * G[2][2];
      adj[0][2] = G[0][1] * G[1][2] - G[0][2] * G[1][1];
      adj[1][0] = G[1][2] * G[2][0] - G[1][0] * G[2][2];
      adj[1][1] = G[0][0] * G[2][2] - G[0][2] * G[2][0];
      adj[1][2] = G[0][2] * G[1][0] - G[0][0] * G[1][2];
      adj[2][0] = G[1][0] * G[2][1] - G[1][1] * G[2][0];
      adj[2][1] = G[0][1] * G[2][0] - G[0][0] * G[2][1];
      adj[2][2] = G[0][0] * G[1][1] - G[0][1] * G[1][0];
      const double det = G[0][0] * adj[0][0] + G[0][1] * adj[1][0] + G[0][2] * adj[2][0];
      const double inv = 1.0 / det;
      double GiT[3][3], P[3][3];  // G^{-T}, G^{-1} G^{-T}
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) GiT[r][c] = adj[c][r] * inv;
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) P[r][c] = (adj[r][0] * adj[c][0] + adj[r][1] * adj[c][1] + adj[r][2] * adj[c][2]) * inv * inv;
      double KP = 0.0;
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) KP = fma(Kb[r][c], P[r][c], KP);
      double KsP[3][3];  // (Kb + Kb^T) P
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
          double s = 0.0;
          for (int k = 0; k < 3; ++k) s = fma(Kb[r][k] + Kb[k][r], P[k][c], s);
          KsP[r][c] = s;
        }
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
          double s = 0.0;
          for (int k = 0; k < 3; ++k) s = fma(GiT[r][k], KsP[k][c], s);
          a.gbar[(3 * r + c) * N + q] = det * ((KP + cb) * GiT[r][c] - s);
        }
    }
  }
  // block reduction of J
  __shared__ double red[256];
  red[threadIdx.x] = contrib;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(a.J, red[0]);
}

static unsigned blocks_for(int64_t n, int tb) { return (unsigned)((n + tb - 1) / tb); }

// g(q) = f(q) c(q): the load integrand on the reference cube (c = det DF, Eq. (mass2)).
__global__ void k_load_field(const double* __restrict__ f, const double* __restrict__ c, double* __restrict__ g,
                             int64_t n) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q < n) g[q] = f[q] * c[q];
}

}  // namespace wq

// Load vector by weighted quadrature: b_i = Q_i(f det DF), the (0,0) rules of the
// three directions applied to the point field (Eq. (quadrule) with the test
// function's weights, the WQ approximation of int f R_i dx). Three mode products
// from the points to the functions, as in the adjoint's last pass.
extern "C" wq_status wq_assemble_load(wq_plan_t plan, const double* d_f, double* d_b, void* stream) {
  if (!plan || !d_f || !d_b) return wq::set_error(WQ_ERR_INVALID_ARG, "NULL argument");
  if (plan->nurbs_basis)
    return wq::set_error(WQ_ERR_UNSUPPORTED, "the load vector with NURBS basis functions is not provided");
  cudaStream_t s = (cudaStream_t)stream;
  wq_plan_s* pl = plan;
  const int n1 = (int)pl->n[0], n2 = (int)pl->n[1];
  const int q1 = (int)pl->nqp[0], q2 = (int)pl->nqp[1], q3 = (int)pl->nqp[2];
  const int64_t NQP = pl->n_qp_total;
  if (pl->opt.checked) {
    wq_status sc = wq::check_device_range(pl, d_f, sizeof(double) * (size_t)NQP, "d_f");
    if (sc == WQ_OK) sc = wq::check_device_range(pl, d_b, sizeof(double) * (size_t)pl->n_rows, "d_b");
    if (sc != WQ_OK) return sc;
  }
  const size_t need = (size_t)NQP + (size_t)q3 * q2 * n1 + (size_t)q3 * n2 * n1;
  if (!pl->load_scratch) {
    wq_status st = wq::plan_alloc(pl, (void**)&pl->load_scratch, need * sizeof(double), s, "load vector scratch");
    if (st != WQ_OK) return st;
  }
  double* g = pl->load_scratch;
  double* T1 = g + NQP;
  double* T2 = T1 + (size_t)q3 * q2 * n1;
  const int tb = 256, NQ = pl->nq_max;
  wq::k_load_field<<<wq::blocks_for(NQP, tb), tb, 0, s>>>(d_f, pl->coef + 6 * NQP, g, NQP);
  // rules of kind (0, 0) are the first block of each direction's table
  wq::k_to_functions<<<wq::blocks_for((int64_t)n1 * q2 * q3, tb), tb, 0, s>>>(
      g, T1, q1, q2, q3, 0, n1, pl->dir[0].w, pl->dir[0].q0, pl->dir[0].nq, NQ, 1, 0, 0);
  wq::k_to_functions<<<wq::blocks_for((int64_t)n1 * n2 * q3, tb), tb, 0, s>>>(
      T1, T2, n1, q2, q3, 1, n2, pl->dir[1].w, pl->dir[1].q0, pl->dir[1].nq, NQ, 1, 0, 0);
  wq::k_to_functions<<<wq::blocks_for(pl->n_rows, tb), tb, 0, s>>>(
      T2, d_b, n1, n2, q3, 2, (int)pl->n[2], pl->dir[2].w, pl->dir[2].q0, pl->dir[2].nq, NQ, 1, 0, 0);
  wq::count_launch(4);
  WQ_CUDA_TRY(cudaGetLastError(), "load vector launch");
  return WQ_OK;
}

using wq::set_error;

// Scratch layout of the adjoint (doubles), allocated on the first call.
static size_t adjoint_scratch_doubles(const wq_plan_s* pl, size_t* off) {
  const int64_t n1 = pl->n[0], n2 = pl->n[1], n3 = pl->n[2];
  const int64_t q1 = pl->nqp[0], q2 = pl->nqp[1], q3 = pl->nqp[2];
  const int64_t NQP = pl->n_qp_total;
  const int m = pl->p + 1;
  size_t o = 0;
  off[0] = o; o += 4 * NQP;                                      // U
  off[1] = o; o += 10 * NQP;                                     // Lambda
  off[2] = o; o += 9 * NQP;                                      // dJ/dDF
  off[3] = o; o += (size_t)std::max({4 * q1 * n2 * n3, n1 * q2 * q3});            // pass-1 buffers
  off[4] = o; o += (size_t)std::max({9 * q1 * q2 * n3, n1 * n2 * q3});            // pass-2 buffers
  off[5] = o; o += (size_t)4 * (q1 + q2 + q3) * m;               // point-major rule tables
  off[6] = o; o += 2;                                            // J
  return o;
}

namespace wq {

// Plan-owned fields of the adjoint, allocated on first use (or by wq_plan_reserve).
wq_status reserve_adjoint(wq_plan_s* pl, cudaStream_t s) {
  if (pl->adj_scratch && pl->jac) return WQ_OK;
  size_t off[7];
  const size_t need = adjoint_scratch_doubles(pl, off);
  wq_status st = WQ_OK;
  if (!pl->adj_scratch) st = plan_alloc(pl, (void**)&pl->adj_scratch, need * sizeof(double), s, "adjoint fields");
  if (st == WQ_OK && !pl->jac)
    st = plan_alloc(pl, (void**)&pl->jac, 9 * (size_t)pl->n_qp_total * sizeof(double), s, "adjoint Jacobian");
  return st;
}

}  // namespace wq

extern "C" wq_status wq_adjoint(wq_plan_t plan, int which, const double* d_kappa, const double* d_lambda,
                                const double* d_u, double* h_J, double* d_grad_kappa, double* d_grad_ctrl,
                                void* stream) {
  if (!plan || !d_lambda || !d_u || which < 1 || which > 3) return set_error(WQ_ERR_INVALID_ARG, "bad argument");
  if (plan->wts || plan->Kt)
    return set_error(WQ_ERR_UNSUPPORTED, "the adjoint handles spline maps with a scalar coefficient only");
  cudaStream_t s = (cudaStream_t)stream;
  wq_plan_s* pl = plan;
  const int p = pl->p, m = p + 1, NQ = pl->nq_max;
  const int64_t N = pl->n_rows, NQP = pl->n_qp_total;
  const int n1 = (int)pl->n[0], n2 = (int)pl->n[1], n3 = (int)pl->n[2];
  const int q1 = (int)pl->nqp[0], q2 = (int)pl->nqp[1], q3 = (int)pl->nqp[2];
  if (pl->opt.checked) {
    const size_t nb = sizeof(double) * (size_t)N, qb = sizeof(double) * (size_t)NQP;
    wq_status sc = wq::check_device_range(pl, d_lambda, nb, "d_lambda");
    if (sc == WQ_OK) sc = wq::check_device_range(pl, d_u, nb, "d_u");
    if (sc == WQ_OK && d_kappa) sc = wq::check_device_range(pl, d_kappa, qb, "d_kappa");
    if (sc == WQ_OK && d_grad_kappa) sc = wq::check_device_range(pl, d_grad_kappa, qb, "d_grad_kappa");
    if (sc == WQ_OK && d_grad_ctrl) sc = wq::check_device_range(pl, d_grad_ctrl, 3 * nb, "d_grad_ctrl");
    if (sc != WQ_OK) return sc;
  }
  size_t off[7];
  adjoint_scratch_doubles(pl, off);
  wq_status st0 = wq::reserve_adjoint(pl, s);
  if (st0 != WQ_OK) return st0;
  double* U = pl->adj_scratch + off[0];
  double* L = pl->adj_scratch + off[1];
  double* Gb = pl->adj_scratch + off[2];
  double* T1 = pl->adj_scratch + off[3];
  double* T2 = pl->adj_scratch + off[4];
  double* Wp = pl->adj_scratch + off[5];
  double* Jd = pl->adj_scratch + off[6];
  double* Wpd[3] = {Wp, Wp + (size_t)4 * q1 * m, Wp + (size_t)4 * (q1 + q2) * m};
  // coefficients and the Jacobian for the current geometry
  wq_status st = wq::run_coefficients(pl, s, pl->jac);
  if (st != WQ_OK) return st;
  const int tb = 256;
  for (int l = 0; l < 3; ++l) {
    const wq::DirData& d = pl->dir[l];
    wq::k_point_weights<<<wq::blocks_for(4 * d.nqp, tb), tb, 0, s>>>(d.w, d.first, d.q0, d.nq, d.n, d.nqp, p, NQ,
                                                                      Wpd[l]);
  }
  int launches = 3;
  auto to_points = [&](const double* in, double* out, int d0, int d1, int d2, int axis, const double* T, int dir) {
    int od[3] = {d0, d1, d2};
    od[axis] = (int)pl->nqp[dir];
    const int64_t total = (int64_t)od[0] * od[1] * od[2];
    wq::k_to_points<<<wq::blocks_for(total, tb), tb, 0, s>>>(in, out, d0, d1, d2, axis, od[axis], T,
                                                            pl->dir[dir].first, m);
    ++launches;
  };
  // U: contract j1, then j2, then j3 with B or B'
  const double* bp[3] = {pl->dir[0].bp, pl->dir[1].bp, pl->dir[2].bp};
  const int64_t s1 = (int64_t)q1 * n2 * n3, s2 = (int64_t)q1 * q2 * n3;
  for (int d = 0; d < 2; ++d) to_points(d_u, T1 + d * s1, n1, n2, n3, 0, bp[0] + (size_t)d * q1 * m, 0);
  const int pairs[3][2] = {{0, 0}, {1, 0}, {0, 1}};  // (d1, d2)
  for (int k = 0; k < 3; ++k)
    to_points(T1 + pairs[k][0] * s1, T2 + k * s2, q1, n2, n3, 1, bp[1] + (size_t)pairs[k][1] * q2 * m, 1);
  // U_0 = (0,0,0), U_1 = (1,0,0), U_2 = (0,1,0), U_3 = (0,0,1)
  const int ufrom[4] = {0, 1, 2, 0}, ud3[4] = {0, 0, 0, 1};
  for (int k = 0; k < 4; ++k)
    to_points(T2 + ufrom[k] * s2, U + k * NQP, q1, q2, n3, 2, bp[2] + (size_t)ud3[k] * q3 * m, 2);
  // Lambda: kinds k = 2a + b per direction; term (l, m) uses (2 delta_kl + delta_km)_k
  int kinds[10][3];
  for (int l = 0; l < 3; ++l)
    for (int mm = 0; mm < 3; ++mm)
      for (int k = 0; k < 3; ++k) kinds[3 * l + mm][k] = 2 * (k == l) + (k == mm);
  for (int k = 0; k < 3; ++k) kinds[9][k] = 0;
  for (int k = 0; k < 4; ++k) to_points(d_lambda, T1 + k * s1, n1, n2, n3, 0, Wpd[0] + (size_t)k * q1 * m, 0);
  std::vector<std::pair<int, int>> pk;
  int pidx[10];
  for (int t = 0; t < 10; ++t) {
    std::pair<int, int> key{kinds[t][0], kinds[t][1]};
    auto it = std::find(pk.begin(), pk.end(), key);
    if (it == pk.end()) {
      pk.push_back(key);
      it = pk.end() - 1;
    }
    pidx[t] = (int)(it - pk.begin());
  }
  for (size_t k = 0; k < pk.size(); ++k)
    to_points(T1 + pk[k].first * s1, T2 + k * s2, q1, n2, n3, 1, Wpd[1] + (size_t)pk[k].second * q2 * m, 1);
  for (int t = 0; t < 10; ++t) {
    if (t < 9 && !(which & 1)) continue;
    if (t == 9 && !(which & 2)) continue;
    to_points(T2 + pidx[t] * s2, L + t * NQP, q1, q2, n3, 2, Wpd[2] + (size_t)kinds[t][2] * q3 * m, 2);
  }
  // pointwise: J, dJ/dkappa, dJ/dDF
  WQ_CUDA_TRY(cudaMemsetAsync(Jd, 0, sizeof(double), s), "adjoint reset");
  wq::PointArgs pa;
  pa.nqp = NQP;
  pa.coef = pl->coef;
  pa.jac = pl->jac;
  pa.kappa = d_kappa;
  pa.U = U;
  pa.L = L;
  pa.which = which;
  pa.grad_kappa = d_grad_kappa;
  pa.gbar = d_grad_ctrl ? Gb : nullptr;
  pa.J = Jd;
  wq::k_adjoint_point<<<wq::blocks_for(NQP, tb), tb, 0, s>>>(pa);
  ++launches;
  // dJ/dC_i[r] = sum_c sum_q Gb_rc(q) d_c B_i(q): contract q1, q2, q3 with B or B'
  if (d_grad_ctrl) {
    const double* bt[3] = {pl->dir[0].bt, pl->dir[1].bt, pl->dir[2].bt};
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) {
        const double* g = Gb + (size_t)(3 * r + c) * NQP;
        const int b1 = c == 0, b2 = c == 1, b3 = c == 2;
        int64_t tot = (int64_t)n1 * q2 * q3;
        wq::k_to_functions<<<wq::blocks_for(tot, tb), tb, 0, s>>>(g, T1, q1, q2, q3, 0, n1,
                                                                   bt[0] + (size_t)b1 * n1 * NQ, pl->dir[0].q0,
                                                                   pl->dir[0].nq, NQ, 1, 0, 0);
        tot = (int64_t)n1 * n2 * q3;
        wq::k_to_functions<<<wq::blocks_for(tot, tb), tb, 0, s>>>(T1, T2, n1, q2, q3, 1, n2,
                                                                   bt[1] + (size_t)b2 * n2 * NQ, pl->dir[1].q0,
                                                                   pl->dir[1].nq, NQ, 1, 0, 0);
        tot = N;
        wq::k_to_functions<<<wq::blocks_for(tot, tb), tb, 0, s>>>(T2, d_grad_ctrl, n1, n2, q3, 2, n3,
                                                                   bt[2] + (size_t)b3 * n3 * NQ, pl->dir[2].q0,
                                                                   pl->dir[2].nq, NQ, 3, r, c > 0);
        launches += 3;
      }
  }
  wq::count_launch(launches);
  WQ_CUDA_TRY(cudaGetLastError(), "adjoint kernels");
  if (h_J) {
    WQ_CUDA_TRY(cudaMemcpyAsync(h_J, Jd, sizeof(double), cudaMemcpyDeviceToHost, s), "J copy");
    WQ_CUDA_TRY(cudaStreamSynchronize(s), "stream synchronize");
  }
  return WQ_OK;
}
