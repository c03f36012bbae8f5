// Internal declarations shared by the translation units of libwq.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <cstdio>
#include <string>

#include "../../include/wq.h"

namespace wq {

constexpr int kMaxP = 8;
constexpr int kMaxI = 2 * kMaxP + 1;   // |I_{l,i}| <= 2p+1
constexpr int kMaxQ = 4 * kMaxP + 1;   // |Q_{l,i}| <= 4p+1 (both boundary spans inside one support)

// Device error word bits (OR-ed by kernels, read by wq_sync_check).
enum : int {
  kErrSingularRule = 1,
  kErrBadGeometry = 2,
  kErrTimeout = 4,
  kErrNonFinite = 8,
};

// ---------------------------------------------------------------------------
// Double-double numbers: value = hi + lo with |lo| <= ulp(hi)/2.
// Error-free transformations: Knuth's two-sum and the FMA form of Dekker's
// two-product; renormalisation by the fast two-sum (|a| >= |b|).
struct dd {
  double hi, lo;
};

__host__ __device__ inline dd dd_make(double a) { return dd{a, 0.0}; }

__host__ __device__ inline dd two_sum(double a, double b) {
  double s = a + b;
  double bb = s - a;
  double e = (a - (s - bb)) + (b - bb);
  return dd{s, e};
}

__host__ __device__ inline dd fast_two_sum(double a, double b) {
  double s = a + b;
  double e = b - (s - a);
  return dd{s, e};
}

__device__ inline dd two_prod(double a, double b) {
  double p = a * b;
  double e = fma(a, b, -p);
  return dd{p, e};
}

__device__ inline dd dd_add(dd a, dd b) {
  dd s = two_sum(a.hi, b.hi);
  dd t = two_sum(a.lo, b.lo);
  s.lo += t.hi;
  s = fast_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return fast_two_sum(s.hi, s.lo);
}

__device__ inline dd dd_neg(dd a) { return dd{-a.hi, -a.lo}; }
__device__ inline dd dd_sub(dd a, dd b) { return dd_add(a, dd_neg(b)); }

__device__ inline dd dd_mul(dd a, dd b) {
  dd p = two_prod(a.hi, b.hi);
  p.lo = fma(a.hi, b.lo, fma(a.lo, b.hi, p.lo));
  return fast_two_sum(p.hi, p.lo);
}

__device__ inline dd dd_mul_d(dd a, double b) {
  dd p = two_prod(a.hi, b);
  p.lo = fma(a.lo, b, p.lo);
  return fast_two_sum(p.hi, p.lo);
}

// Long division: three quotient digits, each corrected against the exact
// remainder.
__device__ inline dd dd_div(dd a, dd b) {
  double q1 = a.hi / b.hi;
  dd r = dd_sub(a, dd_mul_d(b, q1));
  double q2 = r.hi / b.hi;
  r = dd_sub(r, dd_mul_d(b, q2));
  double q3 = r.hi / b.hi;
  dd q = fast_two_sum(q1, q2);
  return dd_add(q, dd_make(q3));
}

__device__ inline double dd_to_d(dd a) { return a.hi + a.lo; }

// ---------------------------------------------------------------------------
// Per-direction device data of a plan.
struct DirData {
  int n = 0;         // basis functions
  int n_el = 0;      // spans
  int nqp = 0;       // quadrature points
  double* knots = nullptr;   // full knot vector [n + p + 1]
  double* x = nullptr;       // points [nqp] (rounded)
  dd* x_dd = nullptr;        // points [nqp]
  int* first = nullptr;      // [nqp] first function non-zero on the point's span
  int* q0 = nullptr;         // [n] first point of Q_i
  int* nq = nullptr;         // [n] |Q_i|
  dd* bt_dd = nullptr;       // [2][n][NQ] B^{(b)}_j at q0(j)+t
  double* bt = nullptr;      // [2][n][NQ]
  double* bp = nullptr;      // [2][nqp][p+1] B^{(b)}_{first(q)+t}(x_q)
  dd* gb = nullptr;          // [n_el][p+1][2][p+1] basis at the Gauss points of each span
  dd* integ = nullptr;       // [4][n][2p+1] I^{(a,b)}_{i, i-p+t}, kind = 2a+b
  double* w = nullptr;       // [4][n][NQ] rules w^{(a,b)}_{i, q0(i)+t}
  int64_t* prefix = nullptr; // [n+1] prefix sums of the band widths |I_i|
  dd* greville = nullptr;    // [n] Greville abscissae (xi_{i+1} + ... + xi_{i+p}) / p
  int* pair_row = nullptr;   // [nnz1] row i of each band pair (staged assembly)
  float* tab32 = nullptr;    // [6][n][NQ] float copies of w and bt (staged FP32 assembly)
  void* tabf2 = nullptr;     // [6][n][NQ] double-float copies of w and bt (staged F32X2 assembly)
  dd* recip = nullptr;       // [p+1][n+p+1] 1 / (xi_{j+k} - xi_j), double-double
};

}  // namespace wq

struct wq_plan_s {
  int p = 0;
  int device = 0;
  int nq_max = 0;                 // NQ: row stride of the per-function tables
  wq::DirData dir[3];
  int64_t n[3] = {0, 0, 0};
  int64_t nqp[3] = {0, 0, 0};
  int64_t n_rows = 0, nnz = 0, n_qp_total = 0;
  int64_t nnz1[3] = {0, 0, 0};    // per-direction band totals
  double* ctrl = nullptr;         // [N*3]
  double* ctrl_delta = nullptr;   // [N*3] C_i - g_i, g_i = Greville point of i (rounded once)
  double* coef = nullptr;         // [7][N_QP]
  int64_t* row_ptr = nullptr;     // [N+1]
  int32_t* col = nullptr;         // [nnz]
  wq::dd* gauss = nullptr;        // [2][p+1]: Gauss-Legendre nodes then weights on [-1, 1]
  int* err = nullptr;             // device error word
  int tile[2] = {0, 0};           // assembly tile extents in directions 1, 2 (0 = default)
  double* jac = nullptr;          // [9][N_QP] DF at the points (allocated by the first wq_adjoint)
  double* adj_scratch = nullptr;  // adjoint fields (allocated by the first wq_adjoint)
  int algorithm = WQ_ALGO_AUTO;   // WQ_ALGO_*
  double* coefT = nullptr;        // staged: [8][N_QP] transposed coefficients (+ kappa)
  void* stg_a = nullptr;          // staged: T3
  void* stg_b = nullptr;          // staged: G
  void* stg_c = nullptr;          // staged, mixed precision: double-float edge copy of G
  void* stg_d = nullptr;          // staged, tensor-core stage 1: B fragments of the regular rows
  size_t stg_a_bytes = 0, stg_b_bytes = 0, stg_c_bytes = 0, stg_d_bytes = 0;
  wq_options opt{};               // options given at creation (defaults filled in)
  double* wts = nullptr;          // NULL (spline map), or [N] NURBS weights of the control points
  int nurbs_basis = 0;            // 1: NURBS basis functions (mass only)
  double* Kt = nullptr;           // NULL (identity), or [6][N_QP] coefficient tensor
  double* load_scratch = nullptr; // wq_assemble_load: point field and two mode-product buffers
  cudaStream_t copy_stream = nullptr;  // end-to-end call: copies back slab by slab
  cudaEvent_t slab_done = nullptr;
  cudaStream_t side_stream = nullptr;  // tensor-core stage 1: the edge rows run beside it
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
};

namespace wq {

// Thread-local error message and status helpers.
wq_status set_error(wq_status st, const std::string& msg);
wq_status cuda_error(cudaError_t e, const char* what);
void count_launch(int k = 1);

// Plan-owned device memory: the caller's allocator of wq_options, else cudaMalloc.
// plan_alloc honours WQ_FAULT=alloc; plan_free accepts NULL.
wq_status plan_alloc(wq_plan_s* pl, void** ptr, size_t bytes, cudaStream_t s, const char* what);
void plan_free(wq_plan_s* pl, void* ptr, cudaStream_t s);

// True when the comma-separated list in WQ_FAULT names `step` (host-side fault
// injection for tests).
bool fault(const char* step);

// Checked mode: `bytes` from `p` lie inside one device allocation of the plan's device.
wq_status check_device_range(const wq_plan_s* pl, const void* p, size_t bytes, const char* what);

// Plan-building steps (wq_plan.cu).
wq_status run_setup(wq_plan_s* pl, cudaStream_t s, bool with_pattern);
wq_status run_coefficients(wq_plan_s* pl, cudaStream_t s, double* jac = nullptr);

// Assembly launches (wq_assemble.cu).
wq_status launch_assemble_f64(wq_plan_s* pl, bool mass, const double* kappa, double* vals,
                              cudaStream_t s);
wq_status launch_assemble_f32(wq_plan_s* pl, bool mass, const double* kappa, void* vals,
                              int value_dtype, cudaStream_t s);
// Staged assembly (wq_staged.cu: dispatch on the degree; kernels in wq_staged_impl.cuh).
// Slabs of direction 3 for the staged assembly: `rows` rows i3 per slab (0 = as few
// slabs as the plan's scratch limit allows) and, if given, a callback run after the
// kernels of each slab [i3a, i3b) are enqueued (the values of rows with i3 in the
// slab are then final on `s` once the stream gets there).
struct SlabHook {
  int rows = 0;
  wq_status (*after)(void* ctx, int i3a, int i3b, cudaStream_t s) = nullptr;
  void* ctx = nullptr;
  // vals is page-locked host memory the device addresses: stage 1 (FP64) stores each
  // warp's values as runs of consecutive addresses, so that they cross the host link
  // as whole lines
  bool host_vals = false;
};

// vals = NULL: allocate the mode's scratch only (wq_plan_reserve).
wq_status launch_staged(wq_plan_s* pl, bool mass, const double* kappa, void* vals, int value_dtype, int precision,
                        cudaStream_t s, const SlabHook* hook = nullptr);
// Adjoint fields (wq_adjoint.cu).
wq_status reserve_adjoint(wq_plan_s* pl, cudaStream_t s);

}  // namespace wq

#define WQ_CUDA_TRY(expr, what)                        \
  do {                                                 \
    cudaError_t _e = (expr);                           \
    if (_e != cudaSuccess) return wq::cuda_error(_e, what); \
  } while (0)
