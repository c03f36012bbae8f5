/*
 * Plain C restatement of the WQ entry sums, for rows sampled from large meshes.
 *
 * TEST INFRASTRUCTURE ONLY: called from oracle/wq_oracle_c.py by the tests and
 * by the CPU-baseline legs of bench.py. The product library never links it.
 *
 * For a row i = (i1, i2, i3) and every j in I_i (ascending column order, j3
 * outer, j1 inner) it evaluates the nested sums of Eq. (massquadrature):
 *
 *   m_ij = sum_{q1 in Q_i1} w1(q1) B_j1(q1) sum_{q2 in Q_i2} w2(q2) B_j2(q2)
 *          sum_{q3 in Q_i3} w3(q3) B_j3(q3) c(q1, q2, q3)
 *
 * with the (0,0) rules and c = det DF, and for the stiffness the nine terms of
 * Eq. (stiff): the term (l, m) uses c_lm and, in direction k, the rule of kind
 * (delta_kl, delta_km) with trial values B^{(delta_km)}. Every input comes
 * from the Python oracle as dense float64 arrays:
 *
 *   W[k]   : [2][2][n_k][nqp_k]   rule weights W[a][b][i][q] (zero outside Q_i)
 *   B[k]   : [2][n_k][nqp_k]      B^{(0)}, B^{(1)} of every function at every point
 *   qlo[k], qhi[k] : [n_k]        Q_i = [qlo, qhi)
 *   coef   : [7][nqp3][nqp2][nqp1] c_11 c_12 c_13 c_22 c_23 c_33 c
 *
 * No blocking, reuse or reordering beyond the nesting of the equation.
 */
#include <stdint.h>

static int64_t imax(int64_t a, int64_t b) { return a > b ? a : b; }
static int64_t imin(int64_t a, int64_t b) { return a < b ? a : b; }

static int coef_slot(int l, int m) {
  static const int slot[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
  return slot[l][m];
}

/* which: 0 = stiffness, 1 = mass. out receives, row after row, every nonzero of
 * the row in ascending column order; out_off[r] is the start of row r in out. */
void wq_oracle_rows(int p, const int64_t* n, const int64_t* nqp,
                    const double* W1, const double* W2, const double* W3,
                    const double* B1, const double* B2, const double* B3,
                    const int64_t* qlo1, const int64_t* qhi1,
                    const int64_t* qlo2, const int64_t* qhi2,
                    const int64_t* qlo3, const int64_t* qhi3,
                    const double* coef, int which,
                    int64_t nrows, const int64_t* rows, const int64_t* out_off, double* out) {
  const double* W[3] = {W1, W2, W3};
  const double* B[3] = {B1, B2, B3};
  const int64_t* qlo[3] = {qlo1, qlo2, qlo3};
  const int64_t* qhi[3] = {qhi1, qhi2, qhi3};
  const int64_t npts = nqp[0] * nqp[1] * nqp[2];
  for (int64_t r = 0; r < nrows; ++r) {
    int64_t row = rows[r];
    int64_t i[3];
    i[0] = row % n[0];
    i[1] = (row / n[0]) % n[1];
    i[2] = row / (n[0] * n[1]);
    int64_t jlo[3], jhi[3];
    for (int k = 0; k < 3; ++k) {
      jlo[k] = imax(0, i[k] - p);
      jhi[k] = imin(n[k], i[k] + p + 1);
    }
    double* dst = out + out_off[r];
    int64_t e = 0;
    for (int64_t j3 = jlo[2]; j3 < jhi[2]; ++j3)
      for (int64_t j2 = jlo[1]; j2 < jhi[1]; ++j2)
        for (int64_t j1 = jlo[0]; j1 < jhi[0]; ++j1) {
          int64_t j[3] = {j1, j2, j3};
          double total = 0.0;
          int nterms = which == 1 ? 1 : 9;
          for (int t = 0; t < nterms; ++t) {
            int l = t / 3, m = t % 3;
            int a[3], b[3];
            const double* c;
            for (int k = 0; k < 3; ++k) {
              a[k] = which == 1 ? 0 : (k == l);
              b[k] = which == 1 ? 0 : (k == m);
            }
            c = coef + (int64_t)(which == 1 ? 6 : coef_slot(l, m)) * npts;
            /* w^{(a,b)}_{k, i_k, .} and B^{(b)}_{k, j_k}(.) rows */
            const double* w[3];
            const double* bj[3];
            for (int k = 0; k < 3; ++k) {
              w[k] = W[k] + (((int64_t)a[k] * 2 + b[k]) * n[k] + i[k]) * nqp[k];
              bj[k] = B[k] + ((int64_t)b[k] * n[k] + j[k]) * nqp[k];
            }
            double s1 = 0.0;
            for (int64_t q1 = qlo[0][i[0]]; q1 < qhi[0][i[0]]; ++q1) {
              double s2 = 0.0;
              for (int64_t q2 = qlo[1][i[1]]; q2 < qhi[1][i[1]]; ++q2) {
                double s3 = 0.0;
                for (int64_t q3 = qlo[2][i[2]]; q3 < qhi[2][i[2]]; ++q3)
                  s3 += w[2][q3] * bj[2][q3] * c[(q3 * nqp[1] + q2) * nqp[0] + q1];
                s2 += w[1][q2] * bj[1][q2] * s3;
              }
              s1 += w[0][q1] * bj[0][q1] * s2;
            }
            total += s1;
          }
          dst[e++] = total;
        }
  }
}
