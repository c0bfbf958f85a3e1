/*
 * sv_ref.c -- FP64 state-vector oracle in plain C.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by oracle/cstate.py for the tests and the
 * benchmark's CPU legs; the library never links or calls it, and it shares no
 * code with the CUDA path.
 *
 * What it computes: the action of a one- or two-qubit gate embedded in the
 * n-qubit space, I x ... x U x ... x I (Eq. (singlequbitrotationmultiplequbits)
 * and, for two qubits, the CNOT-style 4x4 layout of Eq. (cnotgate)), on the 2^n
 * amplitudes a_J of Eq. (multiqubitstate).  Qubits are bit positions of J
 * (bit 0 least significant).  The embedded operator leaves every bit outside
 * the gate's qubits unchanged, so it acts independently on each group of
 * amplitudes that differ only in those bits: a pair (one qubit) or a quad (two
 * qubits).  Each loop below runs over those groups, one group per iteration,
 * in FP64; OpenMP spreads the independent groups over the host's cores.
 *
 * Storage: interleaved (re, im) doubles.  U is row-major U[out][in], (re, im)
 * interleaved; for two qubits the local index is 2 * bit(qa) + bit(qb) (qa the
 * most significant, as the control of CNOT).
 */
#include <stdint.h>

/* index J built from group number k by inserting a 0 at bit position p */
static inline uint64_t insert_zero(uint64_t k, int p) {
  const uint64_t low = k & ((1ull << p) - 1ull);
  return ((k >> p) << (p + 1)) | low;
}

/* y = sum over l of U[o][l] x[l] for one output row o (complex, FP64) */
static inline void row_mac(const double* U, int dim, int o, const double* xr, const double* xi,
                           double* yr, double* yi) {
  double sr = 0.0, si = 0.0;
  for (int l = 0; l < dim; ++l) {
    const double ur = U[2 * (o * dim + l)], ui = U[2 * (o * dim + l) + 1];
    sr += ur * xr[l] - ui * xi[l];
    si += ur * xi[l] + ui * xr[l];
  }
  *yr = sr;
  *yi = si;
}

/* psi <- (U on qubit q) psi */
void orc_apply1(double* psi, int n, int q, const double* U) {
  const int64_t groups = (int64_t)1 << (n - 1);
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < groups; ++k) {
    const uint64_t J0 = insert_zero((uint64_t)k, q), J1 = J0 | (1ull << q);
    const double xr[2] = {psi[2 * J0], psi[2 * J1]};
    const double xi[2] = {psi[2 * J0 + 1], psi[2 * J1 + 1]};
    double yr, yi;
    row_mac(U, 2, 0, xr, xi, &yr, &yi);
    psi[2 * J0] = yr;
    psi[2 * J0 + 1] = yi;
    row_mac(U, 2, 1, xr, xi, &yr, &yi);
    psi[2 * J1] = yr;
    psi[2 * J1 + 1] = yi;
  }
}

/* psi <- (U on qubits qa, qb) psi, qa the most significant local bit */
void orc_apply2(double* psi, int n, int qa, int qb, const double* U) {
  const int64_t groups = (int64_t)1 << (n - 2);
  const int lo = qa < qb ? qa : qb, hi = qa < qb ? qb : qa;
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < groups; ++k) {
    const uint64_t base = insert_zero(insert_zero((uint64_t)k, lo), hi);
    uint64_t J[4];
    double xr[4], xi[4];
    for (int l = 0; l < 4; ++l) {
      J[l] = base | ((uint64_t)(l >> 1) << qa) | ((uint64_t)(l & 1) << qb);
      xr[l] = psi[2 * J[l]];
      xi[l] = psi[2 * J[l] + 1];
    }
    for (int o = 0; o < 4; ++o) {
      double yr, yi;
      row_mac(U, 4, o, xr, xi, &yr, &yi);
      psi[2 * J[o]] = yr;
      psi[2 * J[o] + 1] = yi;
    }
  }
}

/* p_J = |a_J|^2 (Born rule) and their sum */
double orc_probs(const double* psi, int n, double* p) {
  const int64_t N = (int64_t)1 << n;
  double s = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : s)
  for (int64_t J = 0; J < N; ++J) {
    const double v = psi[2 * J] * psi[2 * J] + psi[2 * J + 1] * psi[2 * J + 1];
    if (p) p[J] = v;
    s += v;
  }
  return s;
}

int orc_threads(void) {
#ifdef _OPENMP
  extern int omp_get_max_threads(void);
  return omp_get_max_threads();
#else
  return 1;
#endif
}
