// Checks that Pauli transfer matrices describe quantum channels (host code).
//
// A PTM G of an n-qubit map E (N = 2^n, Eq. (paulitransfermatrix)):
//   G_ij = Tr(P_i E(P_j)) / N   over the Pauli strings P of Eq. (paulibasis),
// with P_i's base-4 digit b the Pauli (I, X, Y, Z) on qubit b (qubit 0 the least
// significant digit and the least significant bit of the matrix index).
//
// Trace preservation: G_0j = Tr E(P_j) / N, so E preserves traces iff the first
// row of G is (1, 0, ..., 0).
// Complete positivity: E is completely positive iff its Choi matrix
//   J(E) = (1/N) sum_ij |i><j| (x) E(|i><j|)          (Eq. (choimatrix))
// is positive semidefinite.  Writing |i><j| = sum_k (<j|P_k|i> / N) P_k and
// E(P_k) = sum_l G_lk P_l gives
//   J(E) = (1/N^2) sum_kl G_lk P_k^T (x) P_l,
// an N^2 x N^2 Hermitian matrix.  Its eigenvalues are found with the cyclic
// Jacobi method on the real symmetric form [[Re J, -Im J], [Im J, Re J]], whose
// spectrum is J's with every eigenvalue twice.
#include <cmath>
#include <complex>
#include <cstring>
#include <vector>

#include "abi_guard.h"
#include "internal.h"

namespace qs {
namespace {

using cd = std::complex<double>;

// single-qubit Pauli matrix p (0 = I, 1 = X, 2 = Y, 3 = Z), entry (r, c)
cd pauli1(int p, int r, int c) {
  switch (p) {
    case 0: return r == c ? cd(1, 0) : cd(0, 0);
    case 1: return r != c ? cd(1, 0) : cd(0, 0);
    case 2: return r == c ? cd(0, 0) : (r == 0 ? cd(0, -1) : cd(0, 1));
    default: return r == c ? (r == 0 ? cd(1, 0) : cd(-1, 0)) : cd(0, 0);
  }
}

// entry (r, c) of the Pauli string with index k on n qubits (bit b of r, c and
// base-4 digit b of k belong to qubit b)
cd pauli_string(int k, int n, int r, int c) {
  cd v(1, 0);
  for (int b = 0; b < n; ++b) v *= pauli1((k >> (2 * b)) & 3, (r >> b) & 1, (c >> b) & 1);
  return v;
}

// eigenvalues of a real symmetric m x m matrix a (row-major, destroyed): cyclic
// Jacobi rotations until the off-diagonal mass is negligible
void jacobi_eigenvalues(std::vector<double>& a, int m, std::vector<double>& ev) {
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, diag = 0.0;
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) (i == j ? diag : off) += a[i * m + j] * a[i * m + j];
    if (off <= 1e-30 * (diag + 1e-300)) break;
    for (int p = 0; p < m - 1; ++p)
      for (int q = p + 1; q < m; ++q) {
        const double apq = a[p * m + q];
        if (std::fabs(apq) < 1e-300) continue;
        const double theta = (a[q * m + q] - a[p * m + p]) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < m; ++k) {   // columns p, q
          const double akp = a[k * m + p], akq = a[k * m + q];
          a[k * m + p] = c * akp - s * akq;
          a[k * m + q] = s * akp + c * akq;
        }
        for (int k = 0; k < m; ++k) {   // rows p, q
          const double apk = a[p * m + k], aqk = a[q * m + k];
          a[p * m + k] = c * apk - s * aqk;
          a[q * m + k] = s * apk + c * aqk;
        }
      }
  }
  ev.resize(m);
  for (int i = 0; i < m; ++i) ev[i] = a[i * m + i];
}

}  // namespace

double ptm_tp_deviation(const double* G, int n) {
  const int D = 1 << (2 * n);
  double dev = std::fabs(G[0] - 1.0);
  for (int j = 1; j < D; ++j) dev = std::fmax(dev, std::fabs(G[j]));
  return dev;
}

double ptm_choi_min_eigenvalue(const double* G, int n) {
  const int N = 1 << n, D = N * N;   // D = 4^n Pauli strings; the Choi matrix is D x D
  std::vector<cd> J((size_t)D * D, cd(0, 0));
  const double scale = 1.0 / ((double)N * (double)N);
  for (int l = 0; l < D; ++l)
    for (int k = 0; k < D; ++k) {
      const double g = G[(size_t)l * D + k] * scale;
      if (g == 0.0) continue;
      // (P_k^T (x) P_l)[(r1 r2), (c1 c2)] = P_k[c1][r1] P_l[r2][c2]; the first factor
      // indexes the high half of the Choi index
      for (int r1 = 0; r1 < N; ++r1)
        for (int c1 = 0; c1 < N; ++c1) {
          const cd pk = pauli_string(k, n, c1, r1);
          if (pk == cd(0, 0)) continue;
          for (int r2 = 0; r2 < N; ++r2)
            for (int c2 = 0; c2 < N; ++c2) {
              const cd pl = pauli_string(l, n, r2, c2);
              if (pl == cd(0, 0)) continue;
              J[(size_t)(r1 * N + r2) * D + (c1 * N + c2)] += g * pk * pl;
            }
        }
    }
  const int m = 2 * D;
  std::vector<double> a((size_t)m * m);
  for (int i = 0; i < D; ++i)
    for (int j = 0; j < D; ++j) {
      // Hermitian part only (J is Hermitian for a Hermiticity-preserving map)
      const cd h = 0.5 * (J[(size_t)i * D + j] + std::conj(J[(size_t)j * D + i]));
      a[(size_t)i * m + j] = h.real();
      a[(size_t)(i + D) * m + (j + D)] = h.real();
      a[(size_t)i * m + (j + D)] = -h.imag();
      a[(size_t)(i + D) * m + j] = h.imag();
    }
  std::vector<double> ev;
  jacobi_eigenvalues(a, m, ev);
  double mn = ev[0];
  for (double e : ev) mn = std::fmin(mn, e);
  return mn;
}

// one matrix, named "what index" in the message
qs_status ptm_check_one(const double* G, int n, int index, const char* what) {
  const int D = 1 << (2 * n);
  for (int j = 0; j < D * D; ++j)
    if (!std::isfinite(G[j])) {
      set_error("%s %d: entry %d is not finite", what, index, j);
      return QS_EINVAL;
    }
  const double tp = ptm_tp_deviation(G, n);
  if (tp > kPtmTol) {
    set_error("%s %d: not trace preserving (first row deviates from (1, 0, ..., 0) by %.3g)", what,
              index, tp);
    return QS_EINVAL;
  }
  const double mn = ptm_choi_min_eigenvalue(G, n);
  if (mn < -kPtmTol) {
    set_error("%s %d: not completely positive (Choi matrix eigenvalue %.3g < 0)", what, index, mn);
    return QS_EINVAL;
  }
  return QS_OK;
}

qs_status ptm_validate(const double* ptms, int n, int count, const char* what, int* bad_index) {
  const int D = 1 << (2 * n);
  for (int i = 0; i < count; ++i) {
    const qs_status s = ptm_check_one(ptms + (size_t)i * D * D, n, i, what);
    if (s != QS_OK) {
      if (bad_index) *bad_index = i;
      return s;
    }
  }
  return QS_OK;
}

}  // namespace qs

using namespace qs;

extern "C" qs_status qs_ptm_check(const double* ptms, int n, int count, int* bad_index) {
  return abi_guard(__func__, [&]() -> qs_status {
    if (bad_index) *bad_index = -1;
    if (!ptms || n < 1 || n > 2 || count < 0) {
      set_error("qs_ptm_check: ptms required, n in {1, 2}, count >= 0");
      return QS_EINVAL;
    }
    return ptm_validate(ptms, n, count, "PTM", bad_index);
  });
}
