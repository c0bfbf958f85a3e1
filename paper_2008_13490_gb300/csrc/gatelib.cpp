// Host gate matrices for the C ABI, written from the thesis's definitions:
//   rotations R^a(t) = exp(-i t sigma^a / 2)   Eqs. (singlequbitrotationx)-(singlequbitrotationz)
//   U1, U2, U3, R(k), +-X, +-Y, H, S, T, ...    Tab. (elementarygateset) (matrix column, verbatim)
//   CNOT                                        Eq. (cnotgate)
//   CZ = diag(1,1,1,-1)                         section on the [[4,2,2]] encoded gates
//   CP(l) = diag(1,1,1,e^{il}) (controlled U1), SWAP.
#include <cmath>
#include <cstring>

#include "internal.h"

namespace qs {

namespace {
const double kS2 = 0.70710678118654752440;
inline cd ei(double a) { return cd(std::cos(a), std::sin(a)); }

void set2(cd* m, cd a, cd b, cd c, cd d) {
  m[0] = a;
  m[1] = b;
  m[2] = c;
  m[3] = d;
}
}  // namespace

int gate_nparams(int kind) {
  switch (kind) {
    case QS_RX: case QS_RY: case QS_RZ: case QS_U1: case QS_CP: return 1;
    case QS_U2: return 2;
    case QS_U3: return 3;
    default: return 0;
  }
}

bool gate_is_two_qubit(int kind) { return kind >= QS_CNOT && kind <= QS_MAT2; }

bool gate_matrix(const qs_gate& g, cd* m, int* dim) {
  const double* p = g.param;
  const cd I(0, 1);
  *dim = 2;
  switch (g.kind) {
    case QS_I: set2(m, 1, 0, 0, 1); return true;
    case QS_X: set2(m, 0, 1, 1, 0); return true;
    case QS_Y: set2(m, 0, -I, I, 0); return true;
    case QS_Z: set2(m, 1, 0, 0, -1); return true;
    case QS_H: set2(m, kS2, kS2, kS2, -kS2); return true;
    case QS_S: set2(m, 1, 0, 0, I); return true;
    case QS_SDG: set2(m, 1, 0, 0, -I); return true;
    case QS_T: set2(m, 1, 0, 0, ei(M_PI / 4)); return true;
    case QS_TDG: set2(m, 1, 0, 0, ei(-M_PI / 4)); return true;
    case QS_PX: set2(m, kS2, I * kS2, I * kS2, kS2); return true;
    case QS_MX: set2(m, kS2, -I * kS2, -I * kS2, kS2); return true;
    case QS_PY: set2(m, kS2, kS2, -kS2, kS2); return true;
    case QS_MY: set2(m, kS2, -kS2, kS2, kS2); return true;
    case QS_RX: {
      double c = std::cos(p[0] / 2), s = std::sin(p[0] / 2);
      set2(m, c, -I * s, -I * s, c);
      return true;
    }
    case QS_RY: {
      double c = std::cos(p[0] / 2), s = std::sin(p[0] / 2);
      set2(m, c, -s, s, c);
      return true;
    }
    case QS_RZ: set2(m, ei(-p[0] / 2), 0, 0, ei(p[0] / 2)); return true;
    case QS_U1: set2(m, 1, 0, 0, ei(p[0])); return true;
    case QS_U2:
      set2(m, kS2, -kS2 * ei(p[1]), kS2 * ei(p[0]), kS2 * ei(p[0] + p[1]));
      return true;
    case QS_U3: {
      double c = std::cos(p[0] / 2), s = std::sin(p[0] / 2);
      set2(m, c, -ei(p[2]) * s, ei(p[1]) * s, ei(p[1] + p[2]) * c);
      return true;
    }
    case QS_RK: set2(m, 1, 0, 0, ei(2.0 * M_PI / std::pow(2.0, p[0]))); return true;
    case QS_MAT1:
      for (int i = 0; i < 4; ++i) m[i] = cd(g.m[2 * i], g.m[2 * i + 1]);
      return true;
    default: break;
  }
  *dim = 4;
  for (int i = 0; i < 16; ++i) m[i] = 0;
  switch (g.kind) {
    case QS_CNOT: m[0] = m[5] = m[11] = m[14] = 1; return true;
    case QS_CZ: m[0] = m[5] = m[10] = 1; m[15] = -1; return true;
    case QS_CP: m[0] = m[5] = m[10] = 1; m[15] = ei(p[0]); return true;
    case QS_SWAP: m[0] = m[6] = m[9] = m[15] = 1; return true;
    case QS_MAT2:
      for (int i = 0; i < 16; ++i) m[i] = cd(g.m[2 * i], g.m[2 * i + 1]);
      return true;
    default: return false;
  }
}

bool gate_dmatrix(const qs_gate& g, int k, cd* m) {
  const double* p = g.param;
  const cd I(0, 1);
  for (int i = 0; i < 16; ++i) m[i] = 0;
  switch (g.kind) {
    case QS_RX: {  // d/dt exp(-i t X/2) = -i/2 X R^x(t)
      double c = std::cos(p[0] / 2), s = std::sin(p[0] / 2);
      set2(m, -0.5 * s, -0.5 * I * c, -0.5 * I * c, -0.5 * s);
      return true;
    }
    case QS_RY: {
      double c = std::cos(p[0] / 2), s = std::sin(p[0] / 2);
      set2(m, -0.5 * s, -0.5 * c, 0.5 * c, -0.5 * s);
      return true;
    }
    case QS_RZ: set2(m, -0.5 * I * ei(-p[0] / 2), 0, 0, 0.5 * I * ei(p[0] / 2)); return true;
    case QS_U1: set2(m, 0, 0, 0, I * ei(p[0])); return true;
    case QS_CP: m[15] = I * ei(p[0]); return true;
    case QS_U2:
      if (k == 0) set2(m, 0, 0, kS2 * I * ei(p[0]), kS2 * I * ei(p[0] + p[1]));
      else set2(m, 0, -kS2 * I * ei(p[1]), 0, kS2 * I * ei(p[0] + p[1]));
      return true;
    case QS_U3: {
      double c = std::cos(p[0] / 2), s = std::sin(p[0] / 2);
      if (k == 0) set2(m, -0.5 * s, -0.5 * ei(p[2]) * c, 0.5 * ei(p[1]) * c, -0.5 * ei(p[1] + p[2]) * s);
      else if (k == 1) set2(m, 0, 0, I * ei(p[1]) * s, I * ei(p[1] + p[2]) * c);
      else set2(m, 0, -I * ei(p[2]) * s, 0, I * ei(p[1] + p[2]) * c);
      return true;
    }
    default: return false;
  }
}

qs_status validate_gates(const qs_gate* gates, size_t ngates, int n) {
  if (ngates > 0 && gates == nullptr) {
    set_error("gates is NULL");
    return QS_EINVAL;
  }
  for (size_t i = 0; i < ngates; ++i) {
    const qs_gate& g = gates[i];
    bool two = gate_is_two_qubit(g.kind);
    bool known = (g.kind >= QS_I && g.kind <= QS_MAT1) || two;
    if (!known) {
      set_error("gate %zu: unknown kind %d", i, g.kind);
      return QS_EINVAL;
    }
    int nq = two ? 2 : 1;
    for (int k = 0; k < nq; ++k) {
      if (g.q[k] < 0 || g.q[k] >= n) {
        set_error("gate %zu: qubit %d out of range [0,%d)", i, g.q[k], n);
        return QS_EINVAL;
      }
    }
    if (two && g.q[0] == g.q[1]) {
      set_error("gate %zu: duplicate qubit %d", i, g.q[0]);
      return QS_EINVAL;
    }
    for (int k = 0; k < gate_nparams(g.kind) || (g.kind == QS_RK && k < 1); ++k) {
      if (!std::isfinite(g.param[k])) {
        set_error("gate %zu: non-finite parameter", i);
        return QS_EINVAL;
      }
    }
    if (g.kind == QS_MAT1 || g.kind == QS_MAT2) {
      int cnt = g.kind == QS_MAT1 ? 8 : 32;
      for (int k = 0; k < cnt; ++k)
        if (!std::isfinite(g.m[k])) {
          set_error("gate %zu: non-finite matrix entry", i);
          return QS_EINVAL;
        }
    }
  }
  return QS_OK;
}

}  // namespace qs
