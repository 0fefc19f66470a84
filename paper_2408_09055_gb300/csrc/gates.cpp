// Gate table and insular-qubit classification (Definition 2).
//
// The paper names its gates without writing their matrices; the OpenQASM 2
// conventions are used (see include/qsim.h).  For two-qubit gates the 4x4
// index is b = b0 + 2*b1 with b0 the bit of q0; CX has its control on q0.
#include <cmath>

#include "internal.hpp"

namespace qs {

int gate_arity(int type) { return (type >= QS_CX && type < QS_NUM_GATE_TYPES) ? 2 : 1; }

bool gate_is_diagonal(int type) { return type == QS_RZ || type == QS_CZ || type == QS_CP; }

static inline void put(double* m, int dim, int r, int c, double re, double im) {
  m[2 * (r * dim + c)] = re;
  m[2 * (r * dim + c) + 1] = im;
}

void gate_matrix(const Gate& g, double* m) {
  const int dim = 1 << gate_arity(g.type);
  std::memset(m, 0, sizeof(double) * 2 * dim * dim);
  const double h = std::sqrt(0.5);
  switch (g.type) {
    case QS_H:
      put(m, 2, 0, 0, h, 0); put(m, 2, 0, 1, h, 0);
      put(m, 2, 1, 0, h, 0); put(m, 2, 1, 1, -h, 0);
      break;
    case QS_X:
      put(m, 2, 0, 1, 1, 0); put(m, 2, 1, 0, 1, 0);
      break;
    case QS_RX: {
      double c = std::cos(0.5 * g.p[0]), s = std::sin(0.5 * g.p[0]);
      put(m, 2, 0, 0, c, 0); put(m, 2, 1, 1, c, 0);
      put(m, 2, 0, 1, 0, -s); put(m, 2, 1, 0, 0, -s);
      break;
    }
    case QS_RZ: {
      double c = std::cos(0.5 * g.p[0]), s = std::sin(0.5 * g.p[0]);
      put(m, 2, 0, 0, c, -s); put(m, 2, 1, 1, c, s);
      break;
    }
    case QS_U3: {
      double c = std::cos(0.5 * g.p[0]), s = std::sin(0.5 * g.p[0]);
      double ph = g.p[1], la = g.p[2];
      put(m, 2, 0, 0, c, 0);
      put(m, 2, 0, 1, -s * std::cos(la), -s * std::sin(la));
      put(m, 2, 1, 0, s * std::cos(ph), s * std::sin(ph));
      put(m, 2, 1, 1, c * std::cos(ph + la), c * std::sin(ph + la));
      break;
    }
    case QS_CX:  // |c t> : flips t when c (bit 0) is set
      put(m, 4, 0, 0, 1, 0); put(m, 4, 2, 2, 1, 0);
      put(m, 4, 3, 1, 1, 0); put(m, 4, 1, 3, 1, 0);
      break;
    case QS_CZ:
      for (int b = 0; b < 4; ++b) put(m, 4, b, b, b == 3 ? -1 : 1, 0);
      break;
    case QS_CP:
      for (int b = 0; b < 3; ++b) put(m, 4, b, b, 1, 0);
      put(m, 4, 3, 3, std::cos(g.p[0]), std::sin(g.p[0]));
      break;
    case QS_SWAP:
      put(m, 4, 0, 0, 1, 0); put(m, 4, 3, 3, 1, 0);
      put(m, 4, 2, 1, 1, 0); put(m, 4, 1, 2, 1, 0);
      break;
    case QS_RXX: {
      double c = std::cos(0.5 * g.p[0]), s = std::sin(0.5 * g.p[0]);
      for (int b = 0; b < 4; ++b) {
        put(m, 4, b, b, c, 0);
        put(m, 4, b, 3 - b, 0, -s);  // X (x) X flips both bits: b -> b ^ 3
      }
      break;
    }
    default:
      break;
  }
}

int make_gate(const qs_gate& in, int n, Gate* out) {
  if (in.type < 0 || in.type >= QS_NUM_GATE_TYPES) return QS_EINVAL;
  const int k = gate_arity(in.type);
  if (in.nq != k) return QS_EINVAL;
  if (in.q[0] < 0 || in.q[0] >= n) return QS_EINVAL;
  if (k == 2 && (in.q[1] < 0 || in.q[1] >= n || in.q[1] == in.q[0])) return QS_EINVAL;
  for (int i = 0; i < 3; ++i)
    if (!std::isfinite(in.p[i])) return QS_EINVAL;
  Gate g;
  g.type = in.type;
  g.nq = k;
  g.q0 = in.q[0];
  g.q1 = k == 2 ? in.q[1] : -1;
  for (int i = 0; i < 3; ++i) g.p[i] = in.p[i];
  g.qmask = (1ull << g.q0) | (k == 2 ? (1ull << g.q1) : 0ull);
  if (gate_is_diagonal(g.type))
    g.nimask = 0;  // diagonal in every qubit: all insular
  else if (g.type == QS_CX)
    g.nimask = 1ull << g.q1;  // the control is insular
  else
    g.nimask = g.qmask;
  *out = g;
  return QS_OK;
}

}  // namespace qs
