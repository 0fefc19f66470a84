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

// X on the qubits of `flip` conjugates a gate: g' = X^f g X^f, written as
// gates of the table and a global phase (App. A.2: an anti-diagonal gate
// moved past a control flips the control; a diagonal factor swaps its
// entries).  Only qubits on which g is insular may be flipped (controls and
// diagonal qubits); the parts commute, so their order is free.
//   RZ(t) on q            -> RZ(-t)
//   CX, control flipped   -> CX, then X on the target
//   CZ(a,b), a flipped    -> CZ, Z_b = e^{i pi/2} RZ_b(pi); both: CZ RZ_a(pi) RZ_b(pi)
//   CP(t)(a,b), a flipped -> CP(-t), P_b(t) = e^{i t/2} RZ_b(t); both:
//                            CP(t) RZ_a(-t) RZ_b(-t)
// Returns false when g is not insular on every flipped qubit.
bool conjugate_by_x(const qs_gate& g, uint64_t flip, std::vector<qs_gate>* out, double* phase) {
  const uint64_t fa = (flip >> g.q[0]) & 1ull;
  const uint64_t fb = g.nq == 2 ? ((flip >> g.q[1]) & 1ull) : 0ull;
  if (!fa && !fb) {
    out->push_back(g);
    return true;
  }
  auto rz = [&](int q, double t) {
    qs_gate r{};
    r.type = QS_RZ;
    r.nq = 1;
    r.q[0] = q;
    r.q[1] = -1;
    r.p[0] = t;
    out->push_back(r);
  };
  const double pi = 3.14159265358979323846;
  switch (g.type) {
    case QS_RZ: {
      rz(g.q[0], -g.p[0]);
      return true;
    }
    case QS_CX: {  // q[0] control (insular), q[1] target (never flipped)
      if (fb) return false;
      out->push_back(g);
      qs_gate x{};
      x.type = QS_X;
      x.nq = 1;
      x.q[0] = g.q[1];
      x.q[1] = -1;
      out->push_back(x);
      return true;
    }
    case QS_CZ: {
      out->push_back(g);
      if (fa && fb) {
        rz(g.q[0], pi);
        rz(g.q[1], pi);
      } else {
        rz(fa ? g.q[1] : g.q[0], pi);
        *phase += 0.5 * pi;
      }
      return true;
    }
    case QS_CP: {
      const double t = g.p[0];
      qs_gate c = g;
      if (fa && fb) {
        out->push_back(c);
        rz(g.q[0], -t);
        rz(g.q[1], -t);
      } else {
        c.p[0] = -t;
        out->push_back(c);
        rz(fa ? g.q[1] : g.q[0], t);
        *phase += 0.5 * t;
      }
      return true;
    }
    default:
      return false;
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
