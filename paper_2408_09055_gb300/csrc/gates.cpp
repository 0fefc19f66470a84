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

// Pauli frame (App. A.2's reordering of anti-diagonal insular gates, taken
// to the end of the circuit).  The stored state s relates to the circuit's
// state by psi = e^{i a} (prod_q Z_q^{z_q} X_q^{x_q}) s.  An X gate only
// toggles x_q; a Clifford gate G (H, CX, CZ, SWAP) is applied as it is and
// maps the frame to G P G^dagger; any other gate G is applied as P^dagger G P
// (angles of RZ, RX, RXX, U3 change sign, CP's control flip), with the frame
// unchanged.  At the end the frame is applied as gates: X on x_q, Z = i RZ(pi)
// on z_q, and the global phase as P(a) X P(a) X on qubit 0, P(a) = U3(0,0,a).
namespace {

qs_gate mk1(int type, int q, double t0 = 0, double t1 = 0, double t2 = 0) {
  qs_gate g{};
  g.type = type;
  g.nq = 1;
  g.q[0] = q;
  g.q[1] = -1;
  g.p[0] = t0;
  g.p[1] = t1;
  g.p[2] = t2;
  return g;
}

}  // namespace

int pauli_frame_rewrite(int n, const qs_gate* in, uint64_t count, std::vector<qs_gate>* out) {
  const double pi = 3.14159265358979323846;
  std::vector<uint8_t> x(n, 0), z(n, 0);
  double a = 0;  // global phase, radians
  out->clear();
  out->reserve(count + 2 * (size_t)n + 4);
  for (uint64_t i = 0; i < count; ++i) {
    const qs_gate& g = in[i];
    if (g.type < 0 || g.type >= QS_NUM_GATE_TYPES || g.nq != gate_arity(g.type)) return QS_EINVAL;
    const int q = g.q[0], r = g.nq == 2 ? g.q[1] : -1;
    if (q < 0 || q >= n || (g.nq == 2 && (r < 0 || r >= n || r == q))) return QS_EINVAL;
    switch (g.type) {
      case QS_X:  // X Z^z X^x = (-1)^z Z^z X^(x+1)
        if (z[q]) a += pi;
        x[q] ^= 1;
        break;
      case QS_H:  // H Z^z X^x H = X^z Z^x = (-1)^(xz) Z^x X^z
        out->push_back(g);
        if (x[q] && z[q]) a += pi;
        std::swap(x[q], z[q]);
        break;
      case QS_CX:  // X_c -> X_c X_t, Z_t -> Z_c Z_t; no sign
        out->push_back(g);
        x[r] ^= x[q];
        z[q] ^= z[r];
        break;
      case QS_CZ:  // X_a -> X_a Z_b, X_b -> Z_a X_b; sign (-1)^(x_a x_b)
        out->push_back(g);
        if (x[q] && x[r]) a += pi;
        z[q] ^= x[r];
        z[r] ^= x[q];
        break;
      case QS_SWAP:
        out->push_back(g);
        std::swap(x[q], x[r]);
        std::swap(z[q], z[r]);
        break;
      case QS_RZ: {  // Z commutes; X: RZ(-t)
        qs_gate h = g;
        if (x[q]) h.p[0] = -g.p[0];
        out->push_back(h);
        break;
      }
      case QS_RX: {  // X commutes; Z: RX(-t)
        qs_gate h = g;
        if (z[q]) h.p[0] = -g.p[0];
        out->push_back(h);
        break;
      }
      case QS_RXX: {  // X's commute; Z on one qubit anticommutes with X X: RXX(-t)
        qs_gate h = g;
        if (z[q] ^ z[r]) h.p[0] = -g.p[0];
        out->push_back(h);
        break;
      }
      case QS_U3: {  // P^dagger U P = X^x Z^z U Z^z X^x
        double t = g.p[0], ph = g.p[1], la = g.p[2];
        if (z[q]) {  // Z U3(t, ph, la) Z = U3(t, ph + pi, la + pi)
          ph += pi;
          la += pi;
        }
        if (x[q]) {  // X U3(t, ph, la) X = e^{i(ph + la)} U3(-t, -ph, -la)
          a += ph + la;
          t = -t;
          ph = -ph;
          la = -la;
        }
        out->push_back(mk1(QS_U3, q, t, ph, la));
        break;
      }
      case QS_CP: {  // Z's commute; X's: the control flip (conjugate_by_x)
        const uint64_t f = ((uint64_t)x[q] << q) | ((uint64_t)x[r] << r);
        if (!conjugate_by_x(g, f, out, &a)) return QS_EINVAL;
        break;
      }
      default:
        return QS_EINVAL;
    }
  }
  for (int q = 0; q < n; ++q)
    if (x[q]) out->push_back(mk1(QS_X, q));
  for (int q = 0; q < n; ++q)
    if (z[q]) {  // Z = e^{i pi/2} RZ(pi)
      out->push_back(mk1(QS_RZ, q, pi));
      a += 0.5 * pi;
    }
  a = std::remainder(a, 2 * pi);
  if (std::fabs(a) > 1e-15) {
    const qs_gate p = mk1(QS_U3, 0, 0.0, 0.0, a), xg = mk1(QS_X, 0);
    for (const qs_gate& y : {p, xg, p, xg}) out->push_back(y);
  }
  return QS_OK;
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
