/*
 * FP64 (complex128) reference simulator -- TEST INFRASTRUCTURE ONLY.
 *
 * This is the oracle the CUDA path is checked against.  Only the tests,
 * the smoke check and the benchmark's CPU-baseline leg load it; the product
 * library never links, includes or calls anything here, and shares no code
 * with it.
 *
 * What it computes: the plain definition of circuit simulation.  Gates are
 * applied one at a time, in circuit order, to a 2^n vector of complex128
 * amplitudes (Sec. 2 "Quantum Information Fundamentals").  A 1-qubit gate on
 * qubit q updates the pairs (alpha_f(i), alpha_f(i)+2^q) with
 * f(i) = 2^(q+1) floor(i / 2^q) + (i mod 2^q), i in [0, 2^(n-1)) -- Eq. 1.
 * A 2-qubit gate on (q0, q1) is the same construction with two inserted
 * bits: for every index with both bits clear, the four amplitudes
 * b = b0 + 2 b1 (b0 the bit of q0, b1 the bit of q1) are multiplied by the
 * 4x4 matrix.
 *
 * Gate matrices (the paper names the gates but never writes them; the
 * OpenQASM 2 conventions are used):
 *   H    = [[1, 1], [1, -1]] / sqrt2
 *   X    = [[0, 1], [1, 0]]
 *   RX(t)= [[cos t/2, -i sin t/2], [-i sin t/2, cos t/2]]
 *   RZ(t)= diag(e^{-it/2}, e^{it/2})
 *   U3(t,p,l) = [[cos t/2, -e^{il} sin t/2], [e^{ip} sin t/2, e^{i(p+l)} cos t/2]]
 *   CX   : control q0, target q1: swaps b = 1 (q0=1,q1=0) and b = 3
 *   CZ   = diag(1, 1, 1, -1);  CP(t) = diag(1, 1, 1, e^{it})
 *   SWAP : swaps b = 1 and b = 2
 *   RXX(t) = cos(t/2) I - i sin(t/2) X(x)X
 *
 * Parallelism: OpenMP over independent index groups only; the arithmetic of
 * each group is exactly the definition above.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { G_H = 0, G_X, G_RX, G_RZ, G_U3, G_CX, G_CZ, G_CP, G_SWAP, G_RXX, G_NTYPES };

typedef struct {
  int32_t type, nq, q0, q1;
  double p[3];
} or_gate;

static int gate_nq(int type) { return type >= G_CX ? 2 : 1; }

#define SET(m, dim, r, c, re, im) do { (m)[2 * ((r) * (dim) + (c))] = (re); \
                                       (m)[2 * ((r) * (dim) + (c)) + 1] = (im); } while (0)

/* Writes the 2^k x 2^k matrix of a gate, row-major, complex interleaved. */
int or_gate_matrix(int type, const double* p, double* m) {
  if (type < 0 || type >= G_NTYPES) return -1;
  int dim = 1 << gate_nq(type);
  memset(m, 0, sizeof(double) * 2 * dim * dim);
  double c, s;
  switch (type) {
    case G_H:
      SET(m, 2, 0, 0, M_SQRT1_2, 0); SET(m, 2, 0, 1, M_SQRT1_2, 0);
      SET(m, 2, 1, 0, M_SQRT1_2, 0); SET(m, 2, 1, 1, -M_SQRT1_2, 0);
      break;
    case G_X:
      SET(m, 2, 0, 1, 1, 0); SET(m, 2, 1, 0, 1, 0);
      break;
    case G_RX:
      c = cos(p[0] / 2); s = sin(p[0] / 2);
      SET(m, 2, 0, 0, c, 0); SET(m, 2, 0, 1, 0, -s);
      SET(m, 2, 1, 0, 0, -s); SET(m, 2, 1, 1, c, 0);
      break;
    case G_RZ:
      SET(m, 2, 0, 0, cos(p[0] / 2), -sin(p[0] / 2));
      SET(m, 2, 1, 1, cos(p[0] / 2), sin(p[0] / 2));
      break;
    case G_U3: {
      double t = p[0], ph = p[1], la = p[2];
      c = cos(t / 2); s = sin(t / 2);
      SET(m, 2, 0, 0, c, 0);
      SET(m, 2, 0, 1, -cos(la) * s, -sin(la) * s);
      SET(m, 2, 1, 0, cos(ph) * s, sin(ph) * s);
      SET(m, 2, 1, 1, cos(ph + la) * c, sin(ph + la) * c);
      break;
    }
    case G_CX:
      SET(m, 4, 0, 0, 1, 0); SET(m, 4, 2, 2, 1, 0);
      SET(m, 4, 1, 3, 1, 0); SET(m, 4, 3, 1, 1, 0);
      break;
    case G_CZ:
      SET(m, 4, 0, 0, 1, 0); SET(m, 4, 1, 1, 1, 0);
      SET(m, 4, 2, 2, 1, 0); SET(m, 4, 3, 3, -1, 0);
      break;
    case G_CP:
      SET(m, 4, 0, 0, 1, 0); SET(m, 4, 1, 1, 1, 0);
      SET(m, 4, 2, 2, 1, 0); SET(m, 4, 3, 3, cos(p[0]), sin(p[0]));
      break;
    case G_SWAP:
      SET(m, 4, 0, 0, 1, 0); SET(m, 4, 3, 3, 1, 0);
      SET(m, 4, 1, 2, 1, 0); SET(m, 4, 2, 1, 1, 0);
      break;
    case G_RXX:
      c = cos(p[0] / 2); s = sin(p[0] / 2);
      for (int b = 0; b < 4; ++b) {
        SET(m, 4, b, b, c, 0);
        SET(m, 4, b, b ^ 3, 0, -s);
      }
      break;
  }
  return 0;
}

/* Applies one gate to psi (2^n complex128, interleaved). */
int or_apply_gate(int n, double* psi, const or_gate* g) {
  if (g->type < 0 || g->type >= G_NTYPES) return -1;
  int k = gate_nq(g->type);
  if (g->q0 < 0 || g->q0 >= n) return -2;
  if (k == 2 && (g->q1 < 0 || g->q1 >= n || g->q1 == g->q0)) return -2;
  double m[32];
  or_gate_matrix(g->type, g->p, m);
  if (k == 1) {
    const int64_t q = g->q0;
    const int64_t half = (int64_t)1 << (n - 1);
    const int64_t low = ((int64_t)1 << q) - 1;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < half; ++i) {
      int64_t i0 = ((i >> q) << (q + 1)) | (i & low); /* f(i) of Eq. 1 */
      int64_t i1 = i0 | ((int64_t)1 << q);
      double ar = psi[2 * i0], ai = psi[2 * i0 + 1];
      double br = psi[2 * i1], bi = psi[2 * i1 + 1];
      psi[2 * i0] = m[0] * ar - m[1] * ai + m[2] * br - m[3] * bi;
      psi[2 * i0 + 1] = m[0] * ai + m[1] * ar + m[2] * bi + m[3] * br;
      psi[2 * i1] = m[4] * ar - m[5] * ai + m[6] * br - m[7] * bi;
      psi[2 * i1 + 1] = m[4] * ai + m[5] * ar + m[6] * bi + m[7] * br;
    }
  } else {
    const int64_t q0 = g->q0, q1 = g->q1;
    const int64_t lo = q0 < q1 ? q0 : q1, hi = q0 < q1 ? q1 : q0;
    const int64_t quarter = (int64_t)1 << (n - 2);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < quarter; ++i) {
      /* insert a zero bit at lo, then at hi */
      int64_t t = ((i >> lo) << (lo + 1)) | (i & (((int64_t)1 << lo) - 1));
      int64_t base = ((t >> hi) << (hi + 1)) | (t & (((int64_t)1 << hi) - 1));
      int64_t idx[4];
      double vr[4], vi[4];
      for (int b = 0; b < 4; ++b) {
        idx[b] = base | ((int64_t)(b & 1) << q0) | ((int64_t)(b >> 1) << q1);
        vr[b] = psi[2 * idx[b]];
        vi[b] = psi[2 * idx[b] + 1];
      }
      for (int r = 0; r < 4; ++r) {
        double sr = 0, si = 0;
        for (int c = 0; c < 4; ++c) {
          double ur = m[2 * (4 * r + c)], ui = m[2 * (4 * r + c) + 1];
          sr += ur * vr[c] - ui * vi[c];
          si += ur * vi[c] + ui * vr[c];
        }
        psi[2 * idx[r]] = sr;
        psi[2 * idx[r] + 1] = si;
      }
    }
  }
  return 0;
}

/* Applies the gates in order.  Returns 0, or -(1 + index) of a bad gate. */
int or_apply_circuit(int n, double* psi, const or_gate* g, int64_t ng) {
  for (int64_t i = 0; i < ng; ++i)
    if (or_apply_gate(n, psi, &g[i]) != 0) return (int)(-1 - i);
  return 0;
}

/* psi <- |0...0> */
void or_zero_state(int n, double* psi) {
  int64_t len = (int64_t)2 << n;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < len; ++i) psi[i] = 0.0;
  psi[0] = 1.0;
}

double or_norm2(int n, const double* psi) {
  int64_t len = (int64_t)2 << n;
  double s = 0;
#pragma omp parallel for reduction(+ : s) schedule(static)
  for (int64_t i = 0; i < len; ++i) s += psi[i] * psi[i];
  return s;
}

/*
 * The unitary of a gate sequence restricted to k qubits (qubits[j] is the
 * circuit qubit that becomes bit j of the 2^k index): column c is the
 * result of applying the gates, in order, to basis vector |c>.  This is the
 * fused matrix of a fusion kernel (Sec. "Cost Function": the product of the
 * kernel's gate matrices).  Returns -1 if a gate touches a qubit outside
 * the list.
 */
int or_kernel_unitary(const or_gate* g, int64_t ng, const int32_t* qubits, int k, double* u) {
  int dim = 1 << k;
  or_gate* loc = (or_gate*)malloc(sizeof(or_gate) * (ng > 0 ? ng : 1));
  for (int64_t i = 0; i < ng; ++i) {
    loc[i] = g[i];
    int a = -1, b = -1;
    for (int j = 0; j < k; ++j) {
      if (qubits[j] == g[i].q0) a = j;
      if (gate_nq(g[i].type) == 2 && qubits[j] == g[i].q1) b = j;
    }
    if (a < 0 || (gate_nq(g[i].type) == 2 && b < 0)) { free(loc); return -1; }
    loc[i].q0 = a;
    loc[i].q1 = gate_nq(g[i].type) == 2 ? b : -1;
  }
  double* col = (double*)malloc(sizeof(double) * 2 * dim);
  for (int c = 0; c < dim; ++c) {
    memset(col, 0, sizeof(double) * 2 * dim);
    col[2 * c] = 1.0;
    for (int64_t i = 0; i < ng; ++i) or_apply_gate(k, col, &loc[i]);
    for (int r = 0; r < dim; ++r) {
      u[2 * (r * dim + c)] = col[2 * r];
      u[2 * (r * dim + c) + 1] = col[2 * r + 1];
    }
  }
  free(col);
  free(loc);
  return 0;
}

int or_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void or_set_threads(int t) {
#ifdef _OPENMP
  if (t > 0) omp_set_num_threads(t);
#else
  (void)t;
#endif
}
