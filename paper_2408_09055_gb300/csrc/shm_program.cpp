// Compiles the gates of a shared-memory kernel into a register-phased
// program for the device interpreter (kernels_shm.cu).
//
// Execution model of one batch (2^m amplitudes of the active set A, m in
// [10, 14]): each of the 2^(m-5) threads holds 32 amplitudes in registers,
// indexed by 5 "register" bits of the local index; the other m-5 local bits
// are its thread-index bits.  A gate is applied in registers when its
// non-insular (target) bits are register bits; controls and diagonal factors
// on any other bit use that bit's value, known per thread (thread bits) or
// per batch (non-active qubits, Appendix A.2 "Insular qubits").  When the
// next gates need other target bits, an exchange writes every register to
// the shared-memory tile and reads it back under a new register set ("phase").
//
// The scheduler runs gates in any order consistent with the kernel's
// dependencies (two gates sharing a qubit commute only when it is insular in
// both, Definition 2), choosing each phase's register bits from the targets
// of the ready gates.  The load and store phases keep local bits 0..3 (the
// forced low qubits) as the lowest lane bits so that every global access is a
// run of 16 consecutive amplitudes (128 B).
#include <algorithm>
#include <bit>
#include <cmath>
#include <complex>

#include "internal.hpp"
#include "shm_program.hpp"

namespace qs {

namespace {

using cd = std::complex<double>;

struct HostOp {
  uint32_t kind = PK_END, a = 0, b = REF_NONE, c = 0;
  cd m[4];                 // G1 matrix (row-major) or D* diagonal entries
  double x0 = 0, x1 = 0;   // XX: cos, sin
  bool single_slot = false;  // uncontrolled one-slot op (mergeable)
  PhaseMap map;            // XCHG target map
};

void assign_threads(PhaseMap& pm, int m) {
  uint32_t rmask = 0;
  for (int i = 0; i < kRegBits; ++i) rmask |= 1u << pm.R[i];
  std::vector<int> rest;
  for (int b = 0; b < m; ++b)
    if (!((rmask >> b) & 1)) rest.push_back(b);
  std::vector<int> order;
  std::vector<bool> used(m, false);
  // lanes 0..3: distinct residues mod 4 -> distinct swizzled bank groups
  for (int rho = 0; rho < 4; ++rho)
    for (int b : rest)
      if (!used[b] && (b & 3) == rho) {
        order.push_back(b);
        used[b] = true;
        break;
      }
  for (int b : rest)
    if (!used[b]) {
      order.push_back(b);
      used[b] = true;
    }
  pm.nt = m - kRegBits;
  for (int k = 0; k < pm.nt; ++k) pm.T[k] = order[k];
}

PhaseMap make_map(uint32_t rmask, int m) {
  PhaseMap pm;
  int i = 0;
  for (int b = 0; b < m && i < kRegBits; ++b)
    if ((rmask >> b) & 1) pm.R[i++] = b;
  assign_threads(pm, m);
  return pm;
}

// Fills a register set up to 5 bits: first with target bits of later
// not-yet-run gates (in order) that still fit, then with any allowed bit.
uint32_t fill_regs(uint32_t r, const std::vector<uint32_t>& tmask, const std::vector<char>& done,
                   int m, uint32_t forbid) {
  for (size_t i = 0; i < tmask.size() && std::popcount(r) < kRegBits; ++i) {
    if (done[i] || (tmask[i] & forbid)) continue;
    if (std::popcount(r | tmask[i]) <= kRegBits) r |= tmask[i];
  }
  for (int b = m - 1; b >= 0 && std::popcount(r) < kRegBits; --b)
    if (!((forbid >> b) & 1)) r |= 1u << b;
  return r;
}

uint32_t unit_mask(const cd* d) {
  uint32_t u = 0;
  for (int e = 0; e < 4; ++e) {
    float re = (float)d[e].real(), im = (float)d[e].imag();
    if (re == 1.0f && im == 0.0f) u |= 1u << e;
  }
  return u;
}

void push_floats(std::vector<uint32_t>& w, const cd* v, int n) {
  for (int i = 0; i < n; ++i) {
    float re = (float)v[i].real(), im = (float)v[i].imag();
    uint32_t a, b;
    std::memcpy(&a, &re, 4);
    std::memcpy(&b, &im, 4);
    w.push_back(a);
    w.push_back(b);
  }
}

}  // namespace

bool compile_shm_v2(const PlanImpl* p, const Kernel& K, const ShmProgram& sp, ShmProgramV2* out) {
  const int m = sp.m;
  out->ok = false;
  out->prog.clear();
  if (m < kMinPhasedM || m > kMaxShmActive) return false;
  out->m = m;
  int loc[kMaxQubits];
  for (int q = 0; q < kMaxQubits; ++q) loc[q] = -1;
  for (int j = 0; j < m; ++j) loc[sp.act[j]] = j;

  const size_t G = K.gates.size();
  std::vector<const Gate*> gs(G);
  std::vector<uint32_t> tmask(G, 0);
  for (size_t i = 0; i < G; ++i) {
    gs[i] = &p->gates[K.gates[i]];
    for (int s = 0; s < gs[i]->nq; ++s) {
      int q = s == 0 ? gs[i]->q0 : gs[i]->q1;
      if ((gs[i]->nimask >> q) & 1) {
        if (loc[q] < 0) return false;  // a target outside A: not a valid kernel
        tmask[i] |= 1u << loc[q];
      }
    }
  }
  // dependencies inside the kernel
  std::vector<std::vector<int>> succ(G);
  std::vector<int> npred(G, 0);
  for (size_t j = 0; j < G; ++j)
    for (size_t i = 0; i < j; ++i) {
      uint64_t shared = gs[i]->qmask & gs[j]->qmask;
      if (shared & (gs[i]->nimask | gs[j]->nimask)) {
        succ[i].push_back((int)j);
        npred[j]++;
      }
    }
  std::vector<char> done(G, 0);
  const uint32_t low4 = 0xF;

  std::vector<HostOp> ops;
  // initial (load) phase: register bits avoid the low local bits
  uint32_t r = 0;
  for (size_t i = 0; i < G; ++i)
    if (npred[i] == 0 && !(tmask[i] & low4) && std::popcount(r | tmask[i]) <= kRegBits) r |= tmask[i];
  r = fill_regs(r, tmask, done, m, low4);
  PhaseMap cur = make_map(r, m);
  out->load = cur;
  int slot_of[kMaxShmActive];
  auto set_slots = [&](const PhaseMap& pm) {
    for (int b = 0; b < m; ++b) slot_of[b] = -1;
    for (int i = 0; i < kRegBits; ++i) slot_of[pm.R[i]] = i;
  };
  set_slots(cur);
  auto ref = [&](int q) -> uint32_t {
    int l = loc[q];
    if (l < 0) return REF_GLOBAL | (uint32_t)q;
    if (slot_of[l] >= 0) return (uint32_t)slot_of[l];
    return REF_LOCAL | (uint32_t)l;
  };
  auto is_slot = [](uint32_t rf) { return rf < (uint32_t)kRegBits; };

  auto emit = [&](const Gate& g) {
    double gm[32];
    gate_matrix(g, gm);
    HostOp op;
    if (gate_is_diagonal(g.type)) {
      cd d[4];
      const int dim = 1 << g.nq;
      for (int b = 0; b < 4; ++b) {
        int s = g.nq == 2 ? b : (b & 1);
        d[b] = cd(gm[2 * (s * dim + s)], gm[2 * (s * dim + s) + 1]);
      }
      uint32_t r0 = ref(g.q0), r1 = g.nq == 2 ? ref(g.q1) : REF_NONE;
      // canonical order: a slot first, and ascending slots
      bool swap01 = false;
      if (r1 != REF_NONE && is_slot(r1) && (!is_slot(r0) || r1 < r0)) swap01 = true;
      if (swap01) {
        std::swap(r0, r1);
        std::swap(d[1], d[2]);
      }
      for (int e = 0; e < 4; ++e) op.m[e] = d[e];
      if (is_slot(r0) && r1 != REF_NONE && is_slot(r1)) {
        op.kind = PK_D2;
        op.a = r0;
        op.b = r1;
      } else if (is_slot(r0)) {
        op.kind = PK_D1;
        op.a = r0;
        op.b = r1;
        op.single_slot = (r1 == REF_NONE);
      } else {
        op.kind = PK_D0;
        op.a = r0;
        op.b = r1;
      }
      op.c = unit_mask(op.m);
    } else if (g.type == QS_CX || g.type == QS_X) {
      op.kind = PK_XG;
      int t = g.type == QS_CX ? g.q1 : g.q0;
      op.a = ref(t);
      op.b = g.type == QS_CX ? ref(g.q0) : REF_NONE;
      op.single_slot = (op.b == REF_NONE);
      op.m[0] = 0; op.m[1] = 1; op.m[2] = 1; op.m[3] = 0;
    } else if (g.nq == 1) {
      op.kind = PK_G1;
      op.a = ref(g.q0);
      op.b = REF_NONE;
      op.single_slot = true;
      for (int e = 0; e < 4; ++e) op.m[e] = cd(gm[2 * e], gm[2 * e + 1]);
    } else if (g.type == QS_SWAP) {
      op.kind = PK_SWAPR;
      op.a = std::min(ref(g.q0), ref(g.q1));
      op.b = std::max(ref(g.q0), ref(g.q1));
    } else if (g.type == QS_RXX) {
      op.kind = PK_XX;
      op.a = std::min(ref(g.q0), ref(g.q1));
      op.b = std::max(ref(g.q0), ref(g.q1));
      op.x0 = std::cos(0.5 * g.p[0]);
      op.x1 = std::sin(0.5 * g.p[0]);
    } else {
      return false;
    }
    // merge consecutive uncontrolled one-slot ops on the same slot
    if (op.single_slot && !ops.empty() && ops.back().single_slot && ops.back().a == op.a &&
        ops.back().kind != PK_XCHG) {
      HostOp& pr = ops.back();
      cd A[4], B[4], Cm[4];
      auto as_mat = [](const HostOp& o, cd* M) {
        if (o.kind == PK_D1) {
          M[0] = o.m[0]; M[1] = 0; M[2] = 0; M[3] = o.m[1];
        } else {
          for (int e = 0; e < 4; ++e) M[e] = o.m[e];
        }
      };
      as_mat(pr, A);
      as_mat(op, B);
      Cm[0] = B[0] * A[0] + B[1] * A[2];
      Cm[1] = B[0] * A[1] + B[1] * A[3];
      Cm[2] = B[2] * A[0] + B[3] * A[2];
      Cm[3] = B[2] * A[1] + B[3] * A[3];
      pr.kind = PK_G1;
      pr.b = REF_NONE;
      for (int e = 0; e < 4; ++e) pr.m[e] = Cm[e];
      return true;
    }
    ops.push_back(op);
    return true;
  };

  size_t remaining = G;
  int phases = 1;
  while (remaining) {
    bool progress = true;
    uint32_t rmask = 0;
    for (int i = 0; i < kRegBits; ++i) rmask |= 1u << cur.R[i];
    while (progress) {
      progress = false;
      for (size_t i = 0; i < G; ++i) {
        if (done[i] || npred[i] || (tmask[i] & ~rmask)) continue;
        if (!emit(*gs[i])) return false;
        done[i] = 1;
        --remaining;
        for (int s : succ[i]) --npred[s];
        progress = true;
      }
    }
    if (!remaining) break;
    uint32_t nr = 0;
    for (size_t i = 0; i < G; ++i)
      if (!done[i] && !npred[i] && std::popcount(nr | tmask[i]) <= kRegBits) nr |= tmask[i];
    nr = fill_regs(nr, tmask, done, m, 0);
    cur = make_map(nr, m);
    set_slots(cur);
    HostOp x;
    x.kind = PK_XCHG;
    x.map = cur;
    ops.push_back(x);
    ++phases;
  }
  // store phase: register bits must avoid the low local bits
  uint32_t rmask = 0;
  for (int i = 0; i < kRegBits; ++i) rmask |= 1u << cur.R[i];
  if (rmask & low4) {
    uint32_t nr = fill_regs(rmask & ~low4, tmask, done, m, low4);
    cur = make_map(nr, m);
    HostOp x;
    x.kind = PK_XCHG;
    x.map = cur;
    ops.push_back(x);
    ++phases;
  }
  out->store = cur;

  // serialise
  auto& w = out->prog;
  for (const HostOp& o : ops) {
    w.push_back(o.kind | (o.a << 8) | (o.b << 16) | (o.c << 24));
    switch (o.kind) {
      case PK_G1: push_floats(w, o.m, 4); break;
      case PK_D1: case PK_D2: case PK_D0: push_floats(w, o.m, 4); break;
      case PK_XX: {
        float c = (float)o.x0, s = (float)o.x1;
        uint32_t a, b;
        std::memcpy(&a, &c, 4);
        std::memcpy(&b, &s, 4);
        w.push_back(a);
        w.push_back(b);
        break;
      }
      case PK_XCHG: {
        w.back() = PK_XCHG | ((uint32_t)o.map.nt << 8);
        for (int i = 0; i < kRegBits; ++i) w.push_back(swz(1u << o.map.R[i]));
        for (int k = 0; k < o.map.nt; ++k)
          w.push_back((1u << o.map.T[k]) | (swz(1u << o.map.T[k]) << 16));
        break;
      }
      default: break;
    }
  }
  w.push_back(PK_END);

  for (int i = 0; i < kRegBits; ++i) {
    out->ld_er[i] = swz(1u << out->load.R[i]);
    out->ld_preg[i] = 1ull << sp.act[out->load.R[i]];
    out->st_preg[i] = 1ull << sp.act[out->store.R[i]];
  }
  for (int k = 0; k < kMaxThreadBits; ++k) {
    bool v = k < out->load.nt;
    out->ld_tloc[k] = v ? (1u << out->load.T[k]) : 0;
    out->ld_tswz[k] = v ? swz(1u << out->load.T[k]) : 0;
    out->ld_pthr[k] = v ? (1ull << sp.act[out->load.T[k]]) : 0;
    out->st_pthr[k] = (k < out->store.nt) ? (1ull << sp.act[out->store.T[k]]) : 0;
  }
  out->num_phases = phases;
  out->num_ops = (int)ops.size();
  out->ok = true;
  return true;
}

}  // namespace qs
