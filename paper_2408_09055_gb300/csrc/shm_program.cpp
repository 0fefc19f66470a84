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
#include <cstdlib>
#include <bit>
#include <cmath>
#include <complex>

#include "internal.hpp"
#include "shm_program.hpp"

namespace qs {

namespace {

using cd = std::complex<double>;

// One op before serialisation.  kind PK_G1 with single_slot set is a raw
// uncontrolled one-slot matrix, classified into its cheapest form when the
// program is written out.
struct HostOp {
  uint32_t kind = PK_END, a = 0, b = REF_NONE, c = 0;
  cd m[4];                 // 2x2 matrix (row-major) or diagonal entries d[4]
  cd g[16];                // PK_G2: 4x4, index bit(a) + 2 bit(b)
  double x0 = 0, x1 = 0;   // XX: cos, sin
  bool single_slot = false;  // uncontrolled one-slot matrix (mergeable)
  PhaseMap map;            // XCHG target map
};

bool is_one(cd v) { return (float)v.real() == 1.0f && (float)v.imag() == 0.0f; }
bool is_zero(cd v) { return (float)v.real() == 0.0f && (float)v.imag() == 0.0f; }
bool is_real(cd v) { return (float)v.imag() == 0.0f; }
bool is_imag(cd v) { return (float)v.real() == 0.0f; }

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

bool store_sectors() {
  const char* e = std::getenv("QSIM_STORE_SECTORS");
  return !(e && e[0] == '0' && !e[1]);
}

uint32_t unit_mask(const cd* d) {
  uint32_t u = 0;
  for (int e = 0; e < 4; ++e) {
    float re = (float)d[e].real(), im = (float)d[e].imag();
    if (re == 1.0f && im == 0.0f) u |= 1u << e;
  }
  return u;
}

}  // namespace

// ---- gate fusion inside a phase -------------------------------------------
// Register ops on one or two slots commute with ops on other slots, so within
// a phase the ops touching only slots {s} or {s, t} form blocks whose product
// can replace them: a one-slot block becomes one 2x2, a two-slot block one
// dense 4x4 (PK_G2) when that is cheaper than its ops one by one.

// FP32 FMA-equivalents per amplitude of an op as the kernel applies it
double op_cost(const HostOp& o) {
  if (o.single_slot) {
    const cd* M = o.m;
    if (is_zero(M[1]) && is_zero(M[2])) return is_one(M[3] / M[0]) ? 0.0 : 2.0;
    if (is_zero(M[0]) && is_zero(M[3])) return 0.5;
    if ((is_real(M[0]) && is_real(M[1]) && is_real(M[2]) && is_real(M[3])) ||
        (is_real(M[0]) && is_imag(M[1]) && is_imag(M[2]) && is_real(M[3])))
      return 4.0;
    return 8.0;
  }
  switch (o.kind) {
    case PK_D2: return 4.0;
    case PK_D2P: return 1.0;
    case PK_XX: return 4.0;
    case PK_G2: return 16.0;
    default: return 0.0;  // renames (XGS, SWAPR)
  }
}

bool fusable(const HostOp& o) {
  if (o.single_slot) return true;
  return o.kind == PK_D2 || o.kind == PK_D2P || o.kind == PK_XGS || o.kind == PK_SWAPR || o.kind == PK_XX;
}

// register slots an op reads or writes (known-bit references excluded)
uint32_t slots_of(const HostOp& o) {
  auto bit = [](uint32_t r) { return r < (uint32_t)kRegBits ? 1u << r : 0u; };
  switch (o.single_slot ? PK_G1 : o.kind) {
    case PK_G1: case PK_G1R: case PK_G1X: case PK_XG: case PK_XGK: case PK_D1: case PK_D1B: case PK_D1K:
    case PK_G1C:
      return bit(o.a) | (o.kind == PK_G1C ? bit(o.b) : 0u);
    case PK_XGS: case PK_D2: case PK_D2P: case PK_SWAPR: case PK_XX: case PK_G2:
      return bit(o.a) | bit(o.b);
    default:
      return 0u;  // D0, SCALE: scalar per thread
  }
}

// the op as a 4x4 on slots (sa < sb), index bit(sa) + 2 bit(sb)
void op_matrix4(const HostOp& o, uint32_t sa, uint32_t sb, cd* G) {
  (void)sb;  // index bit 1 is slot sb: every slot of the op that is not sa
  for (int e = 0; e < 16; ++e) G[e] = 0.0;
  auto bits = [&](int i, uint32_t slot) { return slot == sa ? (i & 1) : (i >> 1); };
  if (o.single_slot) {
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) {
        const int other_i = o.a == sa ? (i >> 1) : (i & 1), other_j = o.a == sa ? (j >> 1) : (j & 1);
        if (other_i != other_j) continue;
        G[4 * i + j] = o.m[2 * bits(i, o.a) + bits(j, o.a)];
      }
    return;
  }
  for (int j = 0; j < 4; ++j) {
    const int ja = bits(j, o.a), jb = bits(j, o.b);  // column state on (o.a, o.b)
    auto idx = [&](int xa, int xb) {  // index of the state with o.a = xa, o.b = xb
      int i = 0;
      i |= (o.a == sa ? xa : xb);
      i |= (o.a == sa ? xb : xa) << 1;
      return i;
    };
    switch (o.kind) {
      case PK_D2:
        G[4 * j + j] = o.m[ja + 2 * jb];
        break;
      case PK_D2P:
        G[4 * j + j] = (ja && jb) ? o.m[3] : cd(1.0);
        break;
      case PK_XGS:  // target o.a, control o.b
        G[4 * idx(jb ? 1 - ja : ja, jb) + j] = 1.0;
        break;
      case PK_SWAPR:
        G[4 * idx(jb, ja) + j] = 1.0;
        break;
      case PK_XX:
        G[4 * j + j] = o.x0;
        G[4 * idx(1 - ja, 1 - jb) + j] = cd(0.0, -o.x1);
        break;
      case PK_G2:
        for (int i = 0; i < 4; ++i) G[4 * i + j] = o.g[4 * i + j];  // same slot order by construction
        break;
      default:
        break;
    }
  }
}

void matmul4(const cd* A, const cd* B, cd* C) {  // C = A B
  cd t[16];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      cd acc = 0.0;
      for (int k = 0; k < 4; ++k) acc += A[4 * i + k] * B[4 * k + j];
      t[4 * i + j] = acc;
    }
  for (int e = 0; e < 16; ++e) C[e] = t[e];
}

// Appends one-slot matrix op `op` to ops, merged into the previous op when
// that is a one-slot matrix on the same slot.
void push_merged(std::vector<HostOp>& ops, const HostOp& op) {
  if (op.single_slot && !ops.empty() && ops.back().single_slot && ops.back().a == op.a) {
    HostOp& pr = ops.back();
    const cd* A = pr.m;
    const cd* B = op.m;
    cd Cm[4] = {B[0] * A[0] + B[1] * A[2], B[0] * A[1] + B[1] * A[3],
                B[2] * A[0] + B[3] * A[2], B[2] * A[1] + B[3] * A[3]};
    for (int e = 0; e < 4; ++e) pr.m[e] = Cm[e];
    return;
  }
  ops.push_back(op);
}

// Fuses the ops of one phase (no exchange inside) into `out`.
void fuse_phase(const std::vector<HostOp>& in, std::vector<HostOp>& out) {
  struct Block {
    bool open = false;
    uint32_t sa = 0, sb = 0;   // sb = sa: one-slot block
    cd m2[4];                  // one-slot product
    cd g[16];                  // two-slot product
    std::vector<HostOp> orig;  // the ops, in order
  };
  std::vector<Block> blocks;
  int of[kRegBits];
  for (int i = 0; i < kRegBits; ++i) of[i] = -1;
  auto close = [&](int bi) {
    Block& b = blocks[bi];
    if (!b.open) return;
    b.open = false;
    of[b.sa] = -1;
    of[b.sb] = -1;
    if (b.sa == b.sb) {  // one slot: the product, as one raw matrix
      HostOp o;
      o.kind = PK_G1;
      o.single_slot = true;
      o.a = b.sa;
      for (int e = 0; e < 4; ++e) o.m[e] = b.m2[e];
      push_merged(out, o);
      return;
    }
    double c = 0;
    for (const HostOp& o : b.orig) c += op_cost(o);
    if (c > 16.0) {
      HostOp o;
      o.kind = PK_G2;
      o.a = b.sa;
      o.b = b.sb;
      for (int e = 0; e < 16; ++e) o.g[e] = b.g[e];
      out.push_back(o);
    } else {
      for (const HostOp& o : b.orig) push_merged(out, o);
    }
  };
  auto embed_single = [&](const Block& s1, uint32_t sa, uint32_t sb, cd* G) {
    HostOp t;
    t.single_slot = true;
    t.a = s1.sa;
    for (int e = 0; e < 4; ++e) t.m[e] = s1.m2[e];
    op_matrix4(t, sa, sb, G);
  };
  for (const HostOp& op : in) {
    const uint32_t sl = slots_of(op);
    if (!fusable(op)) {
      for (int s = 0; s < kRegBits; ++s)
        if (((sl >> s) & 1) && of[s] >= 0) close(of[s]);
      out.push_back(op);
      continue;
    }
    if (op.single_slot) {
      const uint32_t s = op.a;
      if (of[s] < 0) {
        Block b;
        b.open = true;
        b.sa = b.sb = s;
        for (int e = 0; e < 4; ++e) b.m2[e] = op.m[e];
        b.orig.push_back(op);
        of[s] = (int)blocks.size();
        blocks.push_back(std::move(b));
        continue;
      }
      Block& b = blocks[of[s]];
      b.orig.push_back(op);
      if (b.sa == b.sb) {
        const cd* A = b.m2;
        const cd* B = op.m;
        cd Cm[4] = {B[0] * A[0] + B[1] * A[2], B[0] * A[1] + B[1] * A[3],
                    B[2] * A[0] + B[3] * A[2], B[2] * A[1] + B[3] * A[3]};
        for (int e = 0; e < 4; ++e) b.m2[e] = Cm[e];
      } else {
        cd G[16];
        op_matrix4(op, b.sa, b.sb, G);
        matmul4(G, b.g, b.g);
      }
      continue;
    }
    // a two-slot op
    const uint32_t sa = std::min(op.a, op.b), sb = std::max(op.a, op.b);
    int ba = of[sa], bb = of[sb];
    if (ba >= 0 && ba == bb && blocks[ba].sa != blocks[ba].sb) {
      Block& b = blocks[ba];
      b.orig.push_back(op);
      cd G[16];
      op_matrix4(op, sa, sb, G);
      matmul4(G, b.g, b.g);
      continue;
    }
    // blocks pairing sa or sb with a third slot end here
    for (int x : {ba, bb})
      if (x >= 0 && blocks[x].open && blocks[x].sa != blocks[x].sb) close(x);
    ba = of[sa];
    bb = of[sb];
    Block nb;
    nb.open = true;
    nb.sa = sa;
    nb.sb = sb;
    for (int e = 0; e < 16; ++e) nb.g[e] = (e % 5 == 0) ? cd(1.0) : cd(0.0);
    for (int x : {ba, bb}) {  // absorb the one-slot blocks (they commute)
      if (x < 0) continue;
      Block& s1 = blocks[x];
      cd G[16];
      embed_single(s1, sa, sb, G);
      matmul4(G, nb.g, nb.g);
      for (const HostOp& o : s1.orig) nb.orig.push_back(o);
      s1.open = false;
    }
    nb.orig.push_back(op);
    cd G[16];
    op_matrix4(op, sa, sb, G);
    matmul4(G, nb.g, nb.g);
    of[sa] = of[sb] = (int)blocks.size();
    blocks.push_back(std::move(nb));
  }
  for (size_t bi = 0; bi < blocks.size(); ++bi) close((int)bi);
}

bool compile_shm_v2(const PlanImpl* p, const Kernel& K, const ShmProgram& sp, ShmProgramV2* out) {
  const int m = sp.m;
  out->ok = false;
  out->prog.clear();
  if (m < kMinPhasedM || m > kMaxShmActive) return false;
  for (int j = 0; j < m; ++j)
    if (sp.act[j] >= 32) return false;  // 32-bit amplitude offsets inside a batch
  out->m = m;
  int loc[kMaxQubits];
  for (int q = 0; q < kMaxQubits; ++q) loc[q] = -1;
  uint64_t amask = 0;
  for (int j = 0; j < m; ++j) {
    loc[sp.act[j]] = j;
    amask |= 1ull << sp.act[j];
  }
  // runs of non-active physical bits, for the batch-index deposit
  out->nruns = 0;
  {
    int src = 0;
    for (int q = 0; q < p->n;) {
      if ((amask >> q) & 1) {
        ++q;
        continue;
      }
      int len = 0;
      while (q + len < p->n && !((amask >> (q + len)) & 1)) ++len;
      if (out->nruns >= 16) return false;
      out->run_src[out->nruns] = (uint8_t)src;
      out->run_len[out->nruns] = (uint8_t)len;
      out->run_dst[out->nruns] = (uint8_t)q;
      out->nruns++;
      src += len;
      q += len;
    }
  }

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
  cd gphase = 1.0;
  // initial (load) phase: register bits avoid the low local bits
  uint32_t r = 0;
  for (size_t i = 0; i < G; ++i)
    if (npred[i] == 0 && !(tmask[i] & low4) && std::popcount(r | tmask[i]) <= kRegBits) r |= tmask[i];
  r = fill_regs(r, tmask, done, m, low4);
  PhaseMap cur = make_map(r, m);
  out->load = cur;
  out->maps.clear();
  out->maps.push_back(cur);
  for (int j = 0; j < m; ++j) out->act[j] = sp.act[j];
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

  // ops of the current phase, fused when the phase ends
  std::vector<HostOp> phase_ops;
  auto push = [&](HostOp op) { phase_ops.push_back(op); };
  auto end_phase = [&]() {
    fuse_phase(phase_ops, ops);
    phase_ops.clear();
  };

  auto emit = [&](const Gate& g) -> bool {
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
      // factor out d[0] as a global phase (it commutes with every gate)
      if (!is_one(d[0])) {
        cd d0 = d[0];
        gphase *= d0;
        for (int b = 0; b < 4; ++b) d[b] /= d0;
      }
      uint32_t r0 = ref(g.q0), r1 = g.nq == 2 ? ref(g.q1) : REF_NONE;
      bool swap01 = false;
      if (r1 != REF_NONE && is_slot(r1) && (!is_slot(r0) || r1 < r0)) swap01 = true;
      if (swap01) {
        std::swap(r0, r1);
        std::swap(d[1], d[2]);
      }
      if (is_slot(r0) && r1 == REF_NONE) {  // one-slot diagonal: mergeable matrix
        op.kind = PK_G1;
        op.single_slot = true;
        op.a = r0;
        op.m[0] = d[0]; op.m[1] = 0; op.m[2] = 0; op.m[3] = d[1];
      } else if (is_slot(r0) && is_slot(r1)) {
        op.a = r0;
        op.b = r1;
        for (int e = 0; e < 4; ++e) op.m[e] = d[e];
        if (is_one(d[0]) && is_one(d[1]) && is_one(d[2])) {
          if (is_one(d[3])) return true;
          op.kind = PK_D2P;
        } else {
          op.kind = PK_D2;
        }
      } else if (is_slot(r0)) {
        op.kind = PK_D1K;
        op.a = r0;
        op.b = r1;
        for (int e = 0; e < 4; ++e) op.m[e] = d[e];
        op.c = unit_mask(op.m);
      } else {
        op.kind = PK_D0;
        op.a = r0;
        op.b = r1;
        for (int e = 0; e < 4; ++e) op.m[e] = d[e];
        op.c = unit_mask(op.m);
        if (op.c == 0xF) return true;
      }
    } else if (g.type == QS_CX) {
      uint32_t t = ref(g.q1), c = ref(g.q0);
      op.a = t;
      op.b = c;
      op.kind = is_slot(c) ? PK_XGS : PK_XGK;
    } else if (g.nq == 1) {  // H, X, RX, U3
      op.kind = PK_G1;
      op.single_slot = true;
      op.a = ref(g.q0);
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
    push(op);
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
    end_phase();
    HostOp x;
    x.kind = PK_XCHG;
    x.map = cur;
    ops.push_back(x);
    out->maps.push_back(cur);
    ++phases;
  }
  end_phase();
  // store phase: local bits 0 and 1 must be lane bits, so that each group
  // of four lanes writes one whole 32-B sector; a last phase holding local
  // bit 2 or 3 in registers then stores without another exchange.
  // Measured at 30 qubits (plan A, one process): mixed circuit 499.3 ->
  // 497.5 ms, entangling circuit 321.5 -> 315.0 ms against also requiring
  // bits 2 and 3 on lanes (whole 128-B runs), which QSIM_STORE_SECTORS=0
  // restores
  uint32_t rmask = 0;
  for (int i = 0; i < kRegBits; ++i) rmask |= 1u << cur.R[i];
  if (rmask & (store_sectors() ? 0x3u : low4)) {
    uint32_t nr = fill_regs(rmask & ~low4, tmask, done, m, low4);
    cur = make_map(nr, m);
    HostOp x;
    x.kind = PK_XCHG;
    x.map = cur;
    ops.push_back(x);
    out->maps.push_back(cur);
    ++phases;
  }
  out->store = cur;

  // serialise; one-slot matrices take their cheapest form
  auto& w = out->prog;
  auto fl = [&](double v) {
    float f = (float)v;
    uint32_t u;
    std::memcpy(&u, &f, 4);
    w.push_back(u);
  };
  int nops = 0;
  for (HostOp o : ops) {
    if (o.single_slot) {
      cd* M = o.m;
      if (is_zero(M[1]) && is_zero(M[2])) {  // diagonal: factor out M[0]
        if (!is_one(M[0])) {
          gphase *= M[0];
          M[3] /= M[0];
          M[0] = 1.0;
        }
        if (is_one(M[3])) continue;  // identity
        w.push_back(PK_D1B | (o.a << 8));
        fl(M[3].real());
        fl(M[3].imag());
      } else if (is_zero(M[0]) && is_zero(M[3]) && is_one(M[1]) && is_one(M[2])) {
        w.push_back(PK_XG | (o.a << 8));
      } else if (is_real(M[0]) && is_real(M[1]) && is_real(M[2]) && is_real(M[3])) {
        w.push_back(PK_G1R | (o.a << 8));
        for (int e = 0; e < 4; ++e) fl(M[e].real());
      } else if (is_real(M[0]) && is_imag(M[1]) && is_imag(M[2]) && is_real(M[3])) {
        w.push_back(PK_G1X | (o.a << 8));
        fl(M[0].real());
        fl(M[1].imag());
        fl(M[2].imag());
        fl(M[3].real());
      } else {
        w.push_back(PK_G1 | (o.a << 8));
        if (out->g1_word < 0) out->g1_word = (int)w.size();
        for (int e = 0; e < 4; ++e) {
          fl(M[e].real());
          fl(M[e].imag());
        }
      }
      ++nops;
      continue;
    }
    w.push_back(o.kind | (o.a << 8) | (o.b << 16) | (o.c << 24));
    ++nops;
    switch (o.kind) {
      case PK_D1K: case PK_D2: case PK_D0:
        for (int e = 0; e < 4; ++e) {
          fl(o.m[e].real());
          fl(o.m[e].imag());
        }
        break;
      case PK_D2P:
        fl(o.m[3].real());
        fl(o.m[3].imag());
        break;
      case PK_XX:
        fl(o.x0);
        fl(o.x1);
        break;
      case PK_G2:
        for (int e = 0; e < 16; ++e) {
          fl(o.g[e].real());
          fl(o.g[e].imag());
        }
        break;
      case PK_XCHG:
        w.back() = PK_XCHG | ((uint32_t)o.map.nt << 8);
        for (int i = 0; i < kRegBits; ++i) w.push_back(swz(1u << o.map.R[i]));
        for (int k = 0; k < o.map.nt; ++k)
          w.push_back((1u << o.map.T[k]) | (swz(1u << o.map.T[k]) << 16));
        break;
      default:
        break;
    }
  }
  w.push_back(PK_END);
  out->phase_re = gphase.real();
  out->phase_im = gphase.imag();

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
  out->num_ops = nops;
  out->ok = true;
  return true;
}

// The global phases factored out of every phased program are applied once:
// folded into the first general 2x2 op of the plan, else appended as a
// scaling op to the last phased program.
void fold_global_phase(std::vector<ShmProgramV2>& progs) {
  cd total = 1.0;
  int last = -1;
  for (size_t i = 0; i < progs.size(); ++i)
    if (progs[i].ok) {
      total *= cd(progs[i].phase_re, progs[i].phase_im);
      last = (int)i;
    }
  if (last < 0 || is_one(total)) return;
  for (auto& pg : progs) {
    if (!pg.ok || pg.g1_word < 0) continue;
    for (int e = 0; e < 4; ++e) {
      float re, im;
      std::memcpy(&re, &pg.prog[pg.g1_word + 2 * e], 4);
      std::memcpy(&im, &pg.prog[pg.g1_word + 2 * e + 1], 4);
      cd v = cd(re, im) * total;
      float nr = (float)v.real(), ni = (float)v.imag();
      std::memcpy(&pg.prog[pg.g1_word + 2 * e], &nr, 4);
      std::memcpy(&pg.prog[pg.g1_word + 2 * e + 1], &ni, 4);
    }
    return;
  }
  auto& w = progs[last].prog;
  w.pop_back();  // PK_END
  w.push_back(PK_SCALE);
  float re = (float)total.real(), im = (float)total.imag();
  uint32_t a, b;
  std::memcpy(&a, &re, 4);
  std::memcpy(&b, &im, 4);
  w.push_back(a);
  w.push_back(b);
  w.push_back(PK_END);
  progs[last].num_ops++;
}

}  // namespace qs
