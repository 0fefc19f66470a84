// Kernelize: the kernelization dynamic program of Alg. 3 with the
// extensible-qubit state reduction of Alg. 4 and the optimisations of
// Appendix A.2.
//
// A DP state is a set of open kernels plus the cost of the kernels already
// closed.  Each open kernel keeps its type (shared-memory or fusion), its
// qubits, its non-insular ("active") qubits -- which set a shared-memory
// kernel's active set and cost -- and its extensible qubit set ExtQ
// (Definition of extensible qubits, Sec. 6.1), maintained by Alg. 4 with its
// plain intersection test.  For every gate
// (or attached gate group) in circuit order each state branches into:
//   * adding the gate to an open kernel whose extensible sets admit it
//     (Alg. 3 line 8) -- only kernels whose ExtQ is not "all qubits"
//     (deferred merging, App. A.2), or, when the gate's qubits contain or are
//     contained in a kernel's qubits, that kernel alone (subsumption);
//   * opening a singleton kernel, once as fusion and once as shared-memory
//     (Alg. 3 line 10; Sec. 6.2).
// After the transition every other kernel's ExtQ is updated by Alg. 4; a
// kernel whose ExtQ is "all qubits" and which the gate touches may instead be
// merged with another such kernel (deferred merging).  Kernels whose
// extensible sets are empty can no longer grow: they are costed and closed.
// When a position holds T states they are ranked by their cost after the
// greedy packing post-process and the best T/2 kept (pruning).  The final
// kernel order is a topological order of the kernel dependency graph, which
// Theorem 2 guarantees to be acyclic.
#include <algorithm>
#include <bit>
#include <cmath>
#include <functional>
#include <limits>
#include <queue>
#include <unordered_map>

#include "internal.hpp"

namespace qs {

namespace {

constexpr double INF = std::numeric_limits<double>::infinity();
constexpr uint64_t ALLQ = ~0ull;  // ExtQ = all qubits
constexpr size_t kMaxDpStates = size_t(1) << 20;  // DP frontier limit (prune_T <= 0)

struct Unit {
  std::vector<int32_t> gates;  // circuit indices in order
  KStat st;
};

struct OpenK {
  uint8_t fusion = 0;
  uint64_t q = 0, ni = 0;  // mirrors of st.q / st.ni for the hot comparisons
  uint64_t ext = ALLQ;
  KStat st;
  double cost = -1;        // the kernel's cost as it stands, once known (< 0: not yet)
  int32_t id = -1;
  bool operator<(const OpenK& o) const {
    if (fusion != o.fusion) return fusion < o.fusion;
    if (q != o.q) return q < o.q;
    if (ni != o.ni) return ni < o.ni;
    return ext < o.ext;
  }
};

// History events (persistent list) for reconstructing the chosen state.
struct Event {
  int32_t kind;   // 0 assign unit -> kernel, 1 merge kernel a into b
  int32_t a, b;
  int32_t parent;
};

struct State {
  std::vector<OpenK> ks;  // sorted canonically
  double closed = 0;
  double open_cost = 0;
  int32_t hist = -1;  // last event of this state's history (Ctx::ev)
  double total() const { return closed + open_cost; }
};

struct Ctx {
  const PlanImpl* p;
  CostModel cm;
  uint64_t low;
  int shm_max, kmax, kmin;
  std::vector<Event> ev;
  std::vector<uint8_t> kfusion;  // kernel id -> type
  int32_t next_id = 0;

  double kcost(const OpenK& k) const { return k.fusion ? cm.fusion(k.st) : cm.shm(k.st); }
  bool fits(const OpenK& k) const {
    const uint64_t lim = cm.plan->exec_limit;
    if (k.fusion) return std::popcount(k.q) <= kmax && !(k.q & ~lim);
    return std::popcount(k.ni | low) <= shm_max && !((k.ni | low) & ~lim);
  }
  int32_t push(int kind, int32_t a, int32_t b, int32_t parent) {
    ev.push_back(Event{kind, a, b, parent});
    return (int32_t)ev.size() - 1;
  }
  int32_t new_id(uint8_t fusion) {
    kfusion.push_back(fusion);
    return next_id++;
  }
};

// Can unit u be appended to open kernel k (extensibility + size)?
bool admits(const Ctx& c, const OpenK& k, const Unit& u) {
  if (k.ext != ALLQ && (u.st.q & ~k.ext)) return false;  // Constraint 1 via ExtQ
  OpenK t = k;
  t.q |= u.st.q;
  t.ni |= u.st.ni;
  return c.fits(t);
}

// Alg. 4's intersection test: the gate shares a qubit with the kernel.
inline uint64_t conflict(uint64_t q1, uint64_t, uint64_t q2, uint64_t) { return q1 & q2; }

// The first pair of open kernels (in index order) that packing merges: both
// of one type and all-extensible, the union feasible and cheaper than the
// two.  Every kernel's cost must be known (OpenK::cost).
bool first_merge(const Ctx& c, const std::vector<OpenK>& ks, size_t* ia, size_t* ib, OpenK* out) {
  // two all-extensible kernels commute with every gate after their first
  // gates, so their union can sit after both sets of predecessors; any other
  // pair could close a dependency cycle.  Only those kernels are paired, in
  // index order.
  constexpr size_t kMaxListed = 256;
  uint32_t all_ext[kMaxListed];
  size_t na = 0, per_type[2] = {0, 0};
  for (size_t i = 0; i < ks.size() && na < kMaxListed; ++i)
    if (ks[i].ext == ALLQ) {
      all_ext[na++] = (uint32_t)i;
      per_type[ks[i].fusion ? 1 : 0]++;
    }
  if (na == kMaxListed) {  // too many to list: every all-extensible kernel, the slow way
    na = 0;
    per_type[0] = per_type[1] = 2;
  }
  if (per_type[0] < 2 && per_type[1] < 2) return false;
  const size_t cnt = na ? na : ks.size();
  for (size_t x = 0; x < cnt; ++x)
    for (size_t y = x + 1; y < cnt; ++y) {
      const size_t i = na ? all_ext[x] : x, j = na ? all_ext[y] : y;
      const OpenK& a = ks[i];
      const OpenK& b = ks[j];
      if (a.fusion != b.fusion) continue;
      if (a.ext != ALLQ || b.ext != ALLQ) continue;
      OpenK m = a;
      m.q |= b.q;
      m.ni |= b.ni;
      m.st.merge(b.st);
      if (!c.fits(m)) continue;
      m.cost = c.kcost(m);
      if (m.cost >= a.cost + b.cost) continue;
      *ia = i;
      *ib = j;
      *out = m;
      return true;
    }
  return false;
}

// Greedy packing of a state's open kernels (App. A.2 post-processing):
// shared-memory kernels towards the largest feasible active set, fusion
// kernels while the merged kernel is cheaper than the two.  Only kernels
// whose ExtQ is "all qubits" are merged.
// Returns the packed open cost and appends merge events when `rec` is set.
double pack(Ctx& c, const std::vector<OpenK>& ks0, bool rec, int32_t* hist) {
  size_t i = 0, j = 0;
  OpenK m;
  if (!first_merge(c, ks0, &i, &j, &m)) {  // nothing to merge: no copy
    double s = 0;
    for (const auto& k : ks0) s += k.cost;
    return s;
  }
  std::vector<OpenK> ks = ks0;
  do {
    if (rec) *hist = c.push(1, ks[j].id, ks[i].id, *hist);
    ks[i] = m;
    ks.erase(ks.begin() + j);
  } while (first_merge(c, ks, &i, &j, &m));
  double s = 0;
  for (const auto& k : ks) s += k.cost;
  return s;
}

uint64_t hash_state(const std::vector<OpenK>& ks) {
  uint64_t h = 1469598103934665603ull;
  auto mix = [&h](uint64_t v) {
    h ^= v + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2);
  };
  for (const auto& k : ks) {
    mix(k.fusion);
    mix(k.q);
    mix(k.ni);
    mix(k.ext);
  }
  return h;
}

bool same_kernels(const std::vector<OpenK>& a, const std::vector<OpenK>& b) {
  if (a.size() != b.size()) return false;
  for (size_t i = 0; i < a.size(); ++i)
    if (a[i].fusion != b[i].fusion || a[i].q != b[i].q || a[i].ni != b[i].ni ||
        a[i].ext != b[i].ext)
      return false;
  return true;
}

// Single-qubit gate attachment (App. A.2): every one-qubit gate joins the
// next multi-qubit gate on its qubit (else the previous one); when a qubit
// has no multi-qubit gate at all, its gates join the closest multi-qubit gate
// of the circuit.  Without multi-qubit gates each gate is its own unit.
std::vector<Unit> make_units(const PlanImpl* p, bool attach) {
  const int L = (int)p->gates.size();
  std::vector<int> owner(L, -1);
  std::vector<int> multi;
  for (int i = 0; i < L; ++i)
    if (p->gates[i].nq > 1) multi.push_back(i);
  if (attach && !multi.empty()) {
    for (int i = 0; i < L; ++i)
      if (p->gates[i].nq > 1) owner[i] = i;
    for (int q = 0; q < p->n; ++q) {
      std::vector<int> chain;
      for (int i = 0; i < L; ++i)
        if ((p->gates[i].qmask >> q) & 1) chain.push_back(i);
      int next_multi = -1;
      for (int t = (int)chain.size() - 1; t >= 0; --t) {
        int i = chain[t];
        if (p->gates[i].nq > 1) next_multi = i;
        else owner[i] = next_multi;
      }
      int prev_multi = -1;
      for (int i : chain) {
        if (p->gates[i].nq > 1) prev_multi = i;
        else if (owner[i] < 0) owner[i] = prev_multi;
      }
    }
    // Gates on a qubit that no multi-qubit gate touches join the closest
    // multi-qubit gate of the circuit (App. A.2), decided qubit by qubit:
    // only when every unit they join still fits a kernel (the paper does not
    // bound a unit's width); otherwise the qubit's gates stay together as a
    // unit of their own, anchored at its first gate.  Nothing else touches
    // such a qubit, so either way its gates keep their order and commute
    // with the rest.
    const uint64_t low = p->opts.forced_low <= 0 ? 0ull : ((1ull << std::min(p->opts.forced_low, p->n)) - 1);
    auto fits_some_kernel = [&](const KStat& st) {
      const uint64_t a = st.ni | low;
      const bool shm = std::popcount(a) <= p->opts.shm_max_active && !(a & ~p->exec_limit);
      const bool fused = p->opts.fuse_kmax > 0 && std::popcount(st.q) <= p->opts.fuse_kmax && !(st.q & ~p->exec_limit);
      return shm || fused;
    };
    std::vector<KStat> ust(L);  // stats of the units formed so far, by anchor
    for (int i = 0; i < L; ++i)
      if (owner[i] >= 0) ust[owner[i]].add(p->gates[i], 0.0);
    for (int q = 0; q < p->n; ++q) {
      std::vector<int> lone;
      for (int i = 0; i < L; ++i)
        if (owner[i] < 0 && ((p->gates[i].qmask >> q) & 1)) lone.push_back(i);
      if (lone.empty()) continue;
      std::vector<int> to(lone.size());
      std::vector<std::pair<int, KStat>> grown;  // anchor -> its stats with this qubit's gates
      for (size_t t = 0; t < lone.size(); ++t) {
        const int i = lone[t];
        auto it = std::lower_bound(multi.begin(), multi.end(), i);
        int best = -1;
        if (it != multi.end()) best = *it;
        if (it != multi.begin() && (best < 0 || i - *(it - 1) < best - i)) best = *(it - 1);
        to[t] = best;
        auto g = std::find_if(grown.begin(), grown.end(), [&](const auto& e) { return e.first == best; });
        if (g == grown.end()) g = grown.insert(grown.end(), {best, ust[best]});
        g->second.add(p->gates[i], 0.0);
      }
      const bool fits = std::all_of(grown.begin(), grown.end(), [&](const auto& e) { return fits_some_kernel(e.second); });
      for (size_t t = 0; t < lone.size(); ++t) owner[lone[t]] = fits ? to[t] : lone[0];
      if (fits)
        for (const auto& e : grown) ust[e.first] = e.second;
    }
  } else {
    for (int i = 0; i < L; ++i) owner[i] = i;
  }
  std::vector<int> unit_of(L, -1);
  std::vector<Unit> units;
  // units in order of their anchor
  std::vector<int> anchor_unit(L, -1);
  for (int i = 0; i < L; ++i)
    if (owner[i] == i) {
      anchor_unit[i] = (int)units.size();
      units.emplace_back();
    }
  for (int i = 0; i < L; ++i) {
    Unit& u = units[anchor_unit[owner[i]]];
    u.gates.push_back(i);
    u.st.add(p->gates[i], p->cost.gate_cost[p->gates[i].type]);
  }
  return units;
}

// Drops history events no live state can reach and renumbers the rest.
void compact(Ctx& c, std::vector<State>& states) {
  std::vector<int32_t> remap(c.ev.size(), -1);
  for (const State& s : states)
    for (int32_t h = s.hist; h >= 0 && remap[h] < 0; h = c.ev[h].parent) remap[h] = 0;
  std::vector<Event> out;
  for (size_t i = 0; i < c.ev.size(); ++i)
    if (remap[i] == 0) {
      Event e = c.ev[i];
      e.parent = e.parent >= 0 ? remap[e.parent] : -1;
      remap[i] = (int32_t)out.size();
      out.push_back(e);
    }
  for (State& s : states) s.hist = s.hist >= 0 ? remap[s.hist] : -1;
  c.ev.swap(out);
}

}  // namespace

int plan_kernelize(PlanImpl* p) {
  Ctx c{p, CostModel{p, p->learned}, 0, p->opts.shm_max_active, p->opts.fuse_kmax, p->opts.fuse_kmin, {}, {}, 0};
  c.low = (p->opts.forced_low <= 0) ? 0ull
          : ((1ull << std::min(p->opts.forced_low, p->n)) - 1);
  const bool attach = p->opts.attach_single != 0;
  std::vector<Unit> units = make_units(p, attach);
  const size_t T = p->opts.prune_T > 0 ? (size_t)p->opts.prune_T : std::numeric_limits<size_t>::max();

  std::vector<State> cur(1);
  uint64_t max_states = 1;
  for (size_t ui = 0; ui < units.size(); ++ui) {
    const Unit& u = units[ui];
    // pruning: rank by cost after packing, keep the best T/2
    if (cur.size() >= T) {
      if (c.cm.learned) {  // the packing below costs merges of all-extensible pairs
        std::vector<std::pair<KStat, bool>> want;
        for (const State& s : cur)
          for (size_t i = 0; i < s.ks.size(); ++i)
            for (size_t j = i + 1; j < s.ks.size(); ++j)
              if (s.ks[i].ext == ALLQ && s.ks[j].ext == ALLQ && s.ks[i].fusion == s.ks[j].fusion) {
                KStat m = s.ks[i].st;
                m.merge(s.ks[j].st);
                want.push_back({m, s.ks[i].fusion != 0});
              }
        c.cm.prefetch(want);
        // merges of merged kernels: discovered and predicted in batches
        c.cm.discover([&]() {
          for (const State& st : cur) {
            int32_t dummy = -1;
            pack(c, st.ks, false, &dummy);
          }
        });
      }
      std::vector<std::pair<double, size_t>> r(cur.size());
      for (size_t s = 0; s < cur.size(); ++s) {
        int32_t dummy = -1;
        r[s] = {cur[s].closed + pack(c, cur[s].ks, false, &dummy), s};
      }
      std::stable_sort(r.begin(), r.end(), [](auto& a, auto& b) { return a.first < b.first; });
      std::vector<State> keep;
      for (size_t s = 0; s < std::max<size_t>(1, T / 2); ++s) keep.push_back(std::move(cur[r[s].second]));
      cur.swap(keep);
    }
    // successors by open-kernel set: an open-addressing table from the hash
    // to the last state with that hash, chained through `chain` to the
    // earlier ones
    constexpr size_t kNone = ~size_t(0);
    std::vector<std::pair<uint64_t, size_t>> table;
    size_t tmask = 0;
    std::vector<size_t> chain;
    std::vector<State> next, staged;
    auto offer = [&](State&& s) {
      std::sort(s.ks.begin(), s.ks.end());
      const uint64_t h = hash_state(s.ks);
      size_t slot = (size_t)(h * 0x9E3779B97F4A7C15ull >> 20) & tmask;
      while (table[slot].second != kNone && table[slot].first != h) slot = (slot + 1) & tmask;
      auto& head = table[slot];
      for (size_t at = head.second; at != kNone; at = chain[at])
        if (same_kernels(next[at].ks, s.ks)) {
          if (s.total() < next[at].total()) next[at] = std::move(s);
          return;
        }
      chain.push_back(head.second);
      head = {h, next.size()};
      next.push_back(std::move(s));
    };

    // buffers reused across states and candidates
    std::vector<int> cands, restrict_now;
    std::vector<State> branch, out;
    for (const State& st : cur) {
      // candidate placements: index of the kernel receiving u, or -1/-2 for a
      // new shared-memory / fusion singleton
      cands.clear();
      int sub = -1;
      for (size_t k = 0; k < st.ks.size(); ++k) {
        const OpenK& K = st.ks[k];
        if (((u.st.q & ~K.q) == 0 || (K.q & ~u.st.q) == 0) && admits(c, K, u)) {
          sub = (int)k;
          break;
        }
      }
      if (sub >= 0) {
        cands.push_back(sub);
      } else {
        for (size_t k = 0; k < st.ks.size(); ++k)
          if (st.ks[k].ext != ALLQ && admits(c, st.ks[k], u)) cands.push_back((int)k);
        cands.push_back(-1);
        cands.push_back(-2);
      }
      for (int cand : cands) {
        State ns;
        ns.closed = st.closed;
        ns.ks = st.ks;
        ns.hist = st.hist;
        int tgt;
        if (cand >= 0) {
          OpenK& K = ns.ks[cand];
          K.q |= u.st.q;
          K.ni |= u.st.ni;
          K.st.merge(u.st);
          K.cost = -1;
          tgt = cand;
        } else {
          OpenK K;
          K.fusion = cand == -2;
          K.q = u.st.q;
          K.ni = u.st.ni;
          K.st = u.st;
          if (!c.fits(K)) continue;
          K.id = c.new_id(K.fusion);
          ns.ks.push_back(K);
          tgt = (int)ns.ks.size() - 1;
        }
        ns.hist = c.push(0, (int32_t)ui, ns.ks[tgt].id, ns.hist);
        // Alg. 4 for every other kernel; kernels about to lose "all qubits"
        // may merge with another all-extensible kernel instead (deferral).
        restrict_now.clear();
        for (size_t k = 0; k < ns.ks.size(); ++k) {
          if ((int)k == tgt) continue;
          OpenK& K = ns.ks[k];
          if (K.ext == ALLQ) {
            if (conflict(u.st.q, u.st.ni, K.q, K.ni)) restrict_now.push_back((int)k);
          } else {
            K.ext &= ~u.st.q;
          }
        }
        // expand the merge choices kernel by kernel
        branch.clear();
        branch.push_back(std::move(ns));
        for (int rk : restrict_now) {
          out.clear();
          for (State& b : branch) {
            // option 1: restrict
            {
              State r = b;
              OpenK& K = r.ks[rk];
              K.ext = K.q & ~u.st.q;
              out.push_back(std::move(r));
            }
            // option 2: merge with an all-extensible kernel
            for (size_t o = 0; o < b.ks.size(); ++o) {
              if ((int)o == rk) continue;
              const OpenK& A = b.ks[rk];
              const OpenK& B = b.ks[o];
              if (A.id == -2 || B.id == -2) continue;
              if (B.ext != ALLQ || B.fusion != A.fusion) continue;
              if (std::find(restrict_now.begin(), restrict_now.end(), (int)o) != restrict_now.end() &&
                  (int)o > rk)
                continue;  // pairs among the restricted set are taken once
              OpenK m = B;
              m.q |= A.q;
              m.ni |= A.ni;
              m.st.merge(A.st);
              m.cost = -1;
              if (!c.fits(m)) continue;
              State r = b;
              r.hist = c.push(1, A.id, B.id, r.hist);
              if ((int)o != tgt && !conflict(u.st.q, u.st.ni, B.q, B.ni)) {
                // the merged kernel is restricted by u through A's qubits
                m.ext = m.q & ~u.st.q;
              }
              r.ks[o] = m;
              r.ks[rk].id = -2;  // removed below
              out.push_back(std::move(r));
            }
          }
          branch.swap(out);
        }
        for (State& b : branch) {
          b.ks.erase(std::remove_if(b.ks.begin(), b.ks.end(), [](const OpenK& k) { return k.id == -2; }),
                     b.ks.end());
          staged.push_back(std::move(b));
        }
      }
    }
    // costs of every successor's kernels (one batch for a learned model),
    // then close the kernels that can no longer grow and keep the best state
    // per open-kernel set
    if (c.cm.learned) {
      std::vector<std::pair<KStat, bool>> want;
      for (const State& b : staged)
        for (const OpenK& K : b.ks)
          if (K.cost < 0) want.push_back({K.st, K.fusion != 0});
      c.cm.prefetch(want);
    }
    size_t tsize = 16;
    while (tsize < 2 * staged.size()) tsize <<= 1;  // at most half full
    table.assign(tsize, {0, kNone});
    tmask = tsize - 1;
    chain.reserve(staged.size());
    next.reserve(staged.size());
    for (State& b : staged) {
      double open = 0;
      size_t w = 0;  // kernels still open, compacted in place
      for (size_t r = 0; r < b.ks.size(); ++r) {
        OpenK& K = b.ks[r];
        if (K.cost < 0) K.cost = c.kcost(K);  // kernels changed by this step
        if (K.ext == 0) {
          b.closed += K.cost;
        } else {
          open += K.cost;
          if (w != r) b.ks[w] = K;
          ++w;
        }
      }
      b.ks.resize(w);
      b.open_cost = open;
      offer(std::move(b));
    }
    if (next.empty()) return QS_EPLAN;  // no feasible kernel for this gate
    if (c.ev.size() > (size_t(1) << 22)) compact(c, next);
    // without pruning the frontier can grow exponentially (Theorem 5's
    // bound): refuse before it takes the host's memory
    if (next.size() > kMaxDpStates) return QS_ENOMEM;
    cur.swap(next);
    max_states = std::max<uint64_t>(max_states, cur.size());
  }
  // final: pack every state's open kernels, keep the cheapest
  c.cm.discover([&]() {
    for (const State& st : cur) {
      int32_t dummy = -1;
      pack(c, st.ks, false, &dummy);
    }
  });
  size_t best = 0;
  double best_cost = INF;
  for (size_t s = 0; s < cur.size(); ++s) {
    int32_t dummy = -1;
    double v = cur[s].closed + pack(c, cur[s].ks, false, &dummy);
    if (v < best_cost) {
      best_cost = v;
      best = s;
    }
  }
  State fin = cur[best];
  pack(c, fin.ks, true, &fin.hist);
  p->dp_states = max_states;

  // replay the chosen history: unit -> kernel id, merges via union-find
  std::vector<int32_t> chain;
  for (int32_t h = fin.hist; h >= 0; h = c.ev[h].parent) chain.push_back(h);
  std::reverse(chain.begin(), chain.end());
  std::vector<int32_t> parent(c.next_id);
  for (int32_t i = 0; i < c.next_id; ++i) parent[i] = i;
  std::function<int32_t(int32_t)> find = [&](int32_t x) {
    while (parent[x] != x) x = parent[x] = parent[parent[x]];
    return x;
  };
  std::vector<int32_t> unit_kernel(units.size(), -1);
  for (int32_t h : chain) {
    const Event& e = c.ev[h];
    if (e.kind == 0) unit_kernel[e.a] = e.b;
    else parent[find(e.a)] = find(e.b);
  }
  std::unordered_map<int32_t, int> kidx;
  std::vector<Kernel> ks;
  std::vector<int32_t> gate_kernel(p->gates.size(), -1);
  for (size_t ui = 0; ui < units.size(); ++ui) {
    if (unit_kernel[ui] < 0) return QS_EPLAN;
    int32_t root = find(unit_kernel[ui]);
    auto it = kidx.find(root);
    if (it == kidx.end()) {
      it = kidx.emplace(root, (int)ks.size()).first;
      ks.emplace_back();
      ks.back().type = c.kfusion[root] ? QS_KERNEL_FUSED : QS_KERNEL_SHM;
    }
    for (int32_t g : units[ui].gates) {
      ks[it->second].gates.push_back(g);
      gate_kernel[g] = it->second;
    }
  }
  for (auto& k : ks) std::sort(k.gates.begin(), k.gates.end());
  // kernel dependency graph and a topological order (Theorem 2)
  const int K = (int)ks.size();
  std::vector<std::vector<int>> adj(K);
  std::vector<int> indeg(K, 0);
  auto edge = [&](int a, int b) {
    if (a < 0 || a == b) return;
    adj[a].push_back(b);
  };
  for (int q = 0; q < p->n; ++q) {
    int last_ni = -1;
    std::vector<int> ins_since;
    for (size_t i = 0; i < p->gates.size(); ++i) {
      const Gate& g = p->gates[i];
      if (!((g.qmask >> q) & 1)) continue;
      int kk = gate_kernel[i];
      if ((g.nimask >> q) & 1) {
        edge(last_ni, kk);
        for (int a : ins_since) edge(a, kk);
        ins_since.clear();
        last_ni = kk;
      } else {
        edge(last_ni, kk);
        ins_since.push_back(kk);
      }
    }
  }
  for (int a = 0; a < K; ++a) {
    std::sort(adj[a].begin(), adj[a].end());
    adj[a].erase(std::unique(adj[a].begin(), adj[a].end()), adj[a].end());
    for (int b : adj[a]) indeg[b]++;
  }
  using QE = std::pair<int32_t, int>;  // (first gate index, kernel)
  std::priority_queue<QE, std::vector<QE>, std::greater<QE>> ready;
  for (int a = 0; a < K; ++a)
    if (!indeg[a]) ready.push({ks[a].gates.front(), a});
  std::vector<int> order;
  while (!ready.empty()) {
    int a = ready.top().second;
    ready.pop();
    order.push_back(a);
    for (int b : adj[a])
      if (--indeg[b] == 0) ready.push({ks[b].gates.front(), b});
  }
  if ((int)order.size() != K) return QS_EPLAN;  // a cycle: Constraint 1 was violated
  // finish kernels in the DP's chosen type
  for (int a : order) {
    Kernel k = std::move(ks[a]);
    KStat s;
    for (int g : k.gates) s.add(p->gates[g], c.cm.gate_cost(p->gates[g].type));
    const uint64_t qm = s.q, nim = s.ni;
    double cf = c.cm.fusion(s), csh = c.cm.shm(s);
    if (k.type == QS_KERNEL_FUSED && cf == INF) k.type = QS_KERNEL_SHM;
    if (k.type == QS_KERNEL_SHM && csh == INF) k.type = QS_KERNEL_FUSED;
    if (k.type == QS_KERNEL_SHM) {
      if (csh == INF) return QS_EPLAN;
      k.mask = nim | c.low;
      k.cost = csh;
    } else {
      if (cf == INF) return QS_EPLAN;
      k.mask = qm;
      k.cost = cf;
    }
    p->kernels.push_back(std::move(k));
  }
  return QS_OK;
}

}  // namespace qs
