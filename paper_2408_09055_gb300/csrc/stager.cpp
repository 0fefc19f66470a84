// Circuit staging for chunked execution (Alg. 1's Stage, Sec. 4): splits the
// circuit into stages, each with a set of L local qubits that contains every
// non-insular qubit of the stage's gates (insular qubits may be regional:
// their value is fixed within a chunk, Definition 2).
//
// The stager searches over sequences of local sets in the spirit of the
// SnuQS baseline the paper compares against (Sec. 6), which takes as many
// gates per stage as it can: the regional qubits of a stage are chosen among
// the freely placeable ones (all but the L - kStageSlots lowest) by trying
// every choice when there are at most kMaxChoices of them (otherwise the
// local set grows in circuit order until the next gate no longer fits and
// the free slots go to the qubits the remaining gates need first), and a beam
// search keeps many partial stagings so that a stage that takes fewer gates
// can still lead to fewer stages overall.  Gates on disjoint qubits
// commute, so a stage takes every gate whose non-insular qubits are local
// and that shares no qubit with an earlier gate left for a later stage.
#include <algorithm>
#include <bit>
#include <numeric>

#include "internal.hpp"

namespace qs {

namespace {

constexpr uint64_t kMaxChoices = 4096;

// Gates of `rest` that a stage with local set S takes (circuit order).
size_t admitted(const std::vector<Gate>& g, const std::vector<int32_t>& rest, uint64_t S, uint64_t all,
                std::vector<int32_t>* take, std::vector<int32_t>* left) {
  uint64_t blocked = 0;
  size_t cnt = 0;
  for (int32_t i : rest) {
    const Gate& x = g[i];
    if ((x.qmask & blocked) || (x.nimask & ~S)) {
      blocked |= x.qmask;
      if (left) left->push_back(i);
      if (!left && blocked == all) break;
    } else {
      ++cnt;
      if (take) take->push_back(i);
    }
  }
  return cnt;
}

uint64_t binom(int a, int b) {
  if (b < 0 || b > a) return 0;
  uint64_t r = 1;
  for (int i = 1; i <= b; ++i) {
    r = r * (uint64_t)(a - b + i) / (uint64_t)i;
    if (r > (1ull << 40)) return r;
  }
  return r;
}

// The first-come local set (used when the choices are too many to try).
uint64_t grow_in_order(const std::vector<Gate>& g, const std::vector<int32_t>& rest, uint64_t low,
                       uint64_t all, int n, int L) {
  uint64_t S = low, blocked = 0;
  for (int32_t i : rest) {
    if (blocked == all) break;
    const Gate& x = g[i];
    if (x.qmask & blocked) {
      blocked |= x.qmask;
      continue;
    }
    const uint64_t T = S | x.nimask;
    if (std::popcount(T) <= L) S = T;
    else blocked |= x.qmask;
  }
  for (int32_t i : rest) {
    if (std::popcount(S) >= L) break;
    const Gate& x = g[i];
    for (int s = 0; s < x.nq && std::popcount(S) < L; ++s) {
      const int q = s == 0 ? x.q0 : x.q1;
      if ((x.nimask >> q) & 1) S |= 1ull << q;
    }
  }
  for (int q = 0; q < n && std::popcount(S) < L; ++q) S |= 1ull << q;
  return S;
}

}  // namespace

// Local sets of a stage: every choice of the regional qubits among the free
// ones (when there are at most kMaxChoices), ranked by the gates they admit;
// else the first-come set alone.
std::vector<std::pair<size_t, uint64_t>> stage_choices(const std::vector<Gate>& g,
                                                       const std::vector<int32_t>& rest, int n, int L,
                                                       int jlow, uint64_t low, uint64_t all) {
  std::vector<std::pair<size_t, uint64_t>> out;
  const int free_q = n - jlow, nreg = n - L;
  if (binom(free_q, nreg) > kMaxChoices) {
    const uint64_t S = grow_in_order(g, rest, low, all, n, L);
    out.push_back({admitted(g, rest, S, all, nullptr, nullptr), S});
    return out;
  }
  std::vector<int> pick(nreg);
  std::iota(pick.begin(), pick.end(), jlow);
  while (true) {
    uint64_t R = 0;
    for (int q : pick) R |= 1ull << q;
    const uint64_t S = all & ~R;
    out.push_back({admitted(g, rest, S, all, nullptr, nullptr), S});
    int t = nreg - 1;  // next combination in lexicographic order
    while (t >= 0 && pick[t] == n - nreg + t) --t;
    if (t < 0) break;
    pick[t]++;
    for (int u = t + 1; u < nreg; ++u) pick[u] = pick[u - 1] + 1;
  }
  // most gates first; ties keep the lexicographic order of the regional set
  std::stable_sort(out.begin(), out.end(), [](const auto& a, const auto& b) { return a.first > b.first; });
  return out;
}

// Beam search over stage sequences.  Every partial staging keeps its
// remaining gates and the qubits that became local at its stage boundaries
// (the objective of Sec. 4's ILP with no global qubits).  Each step expands
// every partial staging by every local set that takes a gate and keeps the
// `width` best children with distinct remaining gates: fewest gates left, then
// the least objective.  The first stage that takes the most gates need not
// be on a shortest staging, so the children are not limited to the best
// few sets of their parent.  All partial stagings of a step have the same
// number of stages, so the first step that covers every gate uses the
// fewest stages the search saw, and of those it takes the least objective.
// The width shrinks as the sets per stage grow (about 2^16 children a step).
constexpr int kMaxBeam = 64, kMinBeam = 6;
constexpr uint64_t kChildrenPerStep = 1u << 16;
constexpr int kScanPerKept = 16;  // children tried per kept one when removing duplicates

std::vector<uint64_t> choose_local_sets(const std::vector<Gate>& g, const std::vector<int32_t>& rest0, int n,
                                        int L, int jlow, uint64_t low, uint64_t all) {
  const uint64_t nsets = std::min<uint64_t>(binom(n - jlow, n - L), kMaxChoices + 1);
  const int width = (int)std::clamp<uint64_t>(kChildrenPerStep / std::max<uint64_t>(nsets, 1), kMinBeam, kMaxBeam);
  struct Partial {
    std::vector<int32_t> rest;
    std::vector<uint64_t> sets;
    int cost = 0;
  };
  struct Child {
    size_t left;    // gates still to stage
    int cost;       // qubits made local so far
    size_t parent;  // index into the beam
    uint64_t S;     // the stage's local set
  };
  std::vector<Partial> beam(1);
  beam[0].rest = rest0;
  while (true) {
    // every child, scored without materialising its remaining gates
    std::vector<Child> next;
    for (size_t b = 0; b < beam.size(); ++b) {
      const Partial& p = beam[b];
      const uint64_t prev = p.sets.empty() ? 0 : p.sets.back();
      for (const auto& [taken, S] : stage_choices(g, p.rest, n, L, jlow, low, all)) {
        if (taken == 0) break;  // ranked: no later set takes a gate
        const int c = p.sets.empty() ? 0 : p.cost + std::popcount(S & ~prev);
        next.push_back({p.rest.size() - taken, c, b, S});
      }
    }
    if (next.empty()) return {};
    std::stable_sort(next.begin(), next.end(), [](const Child& a, const Child& b) {
      return a.left != b.left ? a.left < b.left : a.cost < b.cost;
    });
    if (next[0].left == 0) {  // complete: the least objective among the shortest
      std::vector<uint64_t> sets = beam[next[0].parent].sets;
      sets.push_back(next[0].S);
      return sets;
    }
    // distinct remaining sets only (different choices often leave the same gates)
    std::vector<Partial> keep;
    const size_t scan = std::min(next.size(), (size_t)width * kScanPerKept);
    for (size_t i = 0; i < scan; ++i) {
      const Child& c = next[i];
      Partial q;
      admitted(g, beam[c.parent].rest, c.S, all, nullptr, &q.rest);
      bool dup = false;
      for (const Partial& k : keep)
        if (k.rest == q.rest) {
          dup = true;
          break;
        }
      if (dup) continue;
      q.sets = beam[c.parent].sets;
      q.sets.push_back(c.S);
      q.cost = c.cost;
      keep.push_back(std::move(q));
      if ((int)keep.size() == width) break;
    }
    beam.swap(keep);
  }
}

int stage_circuit(const std::vector<Gate>& g, int n, int L, std::vector<Stage>* out) {
  out->clear();
  if (L < 2 || L > n) return QS_EINVAL;
  const int jlow = std::max(0, L - kStageSlots);
  const uint64_t all = n >= 64 ? ~0ull : (1ull << n) - 1;
  const uint64_t low = jlow ? (1ull << jlow) - 1 : 0;
  std::vector<int32_t> rest(g.size());
  std::iota(rest.begin(), rest.end(), 0);
  for (const Gate& x : g)
    if (std::popcount(low | x.nimask) > L) return QS_EPLAN;
  // the local sets of all stages, by a beam search over the greedy choices
  const std::vector<uint64_t> plan = choose_local_sets(g, rest, n, L, jlow, low, all);
  size_t next = 0;
  while (!rest.empty()) {
    if (next >= plan.size()) return QS_EPLAN;
    const uint64_t S = plan[next++];
    // the stage: every gate the final set admits, in circuit order
    Stage st;
    st.local = S;
    std::vector<int32_t> left;
    admitted(g, rest, S, all, &st.gates, &left);
    if (st.gates.empty()) return QS_EPLAN;  // cannot happen: the first gate always fits
    // positions: local qubits ascending, then regional qubits ascending
    st.pos.assign(n, -1);
    st.order.clear();
    for (int q = 0; q < n; ++q)
      if ((S >> q) & 1) {
        st.pos[q] = (int32_t)st.order.size();
        st.order.push_back(q);
      }
    for (int q = 0; q < n; ++q)
      if (!((S >> q) & 1)) {
        st.pos[q] = (int32_t)st.order.size();
        st.order.push_back(q);
      }
    st.run_log = 0;
    while (st.run_log < n && ((S >> st.run_log) & 1)) st.run_log++;
    out->push_back(std::move(st));
    rest.swap(left);
  }
  return QS_OK;
}

}  // namespace qs
