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
#include <unordered_map>

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

// The objective of Sec. 4's ILP with no global qubits: qubits that become
// local from one stage to the next.
int staging_objective(const std::vector<uint64_t>& sets) {
  int c = 0;
  for (size_t k = 1; k < sets.size(); ++k) c += std::popcount(sets[k] & ~sets[k - 1]);
  return c;
}

namespace {

// Branch and bound over local-set sequences for the fewest stages and then
// the least objective, the two things the ILP of Sec. 4 optimises (Theorem
// 1).  Each stage takes every gate its local set admits: a larger finished
// set never hurts later stages, so that loses no staging.  Bounds at a
// partial staging with remaining gates R, last local set P and d stages:
// the non-insular qubits U of R outside the always-local ones need at least
// ceil(|U| / free slots) more stages (and, while proving the count, as many
// as some dependency path needs: more_stages), and every qubit of U not in P
// must still become local once.  A partial staging is also dropped when one with
// the same remaining gates and last set was reached with no more stages and
// no more objective.
class ExactStager {
  static constexpr uint64_t kNodeCharge = 256;

 public:
  ExactStager(const std::vector<Gate>& g, int n, int L, int jlow, uint64_t low, uint64_t all, int64_t budget)
      : g_(g), n_(n), L_(L), jlow_(jlow), low_(low), all_(all), budget_(budget) {}

  // `best`: the incumbent staging on entry, the best found on return.
  // Returns 0 when the budget ran out first, 1 when the fewest stages are
  // proven, 2 when the least objective at that count is proven too.
  int run(const std::vector<int32_t>& rest0, std::vector<uint64_t>* best) {
    best_ = *best;
    best_s_ = (int)best_.size();
    best_cost_ = staging_objective(best_);
    // phase 1, the stage count (Theorem 1): look for a staging one stage
    // shorter than the incumbent until there is none
    while (!out_) {
      cur_.clear();
      if (!shorter(rest0, 0, best_s_ - 1)) break;
      best_ = cur_;
      best_s_ = (int)best_.size();
      best_cost_ = staging_objective(best_);
    }
    int proven = out_ ? 0 : 1;
    // phase 2, the objective at that count
    if (!out_) {
      cur_.clear();
      dfs(rest0, 0, 0, 0);
      if (!out_) proven = 2;
    }
    *best = best_;
    return proven;
  }

 private:
  struct Key {
    uint64_t h1, h2, last;
    bool operator==(const Key& o) const { return h1 == o.h1 && h2 == o.h2 && last == o.last; }
  };
  struct KeyHash {
    size_t operator()(const Key& k) const { return (size_t)(k.h1 ^ (k.h2 * 0x9E3779B97F4A7C15ull) ^ k.last); }
  };

  static Key key_of(const std::vector<int32_t>& rest, uint64_t last) {
    uint64_t h1 = 1469598103934665603ull, h2 = 0x2545F4914F6CDD1Dull;  // FNV-1a and a multiply-xorshift
    for (int32_t i : rest) {
      h1 = (h1 ^ (uint64_t)(uint32_t)i) * 1099511628211ull;
      h2 = (h2 + (uint64_t)(uint32_t)i + 1) * 0xBF58476D1CE4E5B9ull;
      h2 ^= h2 >> 31;
    }
    return {h1, h2, last};
  }

  // The lower bound on the stages still needed for `rest`: the non-insular
  // qubits it needs beyond the always-local ones, `slots` per stage.
  //
  // With `paths`, a second bound follows dependency paths: along a path of
  // gates that each share a qubit with the next, stages never decrease, and the gates
  // of one stage need at most `slots` free qubits together, so splitting the
  // path greedily into runs that fit gives a number of stages no staging
  // can beat.  One pass keeps a path per gate: the run count and the free
  // qubits of its last run, extended from the last gate on each of its
  // qubits (the most runs, then the fullest last run).
  int more_stages(const std::vector<int32_t>& rest, uint64_t* U_out, bool paths) const {
    uint64_t U = 0;
    for (int32_t i : rest) U |= g_[i].nimask;
    U &= ~low_;
    if (U_out) *U_out = U;
    const int slots = L_ - jlow_;
    int best = std::max(1, (std::popcount(U) + slots - 1) / slots);
    if (!paths) return best;
    struct Path {
      int runs = 0;
      uint64_t last = 0;  // free qubits of the last run
    };
    Path at_qubit[64];  // the path of the last gate seen on each qubit
    for (int32_t i : rest) {
      const Gate& x = g_[i];
      const uint64_t need = x.nimask & ~low_;
      Path p{1, need};
      for (uint64_t m = x.qmask; m; m &= m - 1) {
        const Path& a = at_qubit[std::countr_zero(m)];
        if (a.runs == 0) continue;
        const uint64_t u = a.last | need;
        const Path c = std::popcount(u) > slots ? Path{a.runs + 1, need} : Path{a.runs, u};
        if (c.runs > p.runs || (c.runs == p.runs && std::popcount(c.last) > std::popcount(p.last))) p = c;
      }
      for (uint64_t m = x.qmask; m; m &= m - 1) at_qubit[std::countr_zero(m)] = p;
      best = std::max(best, p.runs);
    }
    return best;
  }

  // A staging of `rest` in at most `limit - depth` more stages, appended to
  // cur_; remembers for each remaining set the allowance already proven
  // too small.
  bool shorter(const std::vector<int32_t>& rest, int depth, int limit) {
    if (rest.empty()) return true;
    if (out_) return false;
    const int allow = limit - depth;
    if (!spend(rest.size())) return false;  // the bounds' pass over the gates
    if (more_stages(rest, nullptr, true) > allow) return false;
    const Key k = key_of(rest, 0);
    auto it = too_few_.find(k);
    if (it != too_few_.end() && it->second >= allow) return false;
    if (!spend(kNodeCharge + (uint64_t)rest.size() * nsets())) return false;
    const auto ch = stage_choices(g_, rest, n_, L_, jlow_, low_, all_);
    std::unordered_map<Key, bool, KeyHash> tried;  // children with the same gates left
    for (const auto& [taken, S] : ch) {
      if (taken == 0 || out_) break;
      std::vector<int32_t> left;
      left.reserve(rest.size() - taken);
      if (!spend(rest.size())) return false;
      admitted(g_, rest, S, all_, nullptr, &left);
      if (!tried.emplace(key_of(left, 0), true).second) continue;
      cur_.push_back(S);
      if (shorter(left, depth + 1, limit)) return true;
      cur_.pop_back();
    }
    if (!out_) {
      int& v = too_few_[k];
      v = std::max(v, allow);
    }
    return false;
  }

  bool spend(uint64_t w) {
    budget_ -= (int64_t)w;
    if (budget_ < 0) out_ = true;
    return !out_;
  }

  // rest: gates left; last: the previous stage's local set; cost: the
  // objective of the stages so far
  void dfs(const std::vector<int32_t>& rest, uint64_t last, int depth, int cost) {
    if (out_) return;
    if (rest.empty()) {
      if (depth < best_s_ || (depth == best_s_ && cost < best_cost_)) {
        best_ = cur_;
        best_s_ = depth;
        best_cost_ = cost;
      }
      return;
    }
    uint64_t U = 0;
    const int more = more_stages(rest, &U, false);  // the count is settled by phase 1
    const int slots = L_ - jlow_;
    const int lb_cost = depth == 0 ? std::max(0, std::popcount(U) - slots) : cost + std::popcount(U & ~last);
    if (depth + more > best_s_ || (depth + more == best_s_ && lb_cost >= best_cost_)) return;
    const Key k = key_of(rest, last);
    auto it = seen_.find(k);
    if (it != seen_.end() && it->second.first <= depth && it->second.second <= cost) return;
    seen_[k] = {depth, cost};
    // a node's memo entry is charged too, which bounds the memo's size
    if (!spend(kNodeCharge + (uint64_t)rest.size() * nsets())) return;
    auto ch = stage_choices(g_, rest, n_, L_, jlow_, low_, all_);
    // most gates first, then the fewest new local qubits
    std::stable_sort(ch.begin(), ch.end(), [&](const auto& a, const auto& b) {
      if (a.first != b.first) return a.first > b.first;
      return depth > 0 && std::popcount(a.second & ~last) < std::popcount(b.second & ~last);
    });
    for (const auto& [taken, S] : ch) {
      if (taken == 0 || out_) break;
      std::vector<int32_t> left;
      left.reserve(rest.size() - taken);
      if (!spend(rest.size())) return;
      admitted(g_, rest, S, all_, nullptr, &left);
      cur_.push_back(S);
      dfs(left, S, depth + 1, cost + (depth > 0 ? std::popcount(S & ~last) : 0));
      cur_.pop_back();
    }
  }

  uint64_t nsets() const { return std::max<uint64_t>(1, binom(n_ - jlow_, n_ - L_)); }

  const std::vector<Gate>& g_;
  int n_, L_, jlow_;
  uint64_t low_, all_;
  int64_t budget_;
  bool out_ = false;
  std::vector<uint64_t> best_, cur_;
  int best_s_ = 0, best_cost_ = 0;
  std::unordered_map<Key, std::pair<int, int>, KeyHash> seen_;
  std::unordered_map<Key, int, KeyHash> too_few_;  // remaining gates -> stages proven too few
};

}  // namespace

int stage_circuit(const std::vector<Gate>& g, int n, int L, int stager, int64_t budget, std::vector<Stage>* out,
                  int* optimal) {
  out->clear();
  *optimal = 0;
  if (L < 2 || L > n) return QS_EINVAL;
  const int jlow = std::max(0, L - kStageSlots);
  const uint64_t all = n >= 64 ? ~0ull : (1ull << n) - 1;
  const uint64_t low = jlow ? (1ull << jlow) - 1 : 0;
  std::vector<int32_t> rest(g.size());
  std::iota(rest.begin(), rest.end(), 0);
  for (const Gate& x : g)
    if (std::popcount(low | x.nimask) > L) return QS_EPLAN;
  // the local sets of all stages, by a beam search over the greedy choices,
  // improved by the exact search when asked for and every set can be tried
  std::vector<uint64_t> plan = choose_local_sets(g, rest, n, L, jlow, low, all);
  if (stager == QS_STAGER_EXACT && !plan.empty() && binom(n - jlow, n - L) <= kMaxChoices) {
    ExactStager ex(g, n, L, jlow, low, all, budget > 0 ? budget : kDefaultStagerBudget);
    *optimal = ex.run(rest, &plan);
  }
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
