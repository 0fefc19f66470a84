// Circuit staging for chunked execution (Alg. 1's Stage, Sec. 4): splits the
// circuit into stages, each with a set of L local qubits that contains every
// non-insular qubit of the stage's gates (insular qubits may be regional:
// their value is fixed within a chunk, Definition 2).
//
// The stager is greedy over stages, in the spirit of the SnuQS baseline the
// paper compares against (Sec. 6): each stage takes as many gates as it can.
// With the frontier fixed, the regional qubits of the next stage are chosen
// among the freely placeable ones (all but the L - kStageSlots lowest) by
// trying every choice when there are at most kMaxChoices of them and keeping
// the one that admits the most gates; otherwise the local set grows in
// circuit order until the next gate no longer fits and the free slots go to
// the qubits the remaining gates need first.  Gates on disjoint qubits
// commute, so a stage takes every gate whose non-insular qubits are local
// and that shares no qubit with an earlier gate left for a later stage.
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
  while (!rest.empty()) {
    uint64_t S = 0;
    const int free_q = n - jlow, nreg = n - L;
    if (binom(free_q, nreg) <= kMaxChoices) {
      // every choice of the regional qubits among the free ones
      std::vector<int> pick(nreg);
      std::iota(pick.begin(), pick.end(), jlow);
      size_t best = 0;
      S = all;
      while (true) {
        uint64_t R = 0;
        for (int q : pick) R |= 1ull << q;
        const size_t c = admitted(g, rest, all & ~R, all, nullptr, nullptr);
        if (c > best || S == all) {
          best = c;
          S = all & ~R;
        }
        int t = nreg - 1;  // next combination in lexicographic order
        while (t >= 0 && pick[t] == n - nreg + t) --t;
        if (t < 0) break;
        pick[t]++;
        for (int u = t + 1; u < nreg; ++u) pick[u] = pick[u - 1] + 1;
      }
    } else {
      S = grow_in_order(g, rest, low, all, n, L);
    }
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
