// Kernelization planners and the analytic cost model.
//
//  * cost model  -- "Cost Function in Kernelize": a fusion kernel on k qubits
//    costs fuse_cost[k]; a shared-memory kernel costs alpha + sum Cost(g) and
//    its active set is its gates' non-insular qubits plus the forced low
//    qubits (footnote of that section, Appendix A.2 "Insular qubits").
//  * PER_GATE    -- one kernel per gate.
//  * GREEDY      -- contiguous greedy packing into kernels of at most
//    fuse_kmax qubits (the greedy baseline of Sec. 6.4).
//  * ORDERED     -- OrderedKernelize, Alg. 5: DP[i+1] = min_j DP[j] +
//    Cost(C[j..i]) over contiguous segments.
//  * KERNELIZE   -- Alg. 3 with Alg. 4 (kernelize.cpp).
#include <algorithm>
#include <cstdlib>
#include <bit>
#include <chrono>
#include <cmath>
#include <limits>

#include "internal.hpp"

namespace qs {

static constexpr double INF = std::numeric_limits<double>::infinity();

static inline int popc(uint64_t x) { return std::popcount(x); }

static uint64_t low_mask(int k, int n) {
  int b = std::min(k, n);
  return b <= 0 ? 0ull : (b >= 64 ? ~0ull : ((1ull << b) - 1));
}

double CostModel::fusion(const KStat& s) const {
  const auto& o = plan->opts;
  int k = popc(s.q);
  if (o.fuse_kmax <= 0 || k > o.fuse_kmax) return INF;
  if (s.q & ~plan->exec_limit) return INF;
  if (learned) return learned_cost(learned, s, true);
  int ke = std::max(k, std::min(o.fuse_kmin, plan->n));  // widened to fuse_kmin
  return plan->cost.fuse_cost[ke];
}

double CostModel::shm(const KStat& s) const {
  const auto& o = plan->opts;
  uint64_t a = s.ni | low_mask(o.forced_low, plan->n);
  if (popc(a) > o.shm_max_active || (a & ~plan->exec_limit)) return INF;
  if (learned) return learned_cost(learned, s, false);
  return plan->cost.alpha + s.gcost;
}

void CostModel::prefetch(const std::vector<std::pair<KStat, bool>>& ks) const {
  if (learned) learned_prefetch(learned, ks);
}

static KStat stat_of(const PlanImpl* p, const std::vector<int32_t>& gates) {
  KStat s;
  for (int g : gates) s.add(p->gates[g], p->cost.gate_cost[p->gates[g].type]);
  return s;
}

// Chooses the cheaper feasible type for a finished kernel (ties: shm).
static bool finish_kernel(const PlanImpl* p, Kernel* k) {
  CostModel cm{p, p->learned};
  const KStat s = stat_of(p, k->gates);
  double cf = cm.fusion(s), cs = cm.shm(s);
  if (cf == INF && cs == INF) return false;
  if (cs <= cf) {
    k->type = QS_KERNEL_SHM;
    k->mask = s.ni | low_mask(p->opts.forced_low, p->n);
    k->cost = cs;
  } else {
    k->type = QS_KERNEL_FUSED;
    k->mask = s.q;
    k->cost = cf;
  }
  return true;
}

static int plan_per_gate(PlanImpl* p) {
  for (size_t i = 0; i < p->gates.size(); ++i) {
    Kernel k;
    k.gates.push_back((int32_t)i);
    if (!finish_kernel(p, &k)) return QS_EPLAN;
    p->kernels.push_back(std::move(k));
  }
  return QS_OK;
}

static int plan_greedy(PlanImpl* p) {
  const bool fuse = p->opts.fuse_kmax > 0;
  const int lim = fuse ? p->opts.fuse_kmax : p->opts.shm_max_active;
  const uint64_t low = fuse ? 0 : low_mask(p->opts.forced_low, p->n);
  // a kernel grows while it still fits: at most `lim` qubits, all of them
  // ones a kernel may execute on (a stage's local positions)
  auto fits = [&](uint64_t m) { return popc(m) <= lim && !(m & ~p->exec_limit); };
  Kernel cur;
  uint64_t cm = low;
  for (size_t i = 0; i < p->gates.size(); ++i) {
    const Gate& g = p->gates[i];
    uint64_t gm = fuse ? g.qmask : g.nimask;
    if (!cur.gates.empty() && !fits(cm | gm)) {
      if (!finish_kernel(p, &cur)) return QS_EPLAN;
      p->kernels.push_back(std::move(cur));
      cur = Kernel();
      cm = low;
    }
    cur.gates.push_back((int32_t)i);
    cm |= gm;
  }
  if (!cur.gates.empty()) {
    if (!finish_kernel(p, &cur)) return QS_EPLAN;
    p->kernels.push_back(std::move(cur));
  }
  return QS_OK;
}

static int plan_ordered(PlanImpl* p) {
  const size_t L = p->gates.size();
  CostModel cm{p, p->learned};
  std::vector<double> dp(L + 1, INF);
  std::vector<int64_t> from(L + 1, -1);
  dp[0] = 0;
  const uint64_t low = low_mask(p->opts.forced_low, p->n);
  std::vector<std::pair<KStat, bool>> want;
  for (size_t i = 0; i < L; ++i) {
    if (cm.learned) {  // batch every segment ending at i
      want.clear();
      KStat s;
      for (int64_t j = (int64_t)i; j >= 0; --j) {
        s.add(p->gates[j], 0.0);
        const bool fok = p->opts.fuse_kmax > 0 && popc(s.q) <= p->opts.fuse_kmax &&
                         !(s.q & ~p->exec_limit);
        const bool sok = popc(s.ni | low) <= p->opts.shm_max_active && !((s.ni | low) & ~p->exec_limit);
        if (!fok && !sok) break;
        if (fok) want.push_back({s, true});
        if (sok) want.push_back({s, false});
      }
      cm.prefetch(want);
    }
    KStat s;
    for (int64_t j = (int64_t)i; j >= 0; --j) {
      const Gate& g = p->gates[j];
      s.add(g, cm.gate_cost(g.type));
      double c = std::min(cm.fusion(s), cm.shm(s));
      if (c == INF) break;  // feasibility only shrinks as the segment grows
      double cand = dp[j] + c;
      if (cand < dp[i + 1]) {
        dp[i + 1] = cand;
        from[i + 1] = j;
      }
    }
    if (dp[i + 1] == INF) return QS_EPLAN;
  }
  std::vector<Kernel> rev;
  for (int64_t e = (int64_t)L; e > 0; e = from[e]) {
    Kernel k;
    for (int64_t g = from[e]; g < e; ++g) k.gates.push_back((int32_t)g);
    if (!finish_kernel(p, &k)) return QS_EPLAN;
    rev.push_back(std::move(k));
  }
  p->kernels.assign(std::make_move_iterator(rev.rbegin()), std::make_move_iterator(rev.rend()));
  return QS_OK;
}

int plan_kernelize(PlanImpl* p);  // kernelize.cpp

int plan_kernels(PlanImpl* p) {
  p->kernels.clear();
  if (p->gates.empty()) return QS_OK;
  if (p->opts.cost_kind == QS_COST_LEARNED) {
    int st = QS_OK;
    p->learned = learned_create(p, const_cast<qs_mlp*>(p->opts.mlp), &st);
    if (!p->learned) return st;
  }
  int rc;
  switch (p->opts.algo) {
    case QS_ALGO_PER_GATE: rc = plan_per_gate(p); break;
    case QS_ALGO_GREEDY: rc = plan_greedy(p); break;
    case QS_ALGO_ORDERED: rc = plan_ordered(p); break;
    case QS_ALGO_KERNELIZE: rc = plan_kernelize(p); break;
    default: rc = QS_EINVAL; break;
  }
  if (rc == QS_OK) rc = learned_status(p->learned);  // a failed inference call
  learned_destroy(p->learned);
  p->learned = nullptr;
  if (rc != QS_OK) return rc;
  p->total_cost = 0;
  for (auto& k : p->kernels) p->total_cost += k.cost;
  return QS_OK;
}

// Theorem 2: the concatenated kernels are topologically equivalent to C.
int validate_plan(const PlanImpl* p) {
  const size_t L = p->gates.size();
  std::vector<int64_t> pos(L, -1);
  int64_t at = 0;
  for (const auto& k : p->kernels)
    for (int g : k.gates) {
      if (g < 0 || (size_t)g >= L || pos[g] >= 0) return QS_EPLAN;
      pos[g] = at++;
    }
  if ((size_t)at != L) return QS_EPLAN;
  // per qubit: a gate non-insular on q follows every earlier gate on q; a
  // gate insular on q follows every earlier gate that is non-insular on q.
  std::vector<int64_t> max_any(p->n, -1), max_ni(p->n, -1);
  for (size_t j = 0; j < L; ++j) {
    const Gate& g = p->gates[j];
    for (int s = 0; s < g.nq; ++s) {
      int q = s == 0 ? g.q0 : g.q1;
      bool ni = (g.nimask >> q) & 1;
      int64_t need = ni ? max_any[q] : max_ni[q];
      if (pos[j] <= need) return QS_EPLAN;
    }
    for (int s = 0; s < g.nq; ++s) {
      int q = s == 0 ? g.q0 : g.q1;
      max_any[q] = std::max(max_any[q], pos[j]);
      if ((g.nimask >> q) & 1) max_ni[q] = std::max(max_ni[q], pos[j]);
    }
  }
  return QS_OK;
}

// ---- program compilation ------------------------------------------------------

// Applies a gate (given on local matrix bits a, b) to every column of the
// 2^k x 2^k matrix u (complex interleaved): u <- G u.
static void left_multiply(double* u, int k, const Gate& g, int a, int b) {
  double m[32];
  gate_matrix(g, m);
  const int dim = 1 << k;
  if (g.nq == 1) {
    for (int r = 0; r < dim; ++r) {
      if ((r >> a) & 1) continue;
      int r1 = r | (1 << a);
      for (int c = 0; c < dim; ++c) {
        double* x = &u[2 * (r * dim + c)];
        double* y = &u[2 * (r1 * dim + c)];
        double xr = x[0], xi = x[1], yr = y[0], yi = y[1];
        x[0] = m[0] * xr - m[1] * xi + m[2] * yr - m[3] * yi;
        x[1] = m[0] * xi + m[1] * xr + m[2] * yi + m[3] * yr;
        y[0] = m[4] * xr - m[5] * xi + m[6] * yr - m[7] * yi;
        y[1] = m[4] * xi + m[5] * xr + m[6] * yi + m[7] * yr;
      }
    }
  } else {
    for (int r = 0; r < dim; ++r) {
      if (((r >> a) & 1) || ((r >> b) & 1)) continue;
      int rows[4];
      for (int s = 0; s < 4; ++s) rows[s] = r | ((s & 1) << a) | ((s >> 1) << b);
      for (int c = 0; c < dim; ++c) {
        double vr[4], vi[4];
        for (int s = 0; s < 4; ++s) {
          vr[s] = u[2 * (rows[s] * dim + c)];
          vi[s] = u[2 * (rows[s] * dim + c) + 1];
        }
        for (int s = 0; s < 4; ++s) {
          double sr = 0, si = 0;
          for (int t = 0; t < 4; ++t) {
            double mr = m[2 * (4 * s + t)], mi = m[2 * (4 * s + t) + 1];
            sr += mr * vr[t] - mi * vi[t];
            si += mr * vi[t] + mi * vr[t];
          }
          u[2 * (rows[s] * dim + c)] = sr;
          u[2 * (rows[s] * dim + c) + 1] = si;
        }
      }
    }
  }
}

static void compile_fused(const PlanImpl* p, const Kernel& K, FusedProgram* fp) {
  int k = 0;
  int loc[kMaxQubits];
  for (int q = 0; q < p->n; ++q) {
    loc[q] = -1;
    if ((K.mask >> q) & 1) {
      fp->targets[k] = q;
      loc[q] = k++;
    }
  }
  fp->k = k;
  const int dim = 1 << k;
  fp->u64.assign(2 * dim * dim, 0.0);
  for (int r = 0; r < dim; ++r) fp->u64[2 * (r * dim + r)] = 1.0;
  for (int gi : K.gates) {
    const Gate& g = p->gates[gi];
    left_multiply(fp->u64.data(), k, g, loc[g.q0], g.nq == 2 ? loc[g.q1] : -1);
  }
  fp->u.resize(fp->u64.size());
  for (size_t i = 0; i < fp->u64.size(); ++i) fp->u[i] = (float)fp->u64[i];
}

// Every op's bit indices must address the tile: dense targets in [0, m),
// diagonal qubits either in [0, m) or a physical bit in [0, n).
static bool op_in_bounds(const DevOp& op, int m, int n) {
  auto loc_ok = [m](int t) { return t >= 0 && t < m; };
  if (op.kind == OP_DENSE1) return loc_ok(op.t0) && (op.cloc >> m) == 0;
  if (op.kind == OP_DENSE2) return loc_ok(op.t0) && loc_ok(op.t1) && op.t0 != op.t1;
  if (op.kind == OP_DIAG) {
    bool q0 = loc_ok(op.t0) != (op.g0 >= 0 && op.g0 < n);
    bool q1 = (op.t1 == -1 && op.g1 == -1) || (loc_ok(op.t1) != (op.g1 >= 0 && op.g1 < n));
    return q0 && q1;
  }
  return false;
}

static bool compile_shm(const PlanImpl* p, const Kernel& K, ShmProgram* sp) {
  int loc[kMaxQubits];
  int m = 0;
  for (int q = 0; q < p->n; ++q) {
    loc[q] = -1;
    if ((K.mask >> q) & 1) {
      sp->act[m] = q;
      loc[q] = m++;
    }
  }
  sp->m = m;
  sp->ops.clear();
  for (int gi : K.gates) {
    const Gate& g = p->gates[gi];
    double gm[32];
    gate_matrix(g, gm);
    DevOp op;
    std::memset(&op, 0, sizeof(op));
    op.t0 = op.t1 = op.g0 = op.g1 = -1;
    if (gate_is_diagonal(g.type)) {
      op.kind = OP_DIAG;
      const int dim = 1 << g.nq;
      for (int b = 0; b < 4; ++b) {
        int src = b < dim ? b : 0;  // 1-qubit diag: qubit 1 absent, reads as 0
        op.m[2 * b] = (float)gm[2 * (src * dim + src)];
        op.m[2 * b + 1] = (float)gm[2 * (src * dim + src) + 1];
      }
      if (loc[g.q0] >= 0) op.t0 = (int8_t)loc[g.q0]; else op.g0 = (int8_t)g.q0;
      if (g.nq == 2) {
        if (loc[g.q1] >= 0) op.t1 = (int8_t)loc[g.q1]; else op.g1 = (int8_t)g.q1;
      }
    } else if (g.type == QS_CX) {
      op.kind = OP_DENSE1;
      op.t0 = (int8_t)loc[g.q1];
      if (loc[g.q0] >= 0) op.cloc = 1u << loc[g.q0]; else op.cglob = 1ull << g.q0;
      op.m[2] = 1.0f;  // X: [[0,1],[1,0]]
      op.m[4] = 1.0f;
    } else if (g.nq == 1) {
      op.kind = OP_DENSE1;
      op.t0 = (int8_t)loc[g.q0];
      for (int i = 0; i < 8; ++i) op.m[i] = (float)gm[i];
    } else {
      op.kind = OP_DENSE2;
      op.t0 = (int8_t)loc[g.q0];
      op.t1 = (int8_t)loc[g.q1];
      for (int i = 0; i < 32; ++i) op.m[i] = (float)gm[i];
    }
    if (!op_in_bounds(op, m, p->n)) return false;
    sp->ops.push_back(op);
  }
  return true;
}

// Widens a kernel's qubit set with the lowest unused qubits up to `want`
// qubits (shared-memory tiles of at least 2^10 amplitudes for coalescing and
// occupancy; fused kernels up to their minimum width).  Extra qubits do not
// change the result.
uint64_t widen_mask(uint64_t mask, int n, int want) {
  for (int q = 0; q < n && std::popcount(mask) < want; ++q) mask |= 1ull << q;
  return mask;
}

// Lowest qubits added to the tile of a compute-heavy shared-memory kernel
// (its gates cost more than a pass over the state in the analytic table),
// while the tile stays within kTileCap qubits.  Measured at 30 qubits: the
// 40-layer entangling circuit's kernels 7.10 -> 6.49 ms per launch with
// qubits 0..5 in every tile; on the mixed circuit, whose kernels are
// memory-bound, wider tiles were 1-3 % slower.  QSIM_TILE_LOW overrides the
// count (0 turns it off).
static int tile_low_qubits() {
  const char* e = std::getenv("QSIM_TILE_LOW");
  if (e && *e >= '0' && *e <= '9') return std::min(8, std::atoi(e));
  return 6;
}
constexpr int kTileCap = 13;

static bool compute_heavy(const PlanImpl* p, const Kernel& k) {
  double g = 0;
  for (int32_t i : k.gates) g += p->cost.gate_cost[p->gates[i].type];
  return g > p->cost.alpha;
}

int compile_programs(PlanImpl* p) {
  const int tile_low = tile_low_qubits();
  const size_t K = p->kernels.size();
  p->shm.assign(K, ShmProgram());
  p->fused.assign(K, FusedProgram());
  p->shm2.assign(K, ShmProgramV2());
  for (size_t i = 0; i < K; ++i) {
    Kernel& k = p->kernels[i];
    if (k.type == QS_KERNEL_SHM) {
      int want = std::min(p->n, std::max(std::min(10, kMaxShmActive), std::popcount(k.mask)));
      k.mask = widen_mask(k.mask, p->n, want);
      for (int q = 0; q < std::min(compute_heavy(p, k) ? tile_low : 0, p->n); ++q)
        if (!((k.mask >> q) & 1) && std::popcount(k.mask) < kTileCap && ((p->exec_limit >> q) & 1))
          k.mask |= 1ull << q;
      if (std::popcount(k.mask) > kMaxShmActive) return QS_EPLAN;
      if (!compile_shm(p, k, &p->shm[i])) return QS_EPLAN;
      if (p->opts.shm_variant != 1 && p->shm[i].m >= kMinPhasedM)
        compile_shm_v2(p, k, p->shm[i], &p->shm2[i]);
      if (p->opts.shm_variant >= 2 && !p->shm2[i].ok) return QS_EUNSUPPORTED;
    } else {
      const bool tc = p->opts.precision != QS_PREC_FP32;
      int kmin = tc ? std::max(p->opts.fuse_kmin, kTcTargets) : p->opts.fuse_kmin;
      int want = std::min(p->n, std::max(kmin, std::popcount(k.mask)));
      k.mask = widen_mask(k.mask, p->n, want);
      if (std::popcount(k.mask) > kMaxFuse) return QS_EPLAN;
      compile_fused(p, k, &p->fused[i]);
      if (tc) {
        if (p->fused[i].k != kTcTargets) return QS_EUNSUPPORTED;
        tc_prepare_weights(p->fused[i].u.data(), p->opts.precision == QS_PREC_TF32X3,
                           &p->fused[i].w_tc);
      }
    }
  }
  fold_global_phase(p->shm2);
  if (p->opts.shm_variant == 0 || p->opts.shm_variant == 3) {
    auto t0 = std::chrono::steady_clock::now();
    int rc = jit_compile_plan(p);
    p->jit_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (rc != QS_OK) return rc;
    if (p->opts.shm_variant == 3)
      for (const auto& pg : p->shm2)
        if (pg.ok && pg.jit_module < 0) return QS_EUNSUPPORTED;
  }
  return QS_OK;
}

}  // namespace qs
