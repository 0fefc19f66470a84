// C ABI of libqsim (include/qsim.h): plans, states, execution (Alg. 1's
// Partition / Execute on one GPU).
#include <algorithm>
#include <bit>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <new>

#include "internal.hpp"

namespace qs {

static thread_local std::string g_last_cuda;
static thread_local std::string g_last_error;  // why the last planning call failed

void set_cuda_error(const char* what, cudaError_t e) {
  g_last_cuda = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
}

int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return QS_OK;
  set_cuda_error("cuda", e);
  return e == cudaErrorMemoryAllocation ? QS_ENOMEM : QS_ECUDA;
}

void widen_unitary(const float* u, int k, int kw, float* out) {
  const int dk = 1 << k, dw = 1 << kw;
  for (int r = 0; r < dw; ++r)
    for (int c = 0; c < dw; ++c) {
      float re = 0.0f, im = 0.0f;
      if ((r >> k) == (c >> k)) {
        re = u[2 * ((r & (dk - 1)) * dk + (c & (dk - 1)))];
        im = u[2 * ((r & (dk - 1)) * dk + (c & (dk - 1))) + 1];
      }
      out[2 * (r * dw + c)] = re;
      out[2 * (r * dw + c) + 1] = im;
    }
}

// targets[k .. kw-1] := the lowest qubits below n not among targets[0 .. k-1]
void widen_targets(int n, int k, int kw, int* targets) {
  uint64_t seen = 0;
  for (int j = 0; j < k; ++j) seen |= 1ull << targets[j];
  for (int q = 0, j = k; q < n && j < kw; ++q)
    if (!((seen >> q) & 1)) {
      targets[j++] = q;
      seen |= 1ull << q;
    }
}

// Uploads every kernel program of the plan to the current device (once per
// device; later calls reuse it).
static int ensure_device(PlanImpl* p, DeviceCache** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_status(e);
  std::lock_guard<std::mutex> lk(p->mu);
  for (auto& d : p->dev)
    if (d.device == dev) {
      *out = &d;
      return QS_OK;
    }
  DeviceCache dc;
  dc.device = dev;
  std::vector<uint8_t> host;
  for (size_t i = 0; i < p->kernels.size(); ++i) {
    uint64_t off = (host.size() + 255) & ~uint64_t(255);
    host.resize(off);
    dc.op_off.push_back(off);
    if (p->kernels[i].type == QS_KERNEL_SHM) {
      const auto& ops = p->shm[i].ops;
      host.resize(off + ops.size() * sizeof(DevOp));
      if (!ops.empty()) std::memcpy(host.data() + off, ops.data(), ops.size() * sizeof(DevOp));
      const auto& pw = p->shm2[i].prog;
      uint64_t poff = (host.size() + 255) & ~uint64_t(255);
      host.resize(poff + pw.size() * sizeof(uint32_t));
      if (!pw.empty()) std::memcpy(host.data() + poff, pw.data(), pw.size() * sizeof(uint32_t));
      dc.prog_off.push_back(poff);
    } else {
      dc.prog_off.push_back(0);
      // tensor-core precisions read the prepared weights, FP32 the matrix
      const bool tc = p->opts.precision != QS_PREC_FP32;
      const auto& u = tc ? p->fused[i].w_tc : p->fused[i].u;
      const size_t need = tc ? size_t(p->opts.precision == QS_PREC_TF32X3 ? 2 : 1) * 128 * 128
                             : size_t(2) << (2 * p->fused[i].k);
      if (u.size() != need) return QS_EPLAN;  // never hand a kernel a short buffer
      host.resize(off + u.size() * sizeof(float));
      std::memcpy(host.data() + off, u.data(), u.size() * sizeof(float));
    }
  }
  // specialised kernels: load the JIT modules and look up each kernel
  dc.jit_kernel.assign(p->kernels.size(), nullptr);
  dc.jit_blocks.assign(p->kernels.size(), 1);
  for (size_t k = 0; k < p->jit_modules.size(); ++k) {
    cudaLibrary_t lib = nullptr;
    if (!p->jit_modules[k].empty()) {
      e = cudaLibraryLoadData(&lib, p->jit_modules[k].data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
      if (e != cudaSuccess) {
        for (auto l : dc.libs)
          if (l) cudaLibraryUnload(l);
        return cuda_status(e);
      }
    }
    dc.libs.push_back(lib);
  }
  for (size_t i = 0; i < p->kernels.size(); ++i) {
    const int mod = (i < p->shm2.size() && p->shm2[i].ok) ? p->shm2[i].jit_module : -1;
    if (mod < 0 || !dc.libs[mod]) continue;
    std::string name = "qsk" + std::to_string(i);
    cudaKernel_t kf = nullptr;
    e = cudaLibraryGetKernel(&kf, dc.libs[mod], name.c_str());
    if (e != cudaSuccess) {
      for (auto l : dc.libs)
        if (l) cudaLibraryUnload(l);
      return cuda_status(e);
    }
    const int smem = p->shm2[i].jit_smem;
    e = cudaKernelSetAttributeForDevice(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, smem, dev);
    int blocks = 0;
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, (const void*)kf, 1 << (p->shm2[i].m - kRegBits),
                                                         (size_t)smem);
    if (e == cudaSuccess && blocks < 1) e = cudaErrorInvalidConfiguration;  // cannot be resident
    if (e != cudaSuccess) {
      for (auto l : dc.libs)
        if (l) cudaLibraryUnload(l);
      return cuda_status(e);
    }
    dc.jit_kernel[i] = kf;
    dc.jit_blocks[i] = blocks;
  }
  if (host.empty()) host.resize(256);
  e = cudaMalloc(&dc.buf, host.size());
  if (e != cudaSuccess) dc.buf = nullptr;
  else e = cudaMemcpy(dc.buf, host.data(), host.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    if (dc.buf) cudaFree(dc.buf);
    for (auto l : dc.libs)
      if (l) cudaLibraryUnload(l);
    return cuda_status(e);
  }
  p->dev.push_back(std::move(dc));
  *out = &p->dev.back();
  return QS_OK;
}

}  // namespace qs

using namespace qs;

extern "C" {

const char* qs_strerror(int s) {
  switch (s) {
    case QS_OK: return "ok";
    case QS_EINVAL: return "invalid argument";
    case QS_ENOMEM: return "out of memory";
    case QS_EUNSUPPORTED: return "unsupported";
    case QS_ETIMEDOUT: return "timed out";
    case QS_ECUDA: return "CUDA error";
    case QS_EPLAN: return "planning failed or invalid plan";
    default: return "unknown status";
  }
}

const char* qs_last_cuda_error(void) { return g_last_cuda.c_str(); }
const char* qs_last_error(void) { return g_last_error.c_str(); }

void qs_cost_table_default(qs_cost_table* t) {
  if (!t) return;
  std::memset(t, 0, sizeof(*t));
  // Microseconds per kernel on a 30-qubit state (GB300): alpha = one
  // read+write pass of 16 GiB at HBM speed; per-gate costs and fused costs
  // from the calibration runs of the timing generator.
  t->alpha = 2600.0;
  const double dense1 = 60.0, diag = 40.0, dense2 = 120.0;
  t->gate_cost[QS_H] = dense1;
  t->gate_cost[QS_X] = dense1;
  t->gate_cost[QS_RX] = dense1;
  t->gate_cost[QS_U3] = dense1;
  t->gate_cost[QS_RZ] = diag;
  t->gate_cost[QS_CZ] = diag;
  t->gate_cost[QS_CP] = diag;
  t->gate_cost[QS_CX] = dense1;
  t->gate_cost[QS_SWAP] = dense2;
  t->gate_cost[QS_RXX] = dense2;
  const double fuse[16] = {0, 2700, 2700, 2700, 2800, 3200, 5200, 10400,
                           20800, 41600, 83200, 166400, 332800, 665600, 1331200, 2662400};
  std::memcpy(t->fuse_cost, fuse, sizeof(fuse));
}

void qs_plan_opts_default(qs_plan_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->algo = QS_ALGO_KERNELIZE;
  o->cost_kind = QS_COST_ANALYTIC;
  o->precision = QS_PREC_FP32;
  o->shm_max_active = 13;
  o->forced_low = 4;
  o->fuse_kmin = 1;
  o->fuse_kmax = 6;
  o->prune_T = 500;
  o->attach_single = 1;
  o->local_qubits = 0;
  o->shm_variant = 0;
  o->cost = nullptr;
  o->mlp = nullptr;
  o->stager_budget = 0;
  o->stager = QS_STAGER_BEAM;
  o->insular_x = 0;
}

}  // extern "C"

namespace qs {

// Plans `count` gates (given by index into `gates`, relabelled through `pos`
// when it is set) into P: Kernelize/Ordered, program compilation, Theorem 2
// check.
static int build_impl(PlanImpl& P, int n, const qs_gate* gates, const int32_t* ids,
                      const int32_t* pos, uint64_t count) {
  P.gates.resize(count);
  for (uint64_t i = 0; i < count; ++i) {
    qs_gate x = gates[ids ? ids[i] : i];
    if (pos) {
      if (x.q[0] < 0 || x.q[0] >= n || (x.nq == 2 && (x.q[1] < 0 || x.q[1] >= n))) return QS_EINVAL;
      x.q[0] = pos[x.q[0]];
      if (x.nq == 2) x.q[1] = pos[x.q[1]];
    }
    int rc = make_gate(x, n, &P.gates[i]);
    if (rc != QS_OK) return rc;
  }
  int rc = plan_kernels(&P);
  if (rc == QS_OK) rc = compile_programs(&P);
  if (rc == QS_OK) rc = validate_plan(&P);
  return rc;
}

// Staged plan: stage the circuit, plan every stage on its relabelled qubits
// and flatten the kernels (logical qubits, circuit gate indices) into p->impl.
static int build_staged(qs_plan* p, const qs_gate* gates, const qs_plan_opts& o) {
  PlanImpl& P = p->impl;
  const int n = P.n, L = o.local_qubits;
  // with insular_x the stager sees X as insular (anti-diagonal, Definition 2)
  std::vector<Gate> sg = P.gates;
  const bool relabel = (o.insular_x & QS_INSULAR_X_STAGED) != 0;
  if (relabel)
    for (Gate& x : sg)
      if (x.type == QS_X) x.nimask = 0;
  int rc = stage_circuit(sg, n, L, o.stager, o.stager_budget, &p->stages, &p->staging_optimal);
  if (rc != QS_OK) return rc;
  double phase = 0;  // global phase of the conjugated gates (radians)
  for (size_t si = 0; si < p->stages.size(); ++si) {
    Stage& st = p->stages[si];
    // the stage's gates on the stored state: an X on a regional qubit flips
    // the frame f (the stored chunks are the logical ones relabelled by f);
    // a later gate is conjugated by X^f (App. A.2's control flip)
    std::vector<qs_gate> sgates;
    st.src.clear();
    st.flips.clear();
    uint64_t f = 0;
    for (int32_t i : st.gates) {
      const qs_gate& x = gates[i];
      if (relabel && x.type == QS_X && !((st.local >> x.q[0]) & 1)) {
        f ^= 1ull << x.q[0];
        st.flips.push_back(i);
        continue;
      }
      const size_t first = sgates.size();
      if (!conjugate_by_x(x, f, &sgates, &phase)) return QS_EPLAN;  // f is regional: insular qubits only
      for (size_t j = first; j < sgates.size(); ++j) st.src.push_back(j == first ? i : -1);
    }
    st.frame = f;
    const double two_pi = 6.283185307179586;
    phase = std::fmod(phase, two_pi);
    if (si + 1 == p->stages.size() && std::fabs(phase) > 1e-15 && std::fabs(std::fabs(phase) - two_pi) > 1e-15) {
      // e^{i a} = P(a) X P(a) X on a local qubit, P(a) = U3(0, 0, a) exactly
      const int q = st.order[0];
      qs_gate pg{}, xg{};
      pg.type = QS_U3;
      pg.nq = 1;
      pg.q[0] = q;
      pg.q[1] = -1;
      pg.p[2] = phase;
      xg.type = QS_X;
      xg.nq = 1;
      xg.q[0] = q;
      xg.q[1] = -1;
      for (const qs_gate& y : {pg, xg, pg, xg}) {
        sgates.push_back(y);
        st.src.push_back(-1);
      }
    }
    st.plan = std::make_unique<PlanImpl>();
    PlanImpl& S = *st.plan;
    S.n = n;
    S.opts = o;
    S.opts.local_qubits = 0;
    S.cost = P.cost;
    S.exec_limit = (1ull << L) - 1;
    rc = build_impl(S, n, sgates.data(), nullptr, st.pos.data(), sgates.size());
    if (rc != QS_OK) return rc;
    for (size_t k = 0; k < S.kernels.size(); ++k) {
      Kernel K = S.kernels[k];
      K.stage = (int32_t)si;
      std::vector<int32_t> ids;  // circuit indices of the kernel's gates
      for (int32_t g : K.gates)
        if (st.src[g] >= 0) ids.push_back(st.src[g]);
      K.gates.swap(ids);
      uint64_t m = 0;
      for (int b = 0; b < n; ++b)
        if ((K.mask >> b) & 1) m |= 1ull << st.order[b];
      K.mask = m;
      P.kernels.push_back(std::move(K));
      p->kmap.push_back({(int32_t)si, (int32_t)k});
    }
    P.total_cost += S.total_cost;
    P.dp_states += S.dp_states;
    P.jit_ms += S.jit_ms;
  }
  return QS_OK;
}

// A staged plan's own invariants on top of Theorem 2 over the flattened
// kernel list: each gate's non-insular qubits and each kernel's qubits are
// local in its stage, and the stage's programs are those of its gates.
static int validate_staged(const qs_plan* p) {
  const PlanImpl& P = p->impl;
  int rc;
  if (!(P.opts.insular_x & QS_INSULAR_X_STAGED)) {
    rc = validate_plan(&P);
  } else {
    // Theorem 2 with X insular (Definition 2): the X gates a stage executes
    // as relabellings count as placed at the start of their stage, and
    // gates that pass an X on an insular qubit are its conjugates
    PlanImpl V;
    V.n = P.n;
    V.gates = P.gates;
    for (Gate& x : V.gates)
      if (x.type == QS_X) x.nimask = 0;
    size_t k = 0;
    for (size_t si = 0; si < p->stages.size(); ++si) {
      const Stage& st = p->stages[si];
      if (st.frame & st.local) return QS_EPLAN;
      uint64_t f = 0;
      for (int32_t i : st.flips) {
        if (i < 0 || (size_t)i >= P.gates.size() || P.gates[i].type != QS_X) return QS_EPLAN;
        if ((st.local >> P.gates[i].q0) & 1) return QS_EPLAN;
        f ^= 1ull << P.gates[i].q0;
      }
      if (f != st.frame) return QS_EPLAN;
      if (!st.flips.empty()) {
        Kernel F;
        F.gates = st.flips;
        V.kernels.push_back(std::move(F));
      }
      for (; k < P.kernels.size() && P.kernels[k].stage == (int32_t)si; ++k) V.kernels.push_back(P.kernels[k]);
    }
    if (k != P.kernels.size()) return QS_EPLAN;
    rc = validate_plan(&V);
  }
  if (rc != QS_OK) return rc;
  if (P.kernels.size() != p->kmap.size()) return QS_EPLAN;
  int32_t last = 0;
  for (size_t k = 0; k < P.kernels.size(); ++k) {
    const Kernel& K = P.kernels[k];
    const int32_t si = p->kmap[k].first;
    if (si < last || si >= (int32_t)p->stages.size() || K.stage != si) return QS_EPLAN;
    last = si;
    const Stage& st = p->stages[si];
    if (K.mask & ~st.local) return QS_EPLAN;
    for (int32_t g : K.gates)
      if (P.gates[g].nimask & ~st.local) return QS_EPLAN;
  }
  for (const Stage& st : p->stages)
    if (std::popcount(st.local) != P.opts.local_qubits || !st.plan || validate_plan(st.plan.get()) != QS_OK)
      return QS_EPLAN;
  return QS_OK;
}

static void free_device(PlanImpl& P) {
  for (auto& d : P.dev) {
    cudaSetDevice(d.device);
    if (d.buf) cudaFree(d.buf);
    for (auto l : d.libs)
      if (l) cudaLibraryUnload(l);
  }
  P.dev.clear();
}

}  // namespace qs

extern "C" {

static int plan_circuit_impl(int32_t n, const qs_gate* gates, uint64_t ngates, const qs_plan_opts* opts,
                             qs_plan** out);

// Why planning failed, for the caller: the first gate that fits no kernel
// on its own under the options' limits, else the limits that block a plan.
static std::string plan_failure(int rc, int32_t n, const qs_gate* gates, uint64_t ngates, const qs_plan_opts& o) {
  static const char* names[QS_NUM_GATE_TYPES] = {"H", "X", "RX", "RZ", "U3", "CX", "CZ", "CP", "SWAP", "RXX"};
  char buf[256];
  if (rc == QS_EPLAN) {
    const uint64_t low = o.forced_low <= 0 ? 0ull : ((1ull << std::min(o.forced_low, (int)n)) - 1);
    for (uint64_t i = 0; i < ngates; ++i) {
      Gate g;
      if (make_gate(gates[i], n, &g) != QS_OK) continue;
      const int a = std::popcount(g.nimask | low), k = std::popcount(g.qmask);
      if (a > o.shm_max_active && (o.fuse_kmax == 0 || k > o.fuse_kmax)) {
        std::snprintf(buf, sizeof buf,
                      "gate %llu (%s) fits no kernel: shared-memory needs %d active qubits > shm_max_active %d, "
                      "fused needs %d > fuse_kmax %d",
                      (unsigned long long)i, names[g.type], a, o.shm_max_active, k, o.fuse_kmax);
        return buf;
      }
    }
    return "no kernelization fits the options' limits (|A|, fused width, a stage's local qubits)";
  }
  if (rc == QS_EUNSUPPORTED) {
    if (o.precision != QS_PREC_FP32 && o.fuse_kmax > 0 && (o.fuse_kmax > kTcTargets || n < kTcTargets + 5))
      return "tensor-core precisions need n >= 11 and fuse_kmax <= 6";
    if (o.shm_variant >= 2)
      return "the forced shm_variant cannot serve every shared-memory kernel of this plan";
  }
  if (rc == QS_ENOMEM && o.prune_T <= 0) return "the unpruned Kernelize frontier passed 2^20 states";
  return "";
}

int qs_plan_circuit(int32_t n, const qs_gate* gates, uint64_t ngates, const qs_plan_opts* opts,
                    qs_plan** out) {
  g_last_error.clear();
  const int rc = plan_circuit_impl(n, gates, ngates, opts, out);
  if (rc != QS_OK && rc != QS_EINVAL) {
    qs_plan_opts o;
    if (opts) o = *opts; else qs_plan_opts_default(&o);
    g_last_error = plan_failure(rc, n, gates, ngates, o);
  }
  return rc;
}

static int plan_circuit_impl(int32_t n, const qs_gate* gates, uint64_t ngates, const qs_plan_opts* opts,
                             qs_plan** out) {
  if (!out) return QS_EINVAL;
  *out = nullptr;
  if (n < 1 || n > kMaxQubits || (ngates > 0 && !gates)) return QS_EINVAL;
  qs_plan_opts o;
  if (opts) o = *opts; else qs_plan_opts_default(&o);
  if (o.shm_max_active < 1 || o.shm_max_active > kMaxShmActive) return QS_EINVAL;
  if (o.forced_low < 0 || o.forced_low > o.shm_max_active) return QS_EINVAL;
  if (o.fuse_kmax < 0 || o.fuse_kmax > kMaxFuse) return QS_EINVAL;
  if (o.fuse_kmin < 0 || (o.fuse_kmax > 0 && o.fuse_kmin > o.fuse_kmax)) return QS_EINVAL;
  if (o.precision < QS_PREC_FP32 || o.precision > QS_PREC_TF32X3) return QS_EINVAL;
  if (o.algo < QS_ALGO_PER_GATE || o.algo > QS_ALGO_KERNELIZE) return QS_EINVAL;
  if (o.cost_kind == QS_COST_LEARNED && !o.mlp) return QS_EINVAL;
  if (o.cost_kind != QS_COST_ANALYTIC && o.cost_kind != QS_COST_LEARNED) return QS_EINVAL;
  if (o.shm_variant < 0 || o.shm_variant > 3) return QS_EINVAL;
  if (o.local_qubits < 0) return QS_EINVAL;
  if (o.stager != QS_STAGER_BEAM && o.stager != QS_STAGER_EXACT) return QS_EINVAL;
  if (o.insular_x < 0 || o.insular_x > (QS_INSULAR_X_REWRITE | QS_INSULAR_X_STAGED)) return QS_EINVAL;
  if (o.local_qubits >= n) o.local_qubits = 0;
  const bool staged = o.local_qubits > 0;
  // insular X: plan the Pauli-frame rewrite of the circuit (no X gate before
  // its final frame layer)
  std::vector<qs_gate> rewritten;
  if (o.insular_x & QS_INSULAR_X_REWRITE) {
    const int rrc = pauli_frame_rewrite(n, gates, ngates, &rewritten);
    if (rrc != QS_OK) return rrc;
    gates = rewritten.data();
    ngates = rewritten.size();
  }
  // a chunk holds the widest kernel (a 2^14 tile, a widened fused kernel)
  if (staged && (o.local_qubits < kMinLocalQubits || o.local_qubits < o.shm_max_active ||
                 o.local_qubits < o.forced_low + 2))
    return QS_EINVAL;
  if (o.precision != QS_PREC_FP32 && o.fuse_kmax > 0) {
    // tensor-core fused kernels are 2^6 wide: narrower kernels are widened
    if (o.fuse_kmax > kTcTargets || n < kTcTargets + 5) return QS_EUNSUPPORTED;
    o.fuse_kmin = kTcTargets;
  }
  auto t0 = std::chrono::steady_clock::now();
  qs_plan* p = new (std::nothrow) qs_plan();
  if (!p) return QS_ENOMEM;
  PlanImpl& P = p->impl;
  P.n = n;
  P.opts = o;
  if (o.cost) P.cost = *o.cost; else qs_cost_table_default(&P.cost);
  P.opts.cost = nullptr;
  o.cost = &P.cost;
  try {
    int rc = QS_OK;
    if (!staged) {
      rc = build_impl(P, n, gates, nullptr, nullptr, ngates);
    } else {
      P.gates.resize(ngates);
      for (uint64_t i = 0; i < ngates && rc == QS_OK; ++i) rc = make_gate(gates[i], n, &P.gates[i]);
      if (rc == QS_OK) rc = build_staged(p, gates, o);
      if (rc == QS_OK) rc = validate_staged(p);
    }
    if (rc != QS_OK) {
      qs_plan_free(p);
      return rc;
    }
  } catch (const std::bad_alloc&) {
    qs_plan_free(p);
    return QS_ENOMEM;
  } catch (...) {
    qs_plan_free(p);
    return QS_EPLAN;
  }
  P.planner_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  *out = p;
  return QS_OK;
}

void qs_plan_free(qs_plan* p) {
  if (!p) return;
  int cur = -1;
  cudaGetDevice(&cur);
  bool any = !p->impl.dev.empty();
  free_device(p->impl);
  for (auto& st : p->stages)
    if (st.plan) {
      any = any || !st.plan->dev.empty();
      free_device(*st.plan);
    }
  if (cur >= 0 && any) cudaSetDevice(cur);
  delete p;
}

int qs_plan_stats_get(const qs_plan* p, qs_plan_stats* s) {
  if (!p || !s) return QS_EINVAL;
  const PlanImpl& P = p->impl;
  std::memset(s, 0, sizeof(*s));
  s->n = P.n;
  s->num_stages = p->stages.empty() ? 1 : (int32_t)p->stages.size();
  s->num_gates = P.gates.size();
  s->num_kernels = P.kernels.size();
  for (const auto& k : P.kernels) (k.type == QS_KERNEL_SHM ? s->num_shm : s->num_fused)++;
  s->cost = P.total_cost;
  s->planner_ms = P.planner_ms;
  s->dp_states = P.dp_states;
  auto count = [&](const PlanImpl& Q) {
    for (const auto& pg : Q.shm2)
      if (pg.ok) {
        s->num_phased++;
        s->num_exchanges += (uint64_t)(pg.num_phases - 1);
        if (pg.jit_module >= 0) s->num_jit++;
      }
  };
  if (p->stages.empty()) count(P);
  for (const auto& st : p->stages) count(*st.plan);
  s->jit_ms = P.jit_ms;
  std::vector<uint64_t> sets;
  for (const auto& st : p->stages) sets.push_back(st.local);
  s->staging_cost = staging_objective(sets);
  s->staging_optimal = p->staging_optimal;
  return QS_OK;
}

int qs_plan_kernel(const qs_plan* p, uint64_t k, qs_kernel_desc* out) {
  if (!p || !out || k >= p->impl.kernels.size()) return QS_EINVAL;
  const Kernel& K = p->impl.kernels[k];
  out->type = K.type;
  out->stage = K.stage;
  out->nqubits = std::popcount(K.mask);
  out->num_gates = (int32_t)K.gates.size();
  out->qubit_mask = K.mask;
  out->cost = K.cost;
  return QS_OK;
}

int64_t qs_plan_kernel_gates(const qs_plan* p, uint64_t k, int32_t* ids, uint64_t cap) {
  if (!p || k >= p->impl.kernels.size()) return QS_EINVAL;
  const Kernel& K = p->impl.kernels[k];
  if (ids) {
    if (cap < K.gates.size()) return QS_EINVAL;
    std::copy(K.gates.begin(), K.gates.end(), ids);
  }
  return (int64_t)K.gates.size();
}

// The plan and kernel index that hold kernel k's programs.
static const PlanImpl* program_of(const qs_plan* p, uint64_t k, uint64_t* local) {
  if (p->stages.empty()) {
    *local = k;
    return &p->impl;
  }
  const auto& [si, lk] = p->kmap[k];
  *local = (uint64_t)lk;
  return p->stages[si].plan.get();
}

int qs_plan_fused_matrix(const qs_plan* p, uint64_t k, double* out, uint64_t cap) {
  if (!p || !out || k >= p->impl.kernels.size()) return QS_EINVAL;
  if (p->impl.kernels[k].type != QS_KERNEL_FUSED) return QS_EINVAL;
  uint64_t lk = 0;
  const PlanImpl* Q = program_of(p, k, &lk);
  // positions of a stage's local qubits ascend with the logical qubits, so
  // the matrix's target order is the same in both labellings
  const auto& u = Q->fused[lk].u64;
  if (cap < u.size()) return QS_EINVAL;
  std::copy(u.begin(), u.end(), out);
  return QS_OK;
}

int64_t qs_plan_kernel_source(const qs_plan* p, uint64_t k, char* out, uint64_t cap) {
  if (!p || k >= p->impl.kernels.size()) return QS_EINVAL;
  uint64_t lk = 0;
  const PlanImpl* Q = program_of(p, k, &lk);
  if (lk >= Q->shm2.size() || !Q->shm2[lk].ok) return QS_EINVAL;
  std::string src;
  if (!jit_source(Q->shm2[lk], Q->n, "qsk" + std::to_string(lk), &src)) return QS_EINVAL;
  if (out) {
    if (cap < src.size() + 1) return QS_EINVAL;
    std::memcpy(out, src.c_str(), src.size() + 1);
  }
  return (int64_t)src.size();
}

int64_t qs_plan_kernel_program(const qs_plan* p, uint64_t k, uint32_t* words, uint64_t cap, int32_t* layout) {
  if (!p || k >= p->impl.kernels.size()) return QS_EINVAL;
  uint64_t lk = 0;
  const PlanImpl* Q = program_of(p, k, &lk);
  if (lk >= Q->shm2.size() || !Q->shm2[lk].ok) return QS_EINVAL;
  const ShmProgramV2& pg = Q->shm2[lk];
  if (words) {
    if (cap < pg.prog.size()) return QS_EINVAL;
    std::copy(pg.prog.begin(), pg.prog.end(), words);
  }
  if (layout) {
    layout[0] = pg.m;
    for (int j = 0; j < kMaxShmActive; ++j) layout[1 + j] = j < pg.m ? pg.act[j] : -1;
    for (int i = 0; i < kRegBits; ++i) layout[15 + i] = pg.load.R[i];
  }
  return (int64_t)pg.prog.size();
}

int qs_insular_x_rewrite(int32_t n, const qs_gate* gates, uint64_t ngates, qs_gate* out, uint64_t cap,
                         uint64_t* nout) {
  if (!nout || n < 1 || n > kMaxQubits || (ngates && !gates)) return QS_EINVAL;
  std::vector<qs_gate> r;
  const int rc = pauli_frame_rewrite(n, gates, ngates, &r);
  if (rc != QS_OK) return rc;
  *nout = r.size();
  if (out) {
    if (cap < r.size()) return QS_EINVAL;
    std::copy(r.begin(), r.end(), out);
  }
  return QS_OK;
}

int qs_plan_validate(const qs_plan* p, const qs_gate* gates, uint64_t ngates) {
  if (!p) return QS_EINVAL;
  const PlanImpl& P = p->impl;
  std::vector<qs_gate> rewritten;  // an insular-X plan executes the rewritten circuit
  if ((P.opts.insular_x & QS_INSULAR_X_REWRITE) && (ngates == 0 || gates)) {
    if (pauli_frame_rewrite(P.n, gates, ngates, &rewritten) != QS_OK) return QS_EPLAN;
    gates = rewritten.data();
    ngates = rewritten.size();
  }
  if (ngates != P.gates.size() || (ngates && !gates)) return QS_EPLAN;
  for (uint64_t i = 0; i < ngates; ++i) {
    Gate g;
    if (make_gate(gates[i], P.n, &g) != QS_OK) return QS_EPLAN;
    const Gate& h = P.gates[i];
    if (g.type != h.type || g.q0 != h.q0 || g.q1 != h.q1) return QS_EPLAN;
  }
  return p->stages.empty() ? validate_plan(&P) : validate_staged(p);
}

int qs_plan_stage_frame(const qs_plan* p, int32_t stage, uint64_t* frame, int32_t* flip_gates, int64_t cap,
                        int64_t* num_flips) {
  if (!p || !frame || !num_flips) return QS_EINVAL;
  const int32_t ns = p->stages.empty() ? 1 : (int32_t)p->stages.size();
  if (stage < 0 || stage >= ns) return QS_EINVAL;
  if (p->stages.empty()) {
    *frame = 0;
    *num_flips = 0;
    return QS_OK;
  }
  const Stage& st = p->stages[stage];
  *frame = st.frame;
  *num_flips = (int64_t)st.flips.size();
  if (flip_gates) {
    if (cap < (int64_t)st.flips.size()) return QS_EINVAL;
    std::copy(st.flips.begin(), st.flips.end(), flip_gates);
  }
  return QS_OK;
}

int qs_plan_stage(const qs_plan* p, int32_t stage, uint64_t* local_mask, int64_t* num_gates,
                  int32_t* first_kernel, int32_t* num_kernels) {
  if (!p) return QS_EINVAL;
  const int32_t ns = p->stages.empty() ? 1 : (int32_t)p->stages.size();
  if (stage < 0 || stage >= ns) return QS_EINVAL;
  const PlanImpl& P = p->impl;
  int32_t first = -1, cnt = 0;
  for (size_t k = 0; k < P.kernels.size(); ++k)
    if (P.kernels[k].stage == stage) {
      if (first < 0) first = (int32_t)k;
      cnt++;
    }
  if (local_mask) *local_mask = p->stages.empty() ? (P.n >= 64 ? ~0ull : (1ull << P.n) - 1) : p->stages[stage].local;
  if (num_gates) *num_gates = p->stages.empty() ? (int64_t)P.gates.size() : (int64_t)p->stages[stage].gates.size();
  if (first_kernel) *first_kernel = first < 0 ? 0 : first;
  if (num_kernels) *num_kernels = cnt;
  return QS_OK;
}

int qs_state_create(int32_t n, void* device_ptr, qs_state** out) {
  if (!out) return QS_EINVAL;
  *out = nullptr;
  if (n < 1 || n > 34) return QS_EINVAL;
  if (device_ptr && (reinterpret_cast<uintptr_t>(device_ptr) & 15)) return QS_EINVAL;
  qs_state* s = new (std::nothrow) qs_state();
  if (!s) return QS_ENOMEM;
  s->n = n;
  if (device_ptr) {
    s->psi = static_cast<float2*>(device_ptr);
  } else {
    size_t bytes = sizeof(float2) << n;
    cudaError_t e = cudaMalloc(&s->psi, bytes);
    if (e != cudaSuccess) {
      delete s;
      return cuda_status(e);
    }
    s->owned = true;
  }
  *out = s;
  return QS_OK;
}

int qs_alloc_state(int32_t n, void* stream, qs_state** out) {
  int rc = qs_state_create(n, nullptr, out);
  if (rc != QS_OK) return rc;
  rc = qs_state_set_zero(*out, stream);
  if (rc != QS_OK) {
    qs_state_free(*out);
    *out = nullptr;
  }
  return rc;
}

void qs_state_free(qs_state* s) {
  if (!s) return;
  if (s->owned && s->psi) cudaFree(s->psi);
  delete s;
}

void* qs_state_device_ptr(const qs_state* s) { return s ? s->psi : nullptr; }

int qs_state_set_zero(qs_state* s, void* stream) {
  if (!s) return QS_EINVAL;
  return launch_set_zero(s->psi, s->n, (cudaStream_t)stream);
}

struct qs_timer {
  const qs_plan* plan = nullptr;
  uint64_t max_runs = 0, runs = 0;
  std::vector<cudaEvent_t> ev;  // (nk + 1) per run
};

static int run_plan_impl(const qs_plan* plan, qs_state* st, void* stream, qs_timer* tm);

int qs_timer_create(const qs_plan* plan, uint64_t max_runs, qs_timer** out) {
  if (!plan || !out || max_runs == 0) return QS_EINVAL;
  *out = nullptr;
  if (!plan->stages.empty()) return QS_EUNSUPPORTED;
  qs_timer* t = new (std::nothrow) qs_timer();
  if (!t) return QS_ENOMEM;
  t->plan = plan;
  t->max_runs = max_runs;
  const uint64_t per = plan->impl.kernels.size() + 1;
  t->ev.assign(per * max_runs, nullptr);
  for (auto& e : t->ev) {
    cudaError_t r = cudaEventCreate(&e);
    if (r != cudaSuccess) {
      qs_timer_free(t);
      return cuda_status(r);
    }
  }
  *out = t;
  return QS_OK;
}

void qs_timer_free(qs_timer* t) {
  if (!t) return;
  for (auto e : t->ev)
    if (e) cudaEventDestroy(e);
  delete t;
}

int qs_run_plan_timed(const qs_plan* plan, qs_state* st, qs_timer* t, void* stream) {
  if (!t || t->plan != plan) return QS_EINVAL;
  if (t->runs >= t->max_runs) return QS_EINVAL;
  return run_plan_impl(plan, st, stream, t);
}

int qs_timer_read(qs_timer* t, double* per_kernel_ms, uint64_t cap, uint64_t* runs) {
  if (!t || !runs) return QS_EINVAL;
  const uint64_t nk = t->plan->impl.kernels.size();
  if (nk && (!per_kernel_ms || cap < nk)) return QS_EINVAL;
  for (uint64_t k = 0; k < nk; ++k) per_kernel_ms[k] = 0;
  for (uint64_t r = 0; r < t->runs; ++r) {
    for (uint64_t k = 0; k < nk; ++k) {
      float ms = 0;
      cudaEvent_t a = t->ev[r * (nk + 1) + k], b = t->ev[r * (nk + 1) + k + 1];
      cudaError_t e = cudaEventSynchronize(b);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
      if (e != cudaSuccess) return cuda_status(e);
      per_kernel_ms[k] += ms;
    }
  }
  *runs = t->runs;
  return QS_OK;
}

int qs_run_plan(const qs_plan* plan, qs_state* st, void* stream) {
  return run_plan_impl(plan, st, stream, nullptr);
}

}  // extern "C"

namespace qs {

// Launches the kernels of P on psi, a view of 2^n_addr amplitudes whose
// qubits above n_addr have the known values `hi` (chunked execution; for a
// resident state n_addr = P.n and hi = 0).  ev: nk + 1 events or null.
static int run_kernels(PlanImpl* P, DeviceCache* dc, float2* psi, int n_addr, uint64_t hi,
                       cudaStream_t s, cudaEvent_t* ev) {
  int rc = QS_OK;
  for (size_t i = 0; i < P->kernels.size(); ++i) {
    const Kernel& K = P->kernels[i];
    if (ev) {
      cudaError_t e = cudaEventRecord(ev[i], s);
      if (e != cudaSuccess) return cuda_status(e);
    }
    const uint8_t* base = static_cast<const uint8_t*>(dc->buf) + dc->op_off[i];
    if (K.type == QS_KERNEL_SHM && dc->jit_kernel[i]) {
      rc = launch_jit(dc->jit_kernel[i], P->shm2[i], dc->jit_blocks[i], psi, n_addr, hi, s);
    } else if (K.type == QS_KERNEL_SHM && P->shm2[i].ok) {
      ShmV2Launch a;
      a.psi = psi;
      a.hi = hi;
      a.n = n_addr;
      a.amask = K.mask;
      a.prog = reinterpret_cast<const uint32_t*>(static_cast<const uint8_t*>(dc->buf) + dc->prog_off[i]);
      a.pg = &P->shm2[i];
      rc = launch_shm_v2(a, s);
    } else if (K.type == QS_KERNEL_SHM) {
      const ShmProgram& sp = P->shm[i];
      ShmLaunch a;
      a.psi = psi;
      a.hi = hi;
      a.n = n_addr;
      a.m = sp.m;
      std::copy(sp.act, sp.act + kMaxShmActive, a.act);
      a.ops = reinterpret_cast<const DevOp*>(base);
      a.nops = (int)sp.ops.size();
      rc = launch_shm(a, s);
    } else {
      const FusedProgram& fp = P->fused[i];
      FusedLaunch a;
      a.psi = psi;
      a.n = n_addr;
      a.k = fp.k;
      std::copy(fp.targets, fp.targets + kMaxFuse, a.targets);
      a.u = reinterpret_cast<const float2*>(base);
      a.precision = P->opts.precision;
      rc = launch_fused(a, s);
    }
    if (rc != QS_OK) return rc;
  }
  if (ev) {
    cudaError_t e = cudaEventRecord(ev[P->kernels.size()], s);
    if (e != cudaSuccess) return cuda_status(e);
  }
  return QS_OK;
}

}  // namespace qs

extern "C" {

static int run_plan_impl(const qs_plan* plan, qs_state* st, void* stream, qs_timer* tm) {
  if (!plan || !st) return QS_EINVAL;
  if (!plan->stages.empty()) return QS_EUNSUPPORTED;  // staged plans run through qs_run_plan_host
  PlanImpl* P = const_cast<PlanImpl*>(&plan->impl);
  if (P->n != st->n) return QS_EINVAL;
  DeviceCache* dc = nullptr;
  int rc = ensure_device(P, &dc);
  if (rc != QS_OK) return rc;
  cudaEvent_t* ev = tm ? &tm->ev[tm->runs * (P->kernels.size() + 1)] : nullptr;
  rc = run_kernels(P, dc, st->psi, P->n, 0, (cudaStream_t)stream, ev);
  if (rc == QS_OK && ev) tm->runs++;
  return rc;
}

// ---- host-resident state: Alg. 1's Execute with the shards in host memory ----

struct qs_host_timer {
  const qs_plan* plan = nullptr;
  uint64_t nrec = 0;                // stages x chunks
  std::vector<cudaEvent_t> ev;      // 1 + 4 per record
  bool recorded = false;
};

static int run_plan_host_impl(const qs_plan* plan, float* host_state, void* device_buffer,
                              uint64_t buffer_bytes, void* stream, qs_host_timer* tm);

int qs_run_plan_host(const qs_plan* plan, float* host_state, void* device_buffer,
                     uint64_t buffer_bytes, void* stream) {
  return run_plan_host_impl(plan, host_state, device_buffer, buffer_bytes, stream, nullptr);
}

static uint64_t host_records(const qs_plan* plan) {
  const uint64_t stages = plan->stages.empty() ? 1 : plan->stages.size();
  const int L = plan->stages.empty() ? plan->impl.n : plan->impl.opts.local_qubits;
  return stages << (plan->impl.n - L);
}

int qs_host_timer_create(const qs_plan* plan, qs_host_timer** out) {
  if (!plan || !out) return QS_EINVAL;
  *out = nullptr;
  const uint64_t nrec = host_records(plan);
  if (nrec > kMaxHostTimerRecords) return QS_EINVAL;
  qs_host_timer* t = new (std::nothrow) qs_host_timer();
  if (!t) return QS_ENOMEM;
  t->plan = plan;
  t->nrec = nrec;
  t->ev.assign(1 + 4 * nrec, nullptr);
  for (auto& e : t->ev) {
    cudaError_t r = cudaEventCreate(&e);
    if (r != cudaSuccess) {
      qs_host_timer_free(t);
      return cuda_status(r);
    }
  }
  *out = t;
  return QS_OK;
}

void qs_host_timer_free(qs_host_timer* t) {
  if (!t) return;
  for (auto e : t->ev)
    if (e) cudaEventDestroy(e);
  delete t;
}

int qs_run_plan_host_timed(const qs_plan* plan, float* host_state, void* device_buffer,
                           uint64_t buffer_bytes, qs_host_timer* t, void* stream) {
  if (!t || t->plan != plan) return QS_EINVAL;
  return run_plan_host_impl(plan, host_state, device_buffer, buffer_bytes, stream, t);
}

int qs_host_timer_read(qs_host_timer* t, double* ms, uint64_t cap, uint64_t* nrec) {
  if (!t || !nrec) return QS_EINVAL;
  if (!t->recorded) return QS_EINVAL;
  if (!ms || cap < 4 * t->nrec) return QS_EINVAL;
  cudaError_t e = cudaEventSynchronize(t->ev[0]);
  for (uint64_t i = 0; i < 4 * t->nrec && e == cudaSuccess; ++i) {
    float v = 0;
    e = cudaEventSynchronize(t->ev[1 + i]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&v, t->ev[0], t->ev[1 + i]);
    ms[i] = v;
  }
  if (e != cudaSuccess) return cuda_status(e);
  *nrec = t->nrec;
  return QS_OK;
}

static int run_plan_host_impl(const qs_plan* plan, float* host_state, void* device_buffer,
                              uint64_t buffer_bytes, void* stream, qs_host_timer* tm) {
  if (!plan || !host_state) return QS_EINVAL;
  if (reinterpret_cast<uintptr_t>(host_state) & 15) return QS_EINVAL;
  const PlanImpl& P = plan->impl;
  const int n = P.n;
  // a staged plan of an empty circuit has no stage: nothing to apply (and
  // the state may not fit on the device)
  if (P.opts.local_qubits > 0 && P.opts.local_qubits < n && plan->stages.empty()) return QS_OK;
  const bool staged = !plan->stages.empty();
  const int L = staged ? P.opts.local_qubits : n;
  const uint64_t chunk_bytes = sizeof(float2) << L;
  // the state must be page-locked (cudaMallocHost / cudaHostRegister) for
  // the copies to run asynchronously on the copy engines
  cudaPointerAttributes at{};
  cudaError_t e = cudaPointerGetAttributes(&at, host_state);
  if (e != cudaSuccess) return cuda_status(e);
  if (at.type != cudaMemoryTypeHost) return QS_EINVAL;
  bool framed = false;  // a stage writes its chunks back relabelled: pairs need two buffers
  for (const Stage& st : plan->stages) framed |= st.frame != 0;
  int nbuf = 0;
  float2* dbuf = static_cast<float2*>(device_buffer);
  if (dbuf) {
    if (reinterpret_cast<uintptr_t>(dbuf) & 255) return QS_EINVAL;
    nbuf = (int)std::min<uint64_t>(kMaxChunkBuffers, buffer_bytes / chunk_bytes);
    if (nbuf < (framed ? 2 : 1)) return QS_EINVAL;
  }
  // device programs of every stage, before any work is queued
  std::vector<PlanImpl*> plans;
  if (staged)
    for (const auto& st : plan->stages) plans.push_back(st.plan.get());
  else
    plans.push_back(const_cast<PlanImpl*>(&P));
  std::vector<DeviceCache*> dcs(plans.size(), nullptr);
  for (size_t i = 0; i < plans.size(); ++i) {
    int rc = ensure_device(plans[i], &dcs[i]);
    if (rc != QS_OK) return rc;
  }
  const cudaStream_t user = (cudaStream_t)stream;
  cudaStream_t ss[kMaxChunkBuffers] = {};
  cudaEvent_t evs[kMaxChunkBuffers + 1] = {};
  const int nchunks_log = n - L;
  if (!dbuf) nbuf = nchunks_log == 0 ? 1 : std::min(kMaxChunkBuffers, 2);
  int rc = QS_OK;
  bool allocated = false;
  auto fail = [&](cudaError_t err) {
    if (rc == QS_OK && err != cudaSuccess) rc = cuda_status(err);
    return rc != QS_OK;
  };
  for (int b = 0; b < nbuf && rc == QS_OK; ++b)
    fail(cudaStreamCreateWithFlags(&ss[b], cudaStreamNonBlocking));
  for (int b = 0; b <= nbuf && rc == QS_OK; ++b)
    fail(cudaEventCreateWithFlags(&evs[b], cudaEventDisableTiming));
  // per buffer: its chunk's copy-in and kernels are queued (paired chunks)
  cudaEvent_t inev[kMaxChunkBuffers] = {};
  for (int b = 0; b < nbuf && rc == QS_OK; ++b)
    fail(cudaEventCreateWithFlags(&inev[b], cudaEventDisableTiming));
  if (tm) {
    tm->recorded = false;
    if (rc == QS_OK) fail(cudaEventRecord(tm->ev[0], user));
  }
  // the internal streams start after the caller's stream
  if (rc == QS_OK && !fail(cudaEventRecord(evs[nbuf], user)))
    for (int b = 0; b < nbuf && rc == QS_OK; ++b) fail(cudaStreamWaitEvent(ss[b], evs[nbuf], 0));
  if (rc == QS_OK && !dbuf) {
    void* mem = nullptr;
    if (!fail(cudaMallocAsync(&mem, chunk_bytes * nbuf, ss[0]))) {
      dbuf = static_cast<float2*>(mem);
      allocated = true;
      if (!fail(cudaEventRecord(evs[0], ss[0])))
        for (int b = 1; b < nbuf && rc == QS_OK; ++b) fail(cudaStreamWaitEvent(ss[b], evs[0], 0));
    }
  }
  float2* hs = reinterpret_cast<float2*>(host_state);
  const uint64_t nch = 1ull << nchunks_log;
  int dev = 0;
  cudaGetDevice(&dev);
  int max_pitch = 0;
  cudaDeviceGetAttribute(&max_pitch, cudaDevAttrMaxPitch, dev);
  // done[parity][c]: chunk c of the last stage of that parity is back in
  // host memory.  A chunk of the next stage waits only for the chunks its
  // amplitudes come from, so stages overlap at their boundary.
  const bool multi = plans.size() > 1;
  std::vector<cudaEvent_t> done[2];
  if (multi)
    for (auto& v : done) {
      v.assign(nch, nullptr);
      for (auto& ev : v)
        if (rc == QS_OK) fail(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    }
  uint64_t gchunk = 0;  // chunks take the buffers round-robin across stages
  for (size_t si = 0; si < plans.size() && rc == QS_OK; ++si) {
    const Stage* st = staged ? &plan->stages[si] : nullptr;
    const Stage* prev = staged && si > 0 ? &plan->stages[si - 1] : nullptr;
    // A chunk is 2^(L - run_log) host runs of 2^run_log amplitudes; the
    // local qubits above run_log, ascending, index the runs.  The lowest
    // `g` of them are consecutive qubits, so those runs are evenly spaced in
    // host memory (pitch 2^q0 amplitudes) and move with one 2D copy.
    const int run_log = staged ? st->run_log : n;
    const uint64_t run_amps = 1ull << run_log;
    int g = 0;
    if (staged)
      while (run_log + g + 1 < L && st->order[run_log + g + 1] == st->order[run_log] + g + 1) ++g;
    if (staged && run_log < L) ++g;  // the group holds order[run_log .. run_log + g - 1]
    const uint64_t hpitch = staged && run_log < L ? (sizeof(float2) << st->order[run_log]) : 0;
    if (hpitch == 0 || hpitch > (uint64_t)max_pitch) g = 0;
    const uint64_t rows = 1ull << g;
    const uint64_t nouter = 1ull << (L - run_log - g);
    auto deposit = [&](uint64_t v, int from, int count) {
      uint64_t x = 0;
      for (int t = 0; t < count; ++t)
        if ((v >> t) & 1) x |= 1ull << st->order[from + t];
      return x;
    };
    auto copy = [&](float2* d, uint64_t hbase, cudaStream_t s, bool in) {
      for (uint64_t r = 0; r < nouter && rc == QS_OK; ++r) {
        const uint64_t h = hbase | (staged ? deposit(r << g, run_log, L - run_log) : 0);
        float2* dp = d + ((r << g) << run_log);
        const size_t w = run_amps * sizeof(float2);
        if (rows == 1)
          fail(in ? cudaMemcpyAsync(dp, hs + h, w, cudaMemcpyHostToDevice, s)
                  : cudaMemcpyAsync(hs + h, dp, w, cudaMemcpyDeviceToHost, s));
        else
          fail(in ? cudaMemcpy2DAsync(dp, w, hs + h, hpitch, w, rows, cudaMemcpyHostToDevice, s)
                  : cudaMemcpy2DAsync(hs + h, hpitch, dp, w, w, rows, cudaMemcpyDeviceToHost, s));
      }
    };
    // copy-in after a stage boundary: units of 2^jin amplitudes, each inside
    // one chunk of the previous stage (a previous regional qubit below
    // run_log splits the runs), issued source chunk by source chunk
    int jin = run_log;
    if (prev)
      for (int k = L; k < n; ++k)
        if (prev->order[k] < jin && ((st->local >> prev->order[k]) & 1)) jin = prev->order[k];
    const uint64_t nunits = prev ? 1ull << (L - jin) : 0;
    auto source_of = [&](uint64_t h) {
      uint64_t c = 0;
      for (int k = L; k < n; ++k) c |= ((h >> prev->order[k]) & 1ull) << (k - L);
      return c;
    };
    std::vector<std::pair<uint64_t, uint64_t>> units;  // (source chunk, unit index)
    // the stage's frame in chunk-index bits: the stored chunk c holds the
    // logical chunk c ^ fc, so it is written back there (insular X gates)
    uint64_t fc = 0;
    if (staged)
      for (int k = L; k < n; ++k)
        if ((st->frame >> st->order[k]) & 1) fc |= 1ull << (k - L);
    struct Slot {
      uint64_t c = 0;
      int b = 0;
    };
    // copy-in (after a stage boundary: unit by unit, each after the previous
    // stage's chunk it comes from) and the stage's kernels
    auto load_run = [&](const Slot& x) {
      const cudaStream_t s = ss[x.b];
      float2* d = dbuf + (uint64_t(x.b) << L);
      const uint64_t hbase = staged ? deposit(x.c, L, n - L) : 0;
      cudaEvent_t* te = tm ? &tm->ev[1 + 4 * (si * nch + x.c)] : nullptr;
      if (te && rc == QS_OK) fail(cudaEventRecord(te[0], s));
      if (!prev) {
        copy(d, hbase, s, true);
      } else {
        units.clear();
        for (uint64_t u = 0; u < nunits; ++u) {
          const uint64_t h = hbase | deposit(u, jin, L - jin);
          units.push_back({source_of(h), u});
        }
        std::sort(units.begin(), units.end());
        uint64_t waited = ~0ull;
        for (const auto& [src, u] : units) {
          if (rc != QS_OK) break;
          if (src != waited) {
            fail(cudaStreamWaitEvent(s, done[(si - 1) & 1][src], 0));
            waited = src;
          }
          const uint64_t h = hbase | deposit(u, jin, L - jin);
          fail(cudaMemcpyAsync(d + (u << jin), hs + h, sizeof(float2) << jin, cudaMemcpyHostToDevice, s));
        }
      }
      if (te && rc == QS_OK) fail(cudaEventRecord(te[1], s));
      if (rc == QS_OK) rc = run_kernels(plans[si], dcs[si], d, L, x.c << L, s, nullptr);
      if (te && rc == QS_OK) fail(cudaEventRecord(te[2], s));
    };
    // copy-out of chunk x.c to host chunk x.c ^ fc
    auto store = [&](const Slot& x) {
      const cudaStream_t s = ss[x.b];
      float2* d = dbuf + (uint64_t(x.b) << L);
      const uint64_t to = x.c ^ fc;
      copy(d, staged ? deposit(to, L, n - L) : 0, s, false);
      cudaEvent_t* te = tm ? &tm->ev[1 + 4 * (si * nch + x.c)] : nullptr;
      if (te && rc == QS_OK) fail(cudaEventRecord(te[3], s));
      if (multi && rc == QS_OK) fail(cudaEventRecord(done[si & 1][to], s));
    };
    for (uint64_t c = 0; c < nch && rc == QS_OK; ++c) {
      if (!fc) {
        Slot x{c, (int)(gchunk++ % (uint64_t)nbuf)};
        load_run(x);
        store(x);
        continue;
      }
      if ((c ^ fc) < c) continue;  // handled with its partner
      // a pair: each copy-out overwrites the partner's host chunk, so it
      // waits for the partner's copy-in
      Slot x{c, (int)(gchunk++ % (uint64_t)nbuf)};
      Slot y{c ^ fc, (int)(gchunk++ % (uint64_t)nbuf)};
      load_run(x);
      if (rc == QS_OK) fail(cudaEventRecord(inev[x.b], ss[x.b]));
      load_run(y);
      if (rc == QS_OK) fail(cudaEventRecord(inev[y.b], ss[y.b]));
      if (rc == QS_OK) fail(cudaStreamWaitEvent(ss[x.b], inev[y.b], 0));
      if (rc == QS_OK) fail(cudaStreamWaitEvent(ss[y.b], inev[x.b], 0));
      store(x);
      store(y);
    }
  }
  for (auto& v : done)
    for (auto ev : v)
      if (ev) cudaEventDestroy(ev);
  // join: the caller's stream continues after every chunk is back in host memory
  for (int b = 1; b < nbuf; ++b)
    if (ss[b] && evs[b] && cudaEventRecord(evs[b], ss[b]) == cudaSuccess) cudaStreamWaitEvent(ss[0], evs[b], 0);
  if (allocated) cudaFreeAsync(dbuf, ss[0]);
  if (ss[0] && evs[0] && cudaEventRecord(evs[0], ss[0]) == cudaSuccess) cudaStreamWaitEvent(user, evs[0], 0);
  for (int b = 0; b < nbuf; ++b)
    if (ss[b]) cudaStreamDestroy(ss[b]);
  for (int b = 0; b <= nbuf; ++b)
    if (evs[b]) cudaEventDestroy(evs[b]);
  for (int b = 0; b < nbuf; ++b)
    if (inev[b]) cudaEventDestroy(inev[b]);
  if (tm && rc == QS_OK) tm->recorded = true;
  return rc;
}

// Amplitudes [first, first + count) of a state, to or from host memory;
// the range is checked before any address is formed.
static int copy_amps(const qs_state* st, float* host, uint64_t first, uint64_t count, bool to_host,
                     cudaStream_t s) {
  if (count == 0) return QS_OK;
  const uint64_t size = 1ull << st->n;
  if (first > size || count > size - first) return QS_EINVAL;
  float2* dev = st->psi + first;
  cudaError_t e = to_host ? cudaMemcpyAsync(host, dev, count * sizeof(float2), cudaMemcpyDeviceToHost, s)
                          : cudaMemcpyAsync(dev, host, count * sizeof(float2), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_status(e);
  return tc_check_error(s, true);
}

int qs_read_amplitudes(const qs_state* st, uint64_t first, uint64_t count, float* host_out,
                       void* stream) {
  if (!st || (!host_out && count)) return QS_EINVAL;
  return copy_amps(st, host_out, first, count, true, (cudaStream_t)stream);
}

int qs_write_amplitudes(qs_state* st, uint64_t first, uint64_t count, const float* host_in,
                        void* stream) {
  if (!st || (!host_in && count)) return QS_EINVAL;
  return copy_amps(st, const_cast<float*>(host_in), first, count, false, (cudaStream_t)stream);
}

int qs_state_norm2(const qs_state* st, double* out, void* stream) {
  if (!st || !out) return QS_EINVAL;
  int rc = launch_norm2(st->psi, st->n, out, (cudaStream_t)stream);
  return rc == QS_OK ? tc_check_error((cudaStream_t)stream, true) : rc;
}

int qs_state_compare_c128(const qs_state* st, const double* ref, double* fid, double* maxabs,
                          void* stream) {
  if (!st || !ref || !fid || !maxabs) return QS_EINVAL;
  int rc = launch_compare(st->psi, reinterpret_cast<const double2*>(ref), st->n, fid, maxabs,
                          (cudaStream_t)stream);
  return rc == QS_OK ? tc_check_error((cudaStream_t)stream, true) : rc;
}

int qs_remap(const float* in, float* out, int32_t n, const int32_t* perm, void* stream) {
  if (!in || !out || !perm || n < 1 || n > 34) return QS_EINVAL;
  uint64_t seen = 0;
  for (int j = 0; j < n; ++j) {
    if (perm[j] < 0 || perm[j] >= n || ((seen >> perm[j]) & 1)) return QS_EINVAL;
    seen |= 1ull << perm[j];
  }
  const uint64_t bytes = sizeof(float2) << n;
  const char* a = reinterpret_cast<const char*>(in);
  const char* b = reinterpret_cast<const char*>(out);
  if (a < b + bytes && b < a + bytes) return QS_EINVAL;
  return launch_remap(reinterpret_cast<const float2*>(in), reinterpret_cast<float2*>(out), n, perm,
                      (cudaStream_t)stream);
}

int qs_apply_fused(float* state, int32_t n, const int32_t* targets, int32_t k, const float* u_host,
                   int32_t precision, void* stream) {
  if (!state || !targets || !u_host || k < 1 || k > kMaxFuse || n < k || n > 34) return QS_EINVAL;
  if (precision < QS_PREC_FP32 || precision > QS_PREC_TF32X3) return QS_EINVAL;
  uint64_t seen = 0;
  for (int j = 0; j < k; ++j) {
    if (targets[j] < 0 || targets[j] >= n || ((seen >> targets[j]) & 1)) return QS_EINVAL;
    seen |= 1ull << targets[j];
  }
  cudaStream_t s = (cudaStream_t)stream;
  FusedLaunch a;
  a.psi = reinterpret_cast<float2*>(state);
  a.n = n;
  a.k = k;
  std::fill(a.targets, a.targets + kMaxFuse, -1);
  std::copy(targets, targets + k, a.targets);
  a.precision = precision;
  std::vector<float> staged;  // what the kernel reads: the matrix or tensor-core weights
  if (precision == QS_PREC_FP32) {
    staged.assign(u_host, u_host + (size_t(2) << (2 * k)));
  } else {
    if (k > kTcTargets || n < kTcTargets + 5) return QS_EUNSUPPORTED;
    // widen to 6 targets with the lowest unused qubits: U (x) I
    std::vector<float> uw(size_t(2) << (2 * kTcTargets));
    widen_unitary(u_host, k, kTcTargets, uw.data());
    widen_targets(n, k, kTcTargets, a.targets);
    a.k = kTcTargets;
    tc_prepare_weights(uw.data(), precision == QS_PREC_TF32X3, &staged);
  }
  const size_t bytes = staged.size() * sizeof(float);
  void* du = nullptr;
  cudaError_t e = cudaMallocAsync(&du, bytes, s);
  if (e != cudaSuccess) return cuda_status(e);
  e = cudaMemcpyAsync(du, staged.data(), bytes, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) {
    cudaFreeAsync(du, s);
    return cuda_status(e);
  }
  a.u = static_cast<const float2*>(du);
  int rc = launch_fused(a, s);
  cudaFreeAsync(du, s);
  if (rc == QS_OK) rc = cuda_status(cudaStreamSynchronize(s));
  if (rc == QS_OK) rc = tc_check_error(s, true);
  return rc;
}

int qs_sync(void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  int rc = cuda_status(cudaStreamSynchronize(s));
  if (rc == QS_OK) rc = tc_check_error(s, true);
  return rc;
}

int32_t qs_debug_tc_launch_counts(uint64_t* out, int32_t cap) {
  if (!out || cap < 0) return QS_EINVAL;
  tc_launch_counts(out, cap);
  return kTcVariants;
}

int qs_debug_tc_stall(int64_t limit_us) {
  if (limit_us < 0 || limit_us > 10000000) return QS_EINVAL;
  tc_set_stall((uint64_t)limit_us * 1000ull);
  return QS_OK;
}

}  // extern "C"
