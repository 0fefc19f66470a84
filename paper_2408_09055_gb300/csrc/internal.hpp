// Internal types shared by the planner (host C++) and the CUDA kernels of
// libqsim.  Not part of the public ABI (see include/qsim.h).
#pragma once

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "qsim.h"
#include "shm_program.hpp"

namespace qs {

constexpr int kMaxQubits = 40;
constexpr int kMaxShmActive = 14;  // 2^14 complex64 = 128 KiB tile
constexpr int kMaxFuse = 7;        // widest fused unitary (2^7 x 2^7)

// ---- gates ---------------------------------------------------------------
struct Gate {
  int32_t type = 0, nq = 1, q0 = 0, q1 = -1;
  double p[3] = {0, 0, 0};
  uint64_t qmask = 0;   // all qubits of the gate
  uint64_t nimask = 0;  // non-insular qubits (Definition 2)
};

int gate_arity(int type);
// Fills m (row-major, complex interleaved, 2^nq x 2^nq) with the gate matrix.
void gate_matrix(const Gate& g, double* m);
// Validates a public gate and fills the internal one.  Returns QS_OK/EINVAL.
int make_gate(const qs_gate& in, int n, Gate* out);
bool gate_is_diagonal(int type);
// g' = X^flip g X^flip as table gates appended to out, plus a global phase
// added to *phase (radians); false when g is not insular on a flipped qubit.
bool conjugate_by_x(const qs_gate& g, uint64_t flip, std::vector<qs_gate>* out, double* phase);
// The circuit with every X moved to its end through a Pauli frame (exact,
// global phase included); QS_EINVAL for a malformed gate.
int pauli_frame_rewrite(int n, const qs_gate* in, uint64_t count, std::vector<qs_gate>* out);

struct LearnedCost;  // learned.cpp
// Discovery: between begin and end, a prediction not yet known reads as
// infeasible and is recorded; end runs one batched inference of the recorded
// kernels and returns whether there were any.
void learned_collect_begin(LearnedCost* lc);
bool learned_collect_end(LearnedCost* lc);

// ---- plan ----------------------------------------------------------------
struct Kernel {
  int32_t type = QS_KERNEL_SHM;
  int32_t stage = 0;
  std::vector<int32_t> gates;  // circuit indices, execution order
  uint64_t mask = 0;           // shm: active set; fused: target set (widened)
  double cost = 0;
};

// One device op of a shared-memory kernel program (see shm kernel).
enum : uint8_t { OP_DENSE1 = 0, OP_DENSE2 = 1, OP_DIAG = 2 };
struct alignas(16) DevOp {
  uint8_t kind;
  int8_t t0, t1;   // local bits (DENSE: targets; DIAG: qubit 0/1 if active, else -1)
  int8_t g0, g1;   // DIAG: physical bit of qubit 0/1 when not active, else -1
  uint8_t pad[3];
  uint32_t cloc;   // local control bits, all must be 1
  uint32_t pad2;
  uint64_t cglob;  // physical control bits of the batch, all must be 1
  float m[32];     // DENSE1: 2x2 complex; DENSE2: 4x4 complex; DIAG: 4 complex entries
};
static_assert(sizeof(DevOp) == 160, "DevOp layout");

struct ShmProgram {
  int m = 0;                 // |A|
  int act[kMaxShmActive];    // physical qubit of local bit j (ascending)
  std::vector<DevOp> ops;
};

struct FusedProgram {
  int k = 0;
  int targets[kMaxFuse];     // physical qubit of matrix index bit j
  std::vector<float> u;      // 2^k x 2^k complex64, row-major interleaved
  std::vector<double> u64;   // the FP64 product (kept for export / tests)
  std::vector<float> w_tc;   // tensor-core weights (k = 6, TF32 / 3xTF32), else empty
};

struct DeviceCache {
  int device = -1;
  void* buf = nullptr;       // ops + matrices of every kernel
  std::vector<uint64_t> op_off;  // byte offset of kernel i's ops / matrix
  std::vector<uint64_t> prog_off;  // byte offset of kernel i's phased program
  std::vector<cudaLibrary_t> libs;     // loaded JIT modules
  std::vector<cudaKernel_t> jit_kernel;  // per plan kernel (nullptr: none)
  std::vector<int> jit_blocks;           // its resident CTAs per SM
};

struct PlanImpl {
  int n = 0;
  std::vector<Gate> gates;
  qs_plan_opts opts{};
  qs_cost_table cost{};
  std::vector<Kernel> kernels;
  std::vector<ShmProgram> shm;      // indexed like kernels (empty for fused)
  std::vector<FusedProgram> fused;  // indexed like kernels (empty for shm)
  std::vector<ShmProgramV2> shm2;   // register-phased programs (ok = false: generic kernel)
  std::vector<std::vector<char>> jit_modules;  // cubins of the specialised kernels
  std::string jit_log;              // first NVRTC error log, if any
  double jit_ms = 0;
  double planner_ms = 0, total_cost = 0;
  // qubits a kernel may execute on (shm active set, fused targets); a
  // stage's plan keeps its kernels inside the chunk's local qubits
  uint64_t exec_limit = ~0ull;
  LearnedCost* learned = nullptr;  // set while planning with QS_COST_LEARNED
  uint64_t dp_states = 0;
  std::mutex mu;
  std::deque<DeviceCache> dev;  // one per device the plan ran on; adding one moves no other
};

// ---- planner (planner.cpp) --------------------------------------------------
// What a kernel's cost depends on: its qubits, non-insular qubits, gate
// counts per type, insular-gate count and gate count (and, for the analytic
// model, the sum of per-gate costs).
struct KStat {
  uint64_t q = 0, ni = 0;
  uint16_t cnt[QS_NUM_GATE_TYPES] = {};
  uint16_t nins = 0, ng = 0;
  double gcost = 0;
  void add(const Gate& g, double gc) {
    q |= g.qmask;
    ni |= g.nimask;
    if (cnt[g.type] < 0xFFFF) cnt[g.type]++;
    if ((g.qmask & ~g.nimask) && nins < 0xFFFF) nins++;
    if (ng < 0xFFFF) ng++;
    gcost += gc;
  }
  void merge(const KStat& o) {
    q |= o.q;
    ni |= o.ni;
    for (int t = 0; t < QS_NUM_GATE_TYPES; ++t) cnt[t] = (uint16_t)std::min(0xFFFF, cnt[t] + o.cnt[t]);
    nins = (uint16_t)std::min(0xFFFF, nins + o.nins);
    ng = (uint16_t)std::min(0xFFFF, ng + o.ng);
    gcost += o.gcost;
  }
};

struct CostModel {
  const PlanImpl* plan;
  LearnedCost* learned = nullptr;
  double fusion(const KStat& s) const;  // INF if infeasible
  double shm(const KStat& s) const;     // INF if infeasible
  double gate_cost(int type) const { return plan->cost.gate_cost[type]; }
  // batches the learned predictions of these kernels (no-op for analytic)
  void prefetch(const std::vector<std::pair<KStat, bool>>& ks) const;
  // Runs f (which evaluates costs) with unknown learned predictions read as
  // infeasible and recorded, then predicts the recorded ones in one batch;
  // repeats until f needs nothing new (at most `rounds` times).  No-op for
  // the analytic model.
  template <class F>
  void discover(F&& f, int rounds = 8) const {
    if (!learned) return;
    for (int r = 0; r < rounds; ++r) {
      learned_collect_begin(learned);
      f();
      if (!learned_collect_end(learned)) break;
    }
  }
};
// learned.cpp
LearnedCost* learned_create(const PlanImpl* p, qs_mlp* mlp, int* status);
void learned_destroy(LearnedCost* lc);
double learned_cost(LearnedCost* lc, const KStat& s, bool fusion);
void learned_prefetch(LearnedCost* lc, const std::vector<std::pair<KStat, bool>>& ks);
int learned_status(const LearnedCost* lc);
uint64_t widen_mask(uint64_t mask, int n, int want);
void kernel_features(int n, const KStat& s, bool fusion, uint64_t exec_mask, float* out);
int plan_kernels(PlanImpl* p);         // fills p->kernels
int compile_programs(PlanImpl* p);     // fills p->shm / p->fused
int validate_plan(const PlanImpl* p);  // Theorem 2 check

// ---- staging (stager.cpp) ---------------------------------------------------
// One stage of a staged plan (Alg. 1, Partition/Execute): a set of gates whose
// non-insular qubits are all in `local` (Sec. 4), executed chunk by chunk.
// A chunk holds the 2^L amplitudes that share one value of the regional
// (non-local) qubits; on the GPU its index bits are the local qubits in
// ascending order, so the stage's gates are relabelled by `pos` and planned
// as an n-qubit circuit whose kernels stay in positions < L, with the
// chunk's regional bits known (positions L..n-1, ascending).
struct Stage {
  uint64_t local = 0;            // logical qubits held on the GPU
  std::vector<int32_t> gates;    // circuit indices, execution order
  std::vector<int32_t> pos;      // logical qubit -> position in the chunked view
  std::vector<int32_t> order;    // position -> logical qubit (inverse of pos)
  int run_log = 0;               // local qubits 0..run_log-1: contiguous host runs
  std::unique_ptr<PlanImpl> plan;
  // X gates on regional qubits (qs_plan_opts.insular_x): circuit indices of
  // the X gates the stage executes as a relabelling, and the regional
  // qubits flipped at its end (chunk c is written back to host chunk c ^ frame)
  std::vector<int32_t> flips;
  uint64_t frame = 0;
  // per gate of the stage's own plan: its circuit index, -1 for the extra
  // gates of a conjugated gate and for the closing phase gates
  std::vector<int32_t> src;
};
// local qubits the stager may choose freely; the rest, L - kStageSlots
// lowest qubits, stay local in every stage so host runs are 2^(L-8) long
constexpr int kStageSlots = 8;
constexpr int kMinLocalQubits = 12;  // a chunk holds a 2^12 tile and a tensor-core kernel
constexpr int kMaxChunkBuffers = 4;  // chunks in flight: copy-in, kernels, copy-out, slack
constexpr uint64_t kMaxHostTimerRecords = 1ull << 16;  // stages x chunks of a timed host run
constexpr int64_t kDefaultStagerBudget = 1ll << 28;  // gate visits of the exact stager
// Stages the circuit (QS_STAGER_BEAM or QS_STAGER_EXACT); *optimal: 1 when
// the exact search proved the fewest stages, 2 when also the least objective.
int stage_circuit(const std::vector<Gate>& gates, int n, int L, int stager, int64_t budget,
                  std::vector<Stage>* out, int* optimal);
int staging_objective(const std::vector<uint64_t>& sets);

// ---- device side (kernels_*.cu) ----------------------------------------------
struct ShmLaunch {
  float2* psi;
  uint64_t hi = 0;  // known bits of qubits above n (chunked execution)
  int n, m;
  int act[kMaxShmActive];
  const DevOp* ops;
  int nops;
};
int launch_shm(const ShmLaunch& a, cudaStream_t s);

struct ShmV2Launch {
  float2* psi;
  uint64_t hi = 0;
  int n;
  uint64_t amask;
  const uint32_t* prog;      // device copy of pg->prog
  const ShmProgramV2* pg;
};
int launch_shm_v2(const ShmV2Launch& a, cudaStream_t s);
bool compile_shm_v2(const PlanImpl* p, const Kernel& K, const ShmProgram& sp, ShmProgramV2* out);
void fold_global_phase(std::vector<ShmProgramV2>& progs);
int jit_compile_plan(PlanImpl* p);                 // jit.cpp
bool jit_source(const ShmProgramV2& pg, int n, const std::string& name, std::string* out);
// batch-load form, dynamic shared memory (bytes) and launch-bound CTAs per SM
// of a program's specialised kernel
void jit_shape(const ShmProgramV2& pg, int* form, int* smem, int* min_blocks);
// blocks_per_sm: resident CTAs of the kernel per SM (the grid is that many
// per SM, so the grid-stride loop has no partial last wave)
int launch_jit(cudaKernel_t k, const ShmProgramV2& pg, int blocks_per_sm, float2* psi, int n, uint64_t hi,
               cudaStream_t s);

struct FusedLaunch {
  float2* psi;
  int n, k;
  int targets[kMaxFuse];
  const float2* u;  // device, 2^k x 2^k
  int precision;
};
int launch_fused(const FusedLaunch& a, cudaStream_t s);
constexpr int kTcTargets = 6;  // width of the tensor-core fused kernel
constexpr size_t tc_weight_floats(bool x3) { return size_t(x3 ? 2 : 1) * 128 * 128; }
void tc_prepare_weights(const float* u, bool x3, std::vector<float>* out);
void tc_prepare_weights_into(const float* u, bool x3, float* out);  // tc_weight_floats(x3) floats
// QS_ETIMEDOUT if a tensor-core kernel's bounded wait expired in work queued
// on s before this call (synchronises s); clear resets the flag.
int tc_check_error(cudaStream_t s, bool clear);
void tc_set_stall(uint64_t ns);  // test-only fault injection (qs_debug_tc_stall)
// tensor-core load paths: register gathers with 32-bit offsets, bulk row
// copies (rows in many 2 MiB pages), register gathers with 64-bit offsets,
// cp.async into a raw ring
enum TcVariant { kTcRegister = 0, kTcBulk = 1, kTcWide = 2, kTcCpAsync = 3, kTcVariants = 4 };
void tc_launch_counts(uint64_t* out, int cap);
// U (2^k x 2^k, row-major complex64) widened to 2^kw x 2^kw as U (x) I on
// kw - k added index bits above bit k-1; out: 2 * 4^kw floats.
void widen_unitary(const float* u, int k, int kw, float* out);
// targets[k .. kw-1] := the lowest qubits below n not in targets[0 .. k-1]
void widen_targets(int n, int k, int kw, int* targets);

int launch_set_zero(float2* psi, int n, cudaStream_t s);
int launch_norm2(const float2* psi, int n, double* out_host, cudaStream_t s);
int launch_compare(const float2* psi, const double2* ref, int n, double* fid,
                   double* maxabs, cudaStream_t s);
int launch_remap(const float2* in, float2* out, int n, const int32_t* perm, cudaStream_t s);

int cuda_status(cudaError_t e);  // records the message, maps to QS_ECUDA
void set_cuda_error(const char* what, cudaError_t e);

}  // namespace qs

struct qs_plan {
  qs::PlanImpl impl;  // staged plans: the gates and the flattened kernel list
  std::vector<qs::Stage> stages;  // empty unless local_qubits < n
  int staging_optimal = 0;  // 1: fewest stages proven, 2: and the least objective
  std::vector<std::pair<int32_t, int32_t>> kmap;  // flattened kernel -> (stage, kernel)
};
struct qs_state {
  int n = 0;
  float2* psi = nullptr;
  bool owned = false;
};
