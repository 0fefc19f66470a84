/*
 * qsim -- GB300 (sm_103a) state-vector execution of kernelized circuits.
 *
 * C ABI of libqsim.so.  Every entry point returns an int status (QS_OK = 0,
 * negative on error; qs_strerror() names it) unless stated otherwise.  No
 * C++ exception crosses this boundary and nothing aborts the process.
 * Device pointers are plain CUDA device addresses of the current device;
 * host pointers are ordinary process memory.  `stream` arguments are
 * cudaStream_t values passed as void* (NULL = the legacy default stream).
 *
 * Conventions (Sec. 2 of the paper, Eq. 1): qubit q is bit q of the
 * amplitude index; a state of n qubits is 2^n complex64 amplitudes stored
 * interleaved (re, im) as float pairs.  For a two-qubit gate, q[0] is the
 * less significant bit of its 4x4 matrix index; CX has its control on q[0].
 *
 * Threading: a qs_plan is immutable after qs_plan_circuit and may be used
 * from several threads; a qs_state must not be used concurrently.
 */
#ifndef QSIM_H_
#define QSIM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define QS_OK 0
#define QS_EINVAL (-1)       /* bad argument (size, qubit index, null pointer) */
#define QS_ENOMEM (-2)       /* device or pinned host allocation failed */
#define QS_EUNSUPPORTED (-3) /* valid request this build does not implement */
#define QS_ETIMEDOUT (-4)    /* a bounded wait ran out (host or device) */
#define QS_ECUDA (-5)        /* a CUDA runtime call failed */
#define QS_EPLAN (-6)        /* planning failed or a plan is inconsistent */

const char* qs_strerror(int status);
/* Text of the last CUDA error seen by this thread ("" if none). */
const char* qs_last_cuda_error(void);
/* Why this thread's last qs_plan_circuit call failed, e.g. the first gate
 * that fits no kernel under the options' limits ("" after a success or when
 * there is nothing to add to the status). */
const char* qs_last_error(void);

/* ---- circuit ------------------------------------------------------------
 * Gate set of the paper's benchmark workloads.  Matrices (the paper names
 * the gates without writing them; OpenQASM 2 conventions):
 *   H, X, RX(t)=exp(-i t X/2), RZ(t)=exp(-i t Z/2),
 *   U3(t,p,l)=[[cos t/2, -e^{il} sin t/2],[e^{ip} sin t/2, e^{i(p+l)} cos t/2]],
 *   CX (control q[0]), CZ, CP(t)=diag(1,1,1,e^{it}), SWAP,
 *   RXX(t)=exp(-i t X(x)X/2).
 * Insular qubits (Definition 2): RZ, CZ and CP are diagonal in all their
 * qubits; CX's control is insular.  X is treated as non-insular.          */
enum qs_gate_type {
  QS_H = 0, QS_X = 1, QS_RX = 2, QS_RZ = 3, QS_U3 = 4,
  QS_CX = 5, QS_CZ = 6, QS_CP = 7, QS_SWAP = 8, QS_RXX = 9,
  QS_NUM_GATE_TYPES = 10
};

typedef struct qs_gate {
  int32_t type;  /* enum qs_gate_type */
  int32_t nq;    /* 1 or 2; must match the type */
  int32_t q[2];  /* qubits; q[1] unused (-1) for one-qubit gates */
  double p[3];   /* angles: RX/RZ/CP/RXX use p[0]; U3 uses p[0..2] */
} qs_gate;       /* 40 bytes */

/* ---- planning (Partition / Kernelize, Sec. 4-5, Alg. 3-5) ---------------- */
enum qs_algo {
  QS_ALGO_PER_GATE = 0,  /* one kernel per gate (test baseline)                 */
  QS_ALGO_GREEDY = 1,    /* greedy packing into fusion kernels of <= fuse_kmax
                            qubits (the paper's greedy baseline, Sec. 6.4)       */
  QS_ALGO_ORDERED = 2,   /* OrderedKernelize: optimal contiguous segmentation,
                            O(|C|^2) (Alg. 5)                                    */
  QS_ALGO_KERNELIZE = 3  /* Kernelize DP over ordered kernel sets with the
                            extensible-qubit state reduction (Alg. 3, Alg. 4)
                            and the optimisations of Appendix A.2            */
};
enum qs_cost_kind { QS_COST_ANALYTIC = 0, QS_COST_LEARNED = 1 };
enum qs_precision {
  QS_PREC_FP32 = 0,   /* fused unitaries on CUDA cores, FP32                 */
  QS_PREC_TF32 = 1,   /* fused unitaries on tensor cores, one TF32 product   */
  QS_PREC_TF32X3 = 2  /* split-precision 3xTF32 on tensor cores              */
};
enum qs_kernel_type { QS_KERNEL_SHM = 0, QS_KERNEL_FUSED = 1 };
/* How a staged plan chooses its local sets (Sec. 4).  Both keep the
 * L - 8 lowest qubits local and give each stage every gate it can take. */
enum qs_stager {
  QS_STAGER_BEAM = 0,  /* beam search over local-set sequences: fewest gates
                          left, then the least objective (default)           */
  QS_STAGER_EXACT = 1  /* branch and bound from the beam's staging: the fewest
                          stages (Theorem 1), then the least objective at that
                          count -- what the ILP of Sec. 4 returns -- as far as
                          stager_budget allows; else the best staging found */
};

/* Analytic cost ("Cost Function in Kernelize"): a shared-memory kernel costs
 * alpha + sum of gate_cost[type]; a fused kernel on k qubits costs
 * fuse_cost[k].  Units are arbitrary but shared (microseconds measured on
 * the target GPU for the default table).                                    */
typedef struct qs_cost_table {
  double alpha;
  double gate_cost[QS_NUM_GATE_TYPES];
  double fuse_cost[16]; /* index = qubit count; entries above fuse_kmax unused */
} qs_cost_table;

typedef struct qs_mlp qs_mlp; /* learned cost model, see below */

enum qs_insular_x {
  QS_INSULAR_X_REWRITE = 1, /* plan the Pauli-frame rewrite of the circuit     */
  QS_INSULAR_X_STAGED = 2   /* staged plans: X on regional qubits relabels chunks */
};

typedef struct qs_plan_opts {
  int32_t algo;           /* enum qs_algo                                      */
  int32_t cost_kind;      /* enum qs_cost_kind; LEARNED needs `mlp`            */
  int32_t precision;      /* enum qs_precision of fused kernels                */
  int32_t shm_max_active; /* max |A| of a shared-memory kernel, 1..14          */
  int32_t forced_low;     /* low qubits forced into every shared-memory kernel
                             (the paper forces 3 for complex128; 4 = 128 B
                             runs of complex64)                                */
  int32_t fuse_kmin;      /* fused kernels narrower than this are widened     */
  int32_t fuse_kmax;      /* widest fused kernel; 0 disables fusion            */
  int32_t prune_T;        /* Kernelize pruning threshold T (<= 0: no pruning;
                             a DP frontier above 2^20 states then makes
                             qs_plan_circuit return QS_ENOMEM)              */
  int32_t attach_single;  /* Kernelize: attach one-qubit gates to neighbours   */
  int32_t local_qubits;   /* L: qubits resident on the GPU per chunk (0 or >= n:
                             no staging).  With 12 <= L < n the circuit is
                             staged (Alg. 1's Stage, Sec. 4): each stage holds
                             L local qubits, containing every non-insular
                             qubit of its gates, and runs chunk by chunk
                             through qs_run_plan_host.  L must also be >=
                             shm_max_active and >= forced_low + 2.          */
  int32_t shm_variant;    /* shared-memory kernel: 0 auto (specialised if it
                             compiles, else interpreted, else generic),
                             1 generic tile kernel, 2 register-phased
                             interpreter, 3 register-phased kernel specialised
                             per plan (NVRTC, sm_103a).  2 and 3 make
                             qs_plan_circuit return QS_EUNSUPPORTED when a
                             kernel has no register-phased form (a tile below
                             2^10, an active qubit above 31), 3 also when a
                             kernel fails to compile                        */
  const qs_cost_table* cost; /* NULL: built-in table                           */
  const qs_mlp* mlp;         /* learned cost model (cost_kind = LEARNED)        */
  int64_t stager_budget;  /* QS_STAGER_EXACT: work limit in gate visits
                             (<= 0: 2^28, about a second)                     */
  int32_t stager;         /* enum qs_stager (staged plans only)                */
  int32_t insular_x;      /* bit mask; X is insular (Definition 2: anti-
                             diagonal).  QS_INSULAR_X_REWRITE: the circuit
                             is planned as its Pauli-frame rewrite
                             (qs_insular_x_rewrite): every X moves to the
                             end, flipping the controls and diagonal factors
                             it passes (App. A.2), so no X needs an active
                             qubit before the last kernels; kernel gate
                             indices refer to the rewritten circuit.
                             QS_INSULAR_X_STAGED (staged plans): an X on a
                             regional qubit is a relabelling of the stage's
                             chunks -- the stage's later controls and
                             diagonal factors on it are conjugated, and chunk
                             c is written back to host chunk c ^ (the
                             flipped qubits), which needs >= 2 chunk buffers.
                             0: X is non-insular.                           */
} qs_plan_opts;

/* Fills `opts` with the defaults (Kernelize, analytic cost, FP32, |A| <= 13,
 * 4 forced low qubits, fused k in [1, 6], T = 500, attach on, L = n, beam
 * stager).                                                                  */
void qs_plan_opts_default(qs_plan_opts* opts);
/* The built-in analytic cost table. */
void qs_cost_table_default(qs_cost_table* out);

typedef struct qs_plan qs_plan;

/* Partition + Kernelize a circuit of `ngates` gates on `n` qubits (1..40).
 * The gate array is copied; the plan is owned by the caller and released
 * with qs_plan_free.  Errors: QS_EINVAL (bad gate, qubit or option),
 * QS_EPLAN (a gate fits no kernel under the options' limits),
 * QS_EUNSUPPORTED (tensor-core precisions with fusion below 11 qubits or
 * above 6 targets; a forced shm_variant the plan cannot use), QS_ENOMEM.    */
int qs_plan_circuit(int32_t n, const qs_gate* gates, uint64_t ngates,
                    const qs_plan_opts* opts, qs_plan** out);
void qs_plan_free(qs_plan* plan);

typedef struct qs_plan_stats {
  int32_t n;
  int32_t num_stages;
  uint64_t num_gates;
  uint64_t num_kernels;
  uint64_t num_shm;
  uint64_t num_fused;
  double cost;        /* total model cost (Eq. 2)                           */
  double planner_ms;  /* host time spent in qs_plan_circuit                 */
  uint64_t dp_states; /* Kernelize: largest DP frontier                    */
  uint64_t num_phased;    /* shm kernels run by the register-phased kernel   */
  uint64_t num_exchanges; /* shared-memory exchanges summed over those       */
  uint64_t num_jit;       /* of those, kernels specialised per plan (NVRTC)  */
  double jit_ms;          /* host time compiling them (included in planner_ms) */
  int32_t staging_cost;   /* the objective of Sec. 4 with no global qubits:
                             qubits that become local at stage boundaries    */
  int32_t staging_optimal;/* exact stager: 1 when it proved the fewest
                             stages, 2 when also the least objective at that
                             count; 0 otherwise                              */
} qs_plan_stats;
int qs_plan_stats_get(const qs_plan* plan, qs_plan_stats* out);

typedef struct qs_kernel_desc {
  int32_t type;       /* enum qs_kernel_type                                 */
  int32_t stage;      /* stage index                                        */
  int32_t nqubits;    /* |A| (shm) or k (fused), widening included          */
  int32_t num_gates;
  uint64_t qubit_mask;/* physical qubits of A (shm) or of the fused targets;
                         in a staged plan the circuit's qubit labels, all
                         local to the kernel's stage (the stage's chunk view
                         places local qubit q at its rank in local_mask)    */
  double cost;
} qs_kernel_desc;
int qs_plan_kernel(const qs_plan* plan, uint64_t k, qs_kernel_desc* out);
/* Copies the circuit indices of kernel k's gates, in execution order, into
 * ids[0..cap); returns the count or a negative status.                     */
int64_t qs_plan_kernel_gates(const qs_plan* plan, uint64_t k, int32_t* ids, uint64_t cap);
/* The fused kernel's unitary in FP64, row-major complex interleaved,
 * 2^k x 2^k, index bit j = the j-th lowest qubit of qubit_mask.            */
int qs_plan_fused_matrix(const qs_plan* plan, uint64_t k, double* out, uint64_t cap_doubles);
/* The CUDA source of shared-memory kernel k specialised for this plan (the
 * text compiled with NVRTC), NUL-terminated into out[0..cap); returns its
 * length (excluding the NUL), or a negative status (QS_EINVAL when kernel k
 * has no specialised form).  With out == NULL only the length is returned. */
int64_t qs_plan_kernel_source(const qs_plan* plan, uint64_t k, char* out, uint64_t cap);
/* The register-phased program of shared-memory kernel k -- the words the
 * interpreter runs and the specialised kernel is generated from (opcodes and
 * operand layout in shm_program.hpp) -- for inspection and testing.  Copies
 * up to `cap` words into `words` (NULL: only the count is returned) and, when
 * `layout` is non-NULL, 20 integers into it: m, the physical qubits of the
 * m active local bits (14 entries, -1 past m), and the local bits of the 5
 * register slots in the first phase.  Staged plans report positions in the
 * stage's chunk view.  Returns the word count, or QS_EINVAL when kernel k has
 * no register-phased program (fused kernels, tiles below 2^10).            */
int64_t qs_plan_kernel_program(const qs_plan* plan, uint64_t k, uint32_t* words, uint64_t cap,
                               int32_t* layout);

/* The circuit an insular-X plan executes (qs_plan_opts.insular_x): the
 * Pauli-frame rewrite of gates[0 .. ngates).  The stored state is the
 * circuit's up to a Pauli frame prod_q Z^z X^x and a global phase: an X only
 * updates the frame; H, CX, CZ and SWAP map it; RZ, RX, RXX, U3 and CP are
 * conjugated by it (angle signs, CP's control flip with RZ factors); at the
 * end the frame is applied as X and RZ(pi) gates and the phase as
 * U3(0,0,a) X U3(0,0,a) X on qubit 0.  The result equals the circuit's state
 * exactly in exact arithmetic.  *nout = the rewritten gate count; out may be
 * NULL, else it needs cap >= *nout entries (QS_EINVAL otherwise).        */
int qs_insular_x_rewrite(int32_t n, const qs_gate* gates, uint64_t ngates, qs_gate* out, uint64_t cap,
                         uint64_t* nout);

/* Checks Theorem 2 on a plan: every gate exactly once and, for every pair of
 * gates sharing a qubit that is not insular in both, circuit order kept.
 * QS_OK or QS_EPLAN.                                                        */
int qs_plan_validate(const qs_plan* plan, const qs_gate* gates, uint64_t ngates);

/* Insular X gates of a staged plan (qs_plan_opts.insular_x; App. A.2): the
 * logical regional qubits whose values the stage flips (*frame: the stage's
 * stored chunk c is written back to host chunk c with those bits flipped)
 * and the circuit indices of the X gates it executes that way, in circuit
 * order (*num_flips of them; flip_gates may be NULL, else it needs
 * cap >= *num_flips entries).  Unstaged plans: 0 and none.  QS_EINVAL for a
 * bad stage or cap.                                                          */
int qs_plan_stage_frame(const qs_plan* plan, int32_t stage, uint64_t* frame, int32_t* flip_gates,
                        int64_t cap, int64_t* num_flips);

/* Stage `stage` of a plan (0..num_stages-1; an unstaged plan has one stage
 * holding every qubit): the mask of its local qubits, its gate count and
 * the range [first_kernel, first_kernel + num_kernels) of its kernels in the
 * plan's kernel list (kernels are listed stage by stage).  Staged plans
 * (Sec. 4): a stage's gates have all their non-insular qubits local; its
 * kernels' qubit masks are logical qubits inside the local set.  Outputs
 * may be NULL.                                                              */
int qs_plan_stage(const qs_plan* plan, int32_t stage, uint64_t* local_mask, int64_t* num_gates,
                  int32_t* first_kernel, int32_t* num_kernels);

/* ---- state ---------------------------------------------------------------- */
typedef struct qs_state qs_state;

/* A state of n qubits (1..34) in device memory.  With device_ptr == NULL the
 * library allocates 2^n * 8 bytes (cudaMalloc) and frees it in
 * qs_state_free; otherwise the caller's buffer (>= 2^n * 8 bytes, 16-byte
 * aligned) is used and stays owned by the caller.  Contents are undefined
 * until qs_state_set_zero or qs_write_amplitudes.                          */
int qs_state_create(int32_t n, void* device_ptr, qs_state** out);
/* A library-owned state of n qubits (1..34) initialised to |0...0>,
 * stream-ordered on `stream` (qs_state_create + qs_state_set_zero).        */
int qs_alloc_state(int32_t n, void* stream, qs_state** out);
void qs_state_free(qs_state* st);
void* qs_state_device_ptr(const qs_state* st);
int qs_state_set_zero(qs_state* st, void* stream); /* |0...0> */

/* Applies the plan to the state, stream-ordered and asynchronous.  The first
 * call with a plan uploads its kernel programs (device allocation).  Errors
 * found asynchronously surface at the next synchronising call: qs_sync,
 * qs_read_amplitudes, qs_write_amplitudes, qs_state_norm2,
 * qs_state_compare_c128, qs_apply_fused(_static).  A tensor-core kernel
 * whose bounded wait (2 s) expired leaves its tiles unprocessed; that call
 * then returns QS_ETIMEDOUT (once: the device's flag is cleared) and the
 * state is undefined.                                                      */
int qs_run_plan(const qs_plan* plan, qs_state* st, void* stream);

/* Synchronises `stream` and reports errors of the work queued on it (and of
 * earlier tensor-core work on this device): QS_ETIMEDOUT after an expired
 * bounded wait, QS_ECUDA after a CUDA error, else QS_OK.                   */
int qs_sync(void* stream);

/* Test-only fault injection, no counterpart in the paper.  limit_us > 0:
 * every later tensor-core launch (any process thread) first waits up to
 * limit_us microseconds on an mbarrier that nothing ever signals, then gives
 * up as an expired wait does -- every role leaves its loop, TMEM is freed
 * and the CTA returns, with nothing issued to the tensor pipe -- so the
 * launch leaves the state unchanged and the next synchronising call
 * returns QS_ETIMEDOUT.  limit_us = 0 turns it off.  QS_EINVAL outside
 * 0..10^7.                                                                  */
int qs_debug_tc_stall(int64_t limit_us);

/* Test-only, no counterpart in the paper: tensor-core fused launches made so
 * far in this process, per load path: out[0] register gathers (32-bit
 * offsets), out[1] bulk row copies (cp.async.bulk; chosen when a tile's 64
 * columns are the 64 lowest qubits and five or more targets are at qubit
 * 18 or above), out[2] register gathers with 64-bit offsets (n > 32),
 * out[3] cp.async copies into a raw ring.  Writes min(cap, 4) entries;
 * returns 4 (the number of paths) or QS_EINVAL.                             */
int32_t qs_debug_tc_launch_counts(uint64_t* out, int32_t cap);

/* Alg. 1's Execute with the state in host memory: for each stage, for each
 * chunk of 2^L amplitudes that share one value of the stage's regional
 * qubits, copy the chunk to the GPU, run the stage's kernels on it (the
 * regional values are known bits of insular gates, Definition 2) and copy
 * it back.  Chunks rotate over up to 4 buffers on internal streams, so
 * copies in both directions overlap the kernels of the neighbouring chunks.
 * A chunk's copy-in waits only for the chunks of the previous stage its
 * amplitudes come from, so consecutive stages overlap at their boundary.
 *   host_state   2^n complex64 amplitudes (interleaved float pairs), updated
 *                in place; page-locked (cudaMallocHost / cudaHostRegister),
 *                16-byte aligned, else QS_EINVAL.  Caller-owned.
 *   device_buffer, buffer_bytes
 *                device scratch for min(4, buffer_bytes / (8 * 2^L)) chunk
 *                buffers (>= 1, 256-byte aligned), caller-owned; NULL: the
 *                library allocates two (one when L = n) stream-ordered for
 *                the call.
 * An unstaged plan runs as one stage with L = n (one copy each way).  The
 * call is asynchronous: work is ordered after what `stream` has queued and
 * `stream` continues after the last copy back; the host must not touch
 * host_state until then.  Errors: QS_EINVAL, QS_ECUDA, QS_ENOMEM.  After a
 * failure the host state is undefined.                                       */
int qs_run_plan_host(const qs_plan* plan, float* host_state, void* device_buffer,
                     uint64_t buffer_bytes, void* stream);

/* Timeline of one qs_run_plan_host call, from CUDA events on the internal
 * streams.  A timer holds events for every (stage, chunk) record of its
 * plan (stages x 2^(n-L) records, at most 65536, else QS_EINVAL).
 * qs_run_plan_host_timed runs like qs_run_plan_host and records, per
 * record: copy-in start, copy-in end (= kernels start), kernels end
 * (= copy-out start), copy-out end.  qs_host_timer_read synchronises and
 * writes those 4 times per record, in ms since the call started on
 * `stream`, into ms[0 .. 4*nrec) (stage-major, then chunk), and nrec.  The
 * events add a little work on the streams; timings of the untimed call are
 * those of the whole call (events around it on `stream`).                  */
typedef struct qs_host_timer qs_host_timer;
int qs_host_timer_create(const qs_plan* plan, qs_host_timer** out);
int qs_run_plan_host_timed(const qs_plan* plan, float* host_state, void* device_buffer,
                           uint64_t buffer_bytes, qs_host_timer* timer, void* stream);
int qs_host_timer_read(qs_host_timer* timer, double* ms, uint64_t cap, uint64_t* nrec);
void qs_host_timer_free(qs_host_timer* timer);

/* Per-kernel timing with CUDA events on the launching stream (used by the
 * benchmark for the roofline of each kernel type).  A timer holds
 * (num_kernels + 1) * max_runs events; qs_run_plan_timed records one event
 * before every kernel and one after the last, on `stream`.
 * qs_timer_read synchronises the events and writes, for every kernel of the
 * plan, the sum over recorded runs of its duration in ms (per_kernel_ms
 * has num_kernels entries) and the number of runs.                          */
typedef struct qs_timer qs_timer;
/* (Staged plans have no resident form: QS_EUNSUPPORTED.) */
int qs_timer_create(const qs_plan* plan, uint64_t max_runs, qs_timer** out);
int qs_run_plan_timed(const qs_plan* plan, qs_state* st, qs_timer* timer, void* stream);
int qs_timer_read(qs_timer* timer, double* per_kernel_ms, uint64_t cap, uint64_t* runs);
void qs_timer_free(qs_timer* timer);

/* Copy amplitudes [first, first+count) between the state and host memory
 * (interleaved float pairs).  Synchronises the stream; QS_ETIMEDOUT as for
 * qs_sync.                                                                  */
int qs_read_amplitudes(const qs_state* st, uint64_t first, uint64_t count,
                       float* host_out, void* stream);
int qs_write_amplitudes(qs_state* st, uint64_t first, uint64_t count,
                        const float* host_in, void* stream);

/* a8: reductions accumulated in FP64.  norm2 = sum |a_i|^2.  With a
 * reference state ref (2^n complex128, device memory, interleaved):
 * fidelity = |<ref|psi>|^2 / (<ref|ref> <psi|psi>), maxabs = max_i |ref_i -
 * psi_i|.  Synchronise the stream.                                          */
int qs_state_norm2(const qs_state* st, double* out, void* stream);
int qs_state_compare_c128(const qs_state* st, const double* ref_device,
                          double* fidelity, double* maxabs, void* stream);

/* ---- low-level device operations (each cites its step) ------------------ */

/* a6: out[pi(i)] = in[i] where pi moves bit j of i to bit perm[j]
 * (perm a permutation of 0..n-1; Alg. 1's Shard).  Out of place; in and out
 * (2^n complex64 each, device) must not overlap.  n in 1..34.  For n >= 10
 * the call allocates its 4 KiB of index tables stream-ordered on `stream`
 * and frees them after the launch.  Asynchronous.  Errors: QS_EINVAL (not a
 * permutation, overlap, bad n), QS_ECUDA.                                   */
int qs_remap(const float* in_device, float* out_device, int32_t n,
             const int32_t* perm, void* stream);

/* Applies one fused 2^k x 2^k unitary (row-major complex64 on the host,
 * index bit j = qubit targets[j]) to a device state, in the given precision.
 * A direct entry to the fused-kernel path (a5).  Tensor-core precisions
 * widen k < 6 to 6 (identity on the added qubits) and return
 * QS_EUNSUPPORTED for k > 6 or n < 11.  Errors: QS_EINVAL (bad targets,
 * k outside 1..7, n outside k..34), QS_ENOMEM, QS_ECUDA.                    */
int qs_apply_fused(float* state_device, int32_t n, const int32_t* targets,
                   int32_t k, const float* u_host, int32_t precision, void* stream);

/* ---- learned kernel-cost model (a3, a9) -----------------------------------
 * A three-layer perceptron (features -> hidden -> hidden -> 1, ReLU) that
 * predicts ln(kernel time in microseconds on a 30-qubit state) from a
 * kernel's features (qs_kernel_features).  Parameters live in device memory
 * of the current device, FP32 (layout W1[F x H], b1[H], W2[H x H], b2[H],
 * W3[H], b3[1], row-major).  Training runs the library's FP32-accumulate
 * forward, backpropagation and Adam kernels; inference can use the BF16
 * copy of the weights (BF16 activations, FP32 accumulation).  With
 * qs_plan_opts.cost_kind = QS_COST_LEARNED the planners use exp(prediction)
 * scaled by 2^(n-30) as a kernel's cost (feasibility rules unchanged).     */
#define QS_MLP_FEATURES 44
int qs_mlp_create(int32_t features, int32_t hidden, uint64_t seed, qs_mlp** out);
void qs_mlp_free(qs_mlp* mlp);
int64_t qs_mlp_num_params(const qs_mlp* mlp);
int qs_mlp_shape(const qs_mlp* mlp, int32_t* features, int32_t* hidden);
int qs_mlp_get_params(const qs_mlp* mlp, float* host_out, uint64_t n);
/* Sets the parameters and resets the optimiser state. */
int qs_mlp_set_params(qs_mlp* mlp, const float* host_in, uint64_t n);
/* x: device [batch x features] FP32, t: device [batch] targets.  Gradient of
 * the mean squared error into grad_out (host, num_params floats, or NULL);
 * the loss into loss_out (host, or NULL).  Synchronises the stream.        */
int qs_mlp_gradient(qs_mlp* mlp, const float* x_device, const float* t_device, int32_t batch,
                    float* grad_out, float* loss_out, void* stream);
/* Loss of qs_mlp_gradient and qs_mlp_train_step: the expectile tau of
 * ln(time) -- weight 2 tau on samples the network underestimates, 2 (1 -
 * tau) on those it overestimates, times the squared error.  tau = 0.5 (the
 * default) is the mean squared error; tau > 0.5 trains a pessimistic model,
 * so a planner that minimises predicted cost finds fewer kernels whose cost
 * the network underestimates.  QS_EINVAL unless 0 < tau < 1.                */
int qs_mlp_set_expectile(qs_mlp* mlp, float tau);
/* One Adam step (beta 0.9 / 0.999, eps 1e-8) on the batch's gradient. */
int qs_mlp_train_step(qs_mlp* mlp, const float* x_device, const float* t_device, int32_t batch,
                      float lr, float* loss_out, void* stream);
/* y (device [batch]) = network(x); bf16 != 0 uses the BF16 weights. Async. */
int qs_mlp_forward(qs_mlp* mlp, const float* x_device, int32_t batch, float* y_device,
                   int32_t bf16, void* stream);
/* Host-side features of one kernel: bits 0..29 the kernel's qubit mask (its
 * active set for a shared-memory kernel, its targets for a fused one),
 * 30..39 gate counts per type / 16, 40 insular-gate count / 16, 41 the
 * kernel type, 42 |mask| / 16, 43 gate count / 64.  out: QS_MLP_FEATURES
 * floats.                                                                   */
int qs_kernel_features(int32_t n, const qs_gate* gates, uint64_t ngates, int32_t kernel_type,
                       uint64_t qubit_mask, float* out);

/* Allocation-free form of qs_apply_fused.  The paper has no counterpart:
 * it exists for callers that must not allocate device memory while they
 * apply a gate -- code that runs with every byte of device memory already
 * handed to another allocator or budget, or that cannot accept the
 * synchronisation and failure modes of an allocation in the middle of its
 * work.  qs_apply_fused stages what the kernel reads (the 2^k x 2^k matrix
 * for FP32; the TF32 weights prepared from it, 64 or 128 KiB, for TF32 and
 * 3xTF32) in memory it allocates on every call; this entry point stages it
 * in one fixed device array instead (128 KiB, held by every GPU that loads
 * the library until the process exits) and prepares the weights in static
 * host memory, so it calls no cudaMalloc, cudaFree or other allocating
 * routine.
 *
 * Arguments, layout and results are those of qs_apply_fused, for every
 * precision: tensor-core precisions widen k < 6 to 6 and return
 * QS_EUNSUPPORTED for k > 6 or n < 11.  Limit: k <= 7 (2^7 x 2^7 complex64
 * fills the array); a larger k returns QS_EINVAL.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  Every call on a device shares the array, which
 * keeps the last call's contents (each call overwrites all it reads);
 * calls whose work overlaps on the GPU (for example from two host threads
 * on two streams) race on it and must be serialised by the caller.
 * Synchronises the stream before returning; QS_ETIMEDOUT as for qs_sync.   */
int qs_apply_fused_static(float* state_device, int32_t n, const int32_t* targets,
                          int32_t k, const float* u_host, int32_t precision, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* QSIM_H_ */
