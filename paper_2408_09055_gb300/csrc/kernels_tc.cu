// Fused kernels on the 5th-generation tensor cores (tcgen05, sm_103a):
// TF32 and split-precision 3xTF32 (Sec. 6.2 "Fusion" kernels: the product of
// a kernel's gates applied as one dense unitary).
//
// The complex 2^6 x 2^6 unitary U = Ur + i Ui becomes a real 128 x 128 matrix
// W (the A operand, held in tensor memory for the whole launch): its rows and
// columns interleave real and imaginary parts, so W (Re x0, Im x0, Re x1, ...)
// = (Re y0, Im y0, ...) for y = U x.  A tile of the state -- 64 target rows by
// N columns (the lowest non-target qubits) -- is the real 128 x N B operand
// in shared memory, and D = W B lands in tensor memory as fp32.  For 3xTF32,
// W = Wh + Wl is split on the host and B = Bh + Bl on the device (Bh = B
// rounded to TF32, Bl = B - Bh), and D = Wh Bh + Wh Bl + Wl Bh recovers close
// to FP32 accuracy (Markidis et al. 2018; Ootomo and Yokota 2022).
//
// The B operand uses the K-major, no-swizzle canonical layout: core matrices
// of 8 rows x 16 bytes (4 TF32), adjacent along K 128 B apart (leading byte
// offset) and along N (K/4)*128 B apart (stride byte offset).  One thread
// issues the MMAs; completion is signalled by tcgen05.commit on mbarriers
// whose waits are bounded in time (an expired wait sets an error flag, every
// role leaves its loop, in-flight operations are waited for, tensor memory
// is freed and the CTA returns).
#include <atomic>
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <type_traits>
#include <vector>

#include "internal.hpp"

namespace qs {

namespace {

constexpr int kTcK = 6;                // target qubits handled by the kernel
constexpr int kTcDim = 1 << kTcK;      // 64 complex rows
constexpr int kTcKR = 2 * kTcDim;      // 128: the real block's M = K
constexpr uint32_t kCoreStride = (kTcKR / 4) * 128;  // bytes between 8-row groups
constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s bound on an mbarrier wait

__device__ int g_tc_error;  // 1 after a bounded wait expired

struct TcParams {
  float2* psi;
  const float* w;  // W (hi, then lo for 3xTF32) in the core layout
  int n;
  int contig;      // the column qubits are 0..CB-1: output rows are contiguous
  uint64_t fixed;  // target and column qubits
  int8_t targets[kTcK];
  int8_t cols[8];
  // fault injection for tests: > 0 makes the MMA thread first wait this
  // many ns on a barrier that nothing signals, so the launch gives up
  uint64_t stall_ns;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((128u >> 4) & 0x3FFFu) << 16;          // leading byte offset (K)
  d |= (uint64_t)((kCoreStride >> 4) & 0x3FFFu) << 32;   // stride byte offset (M/N)
  d |= 1ull << 46;                                       // fixed 0b001 at bits 46..48
  return d;                                              // base offset 0, no swizzle
}

template <int N>
__host__ __device__ constexpr uint32_t idesc_tf32() {
  return (1u << 4)        // D: fp32
         | (2u << 7)      // A: tf32
         | (2u << 10)     // B: tf32
         | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(kTcKR >> 4) << 24);  // K-major A and B
}

// D (+)= A B with A read from tensor memory (M = 128 lanes, K along columns)
__device__ __forceinline__ void mma_tf32_ta(uint32_t d_tmem, uint32_t a_tmem, uint64_t b, uint32_t idesc,
                                            uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}\n"
      :
      : "r"(d_tmem), "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

// 32 consecutive columns of this warp's 32 lanes, one lane per thread
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
      "%13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, "
      "%32};"
      :
      : "r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
        "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]),
        "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]),
        "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
               :
               : "r"(mbar)
               : "memory");
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// byte offset of element (row m, k index kk) of a K-major core-matrix operand
__host__ __device__ constexpr uint32_t core_off(uint32_t m, uint32_t kk) {
  return (m >> 3) * kCoreStride + (kk >> 2) * 128u + (m & 7u) * 16u + (kk & 3u) * 4u;
}

__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}

// Bounded wait that also gives up when another role has aborted.
__device__ __forceinline__ bool mbar_wait_or_abort(uint32_t mbar, uint32_t parity, volatile int* abort_flag) {
  const unsigned long long t0 = global_ns();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
    if (*abort_flag || global_ns() - t0 > kWaitNs) return false;
  }
}

// Persistent, warp-specialised kernel.  Rows and columns of the real block
// operands are ordered (re, im)-interleaved: K index 2j + r multiplies the
// real (r = 0) or imaginary (r = 1) part of input row j, and M index 2j' + r'
// produces the real or imaginary part of output row j'.  So a float2
// amplitude is one 8-byte operand store, and output lanes 2j', 2j'+1 of a
// warp hold one complex row.
//   warps 0..7   producers: gather a tile (the next one's loads in flight),
//                round to TF32 (hi, and lo for 3xTF32) into a ring of ST
//                shared-memory stages;
//   warps 8..11  drain: TMEM accumulator -> registers -> global (one warp
//                per TMEM lane quadrant);
//   warp 12      one thread issues the MMAs into two TMEM accumulators;
//   warp 13      (BULK) loader: each tile row -- the N column qubits are the
//                lowest qubits, so a row is N contiguous amplitudes -- is one
//                cp.async.bulk into a ring of RS raw stages (rows padded to
//                keep the producers' reads conflict-free); the producers then
//                read the raw stage instead of global memory, and no register
//                holds data in flight.
constexpr int kProdWarps = 8;
constexpr int kDrainWarps = 4;

__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}

// one contiguous global run into shared memory, completing on an mbarrier
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(dst), "l"(src), "r"(bytes), "r"(mbar)
               : "memory");
}

template <int CB, bool X3, int ST, bool WIDE, bool BULK, int RS, bool CPA = false, int PW = kProdWarps, int NB = 2>
__global__ void __launch_bounds__(32 * (PW + kDrainWarps + 1) + 32, 1)
    fused_tc_kernel(const __grid_constant__ TcParams P) {
  using Off = typename std::conditional<WIDE, uint64_t, uint32_t>::type;  // amplitude offsets
  constexpr int RAW_PITCH = (1 << CB) + 8;      // float2 per raw row (64 B of padding)
  constexpr int RAW_STAGE = kTcDim * RAW_PITCH;  // float2 per raw stage
  constexpr int N = 1 << CB;
  constexpr int NOP = X3 ? 2 : 1;
  constexpr uint32_t A_FLOATS = kTcKR * kTcKR;
  constexpr uint32_t B_FLOATS = N * kTcKR;
  constexpr int TASKS = (N / 8) * (kTcDim / 4);  // warp accesses per tile: 8 columns x 4 rows
  static_assert(TASKS % PW == 0 && NB >= 2, "producer split");
  constexpr int EPT = TASKS / PW;                // per producer thread
  // tensor memory: A (hi, then lo) in columns [0, 128*NOP), two accumulators after it
  constexpr uint32_t ACC0 = kTcKR * NOP;
  constexpr uint32_t TMEM_COLS = (ACC0 + 2 * N) <= 256 ? 256 : 512;
  extern __shared__ __align__(1024) float smem[];
  float* Bop = smem;  // stage s: hi at s*NOP*B_FLOATS, lo after it
  float2* Raw = reinterpret_cast<float2*>(smem + ST * NOP * B_FLOATS);  // BULK raw ring
  __shared__ __align__(8) uint64_t bar_full[ST], bar_empty[ST], bar_accf[2], bar_acce[2], bar_fin;
  __shared__ __align__(8) uint64_t bar_rfull[RS], bar_rempty[RS], bar_never;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_all;
  __shared__ unsigned long long rowoff[kTcDim];
  __shared__ unsigned long long coloff[N];
  // runs of non-fixed qubits: tile index bits [src, src+len) go to [dst, dst+len)
  __shared__ uint8_t run_src[24], run_dst[24], run_len[24];
  __shared__ int nruns;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    int nr = 0, src = 0;
    for (int q = 0; q < P.n;) {
      if ((P.fixed >> q) & 1ull) {
        ++q;
        continue;
      }
      int len = 0;
      while (q + len < P.n && !((P.fixed >> (q + len)) & 1ull)) ++len;
      run_src[nr] = (uint8_t)src;
      run_dst[nr] = (uint8_t)q;
      run_len[nr] = (uint8_t)len;
      ++nr;
      src += len;
      q += len;
    }
    nruns = nr;
  }
  for (int r = tid; r < kTcDim; r += (int)blockDim.x) {
    unsigned long long o = 0;
    for (int j = 0; j < kTcK; ++j)
      if ((r >> j) & 1) o |= 1ull << P.targets[j];
    rowoff[r] = o;
  }
  for (int c = tid; c < N; c += (int)blockDim.x) {
    unsigned long long o = 0;
    for (int j = 0; j < CB; ++j)
      if ((c >> j) & 1) o |= 1ull << P.cols[j];
    coloff[c] = o;
  }
  if (tid == 0) {
    for (int s = 0; s < ST; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bar_full[s])),
                   "r"(32 * PW) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_empty[s])) : "memory");
    }
    for (int a = 0; a < 2; ++a) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_accf[a])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bar_acce[a])),
                   "r"(32 * kDrainWarps) : "memory");
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_fin)) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_never)) : "memory");
    for (int r = 0; r < RS; ++r) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_rfull[r])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bar_rempty[r])),
                   "r"(32 * PW) : "memory");
    }
    abort_all = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  if (warp < 4) {  // the unitary (row m = TMEM lane m, K along columns), once per CTA
    const int m = 32 * warp + lane;
#pragma unroll 1
    for (int h = 0; h < NOP; ++h)
#pragma unroll 1
      for (int c0 = 0; c0 < kTcKR; c0 += 32) {
        const float4* src = reinterpret_cast<const float4*>(P.w + h * A_FLOATS + m * kTcKR + c0);
        uint32_t r[32];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const float4 x = src[i];
          r[4 * i] = __float_as_uint(x.x);
          r[4 * i + 1] = __float_as_uint(x.y);
          r[4 * i + 2] = __float_as_uint(x.z);
          r[4 * i + 3] = __float_as_uint(x.w);
        }
        tmem_st32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(h * kTcKR + c0), r);
      }
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint64_t nb = 1ull << (P.n - kTcK - CB);
  const int nr = nruns;
  const int nbl = P.n - kTcK - CB;  // tile index bits
  // Tiles are visited in bit-reversed order: the CTAs working at the same
  // time hold tiles that differ in their highest index bits, so their rows
  // spread over the whole state instead of one narrow window per row (rows
  // 2^t apart otherwise land in the same few memory channels).
  auto tile_base = [&](uint64_t bt) {
    const uint64_t x = nbl ? (__brevll(bt) >> (64 - nbl)) : 0;
    uint64_t base = 0;
    for (int r = 0; r < nr; ++r)
      base |= ((x >> run_src[r]) & ((1ull << run_len[r]) - 1ull)) << run_dst[r];
    return base;
  };
  auto fail = [&]() {
    abort_all = 1;
    atomicExch(&g_tc_error, 1);
  };

  if (CPA && warp < PW) {
    // ---- producers with cp.async: each thread copies its own elements of
    // the tiles RS - 1 ahead into its private slots of a raw ring (slot r,
    // element e at r * EPT * 256 + e * 256 + tid), waits for its own oldest
    // group, rounds and stores the operand.  No register holds data in
    // flight and no other thread reads a thread's slots.
    float2* const raw = reinterpret_cast<float2*>(smem + ST * NOP * B_FLOATS);
    const uint32_t raw_s = smem_u32(raw + tid);
    Off goff[EPT];
    uint32_t soff[EPT];
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
      const int task = warp + PW * e;
      const int c = 8 * (task % (N / 8)) + (lane & 7), j = 4 * (task / (N / 8)) + (lane >> 3);
      goff[e] = (Off)(rowoff[j] | coloff[c]);
      soff[e] = core_off((uint32_t)c, (uint32_t)(2 * j)) >> 2;
    }
    const uint64_t g = gridDim.x;
    auto issue = [&](uint64_t bt, uint32_t slot) {
      if (bt < nb) {
        const float2* src = P.psi + tile_base(bt);
#pragma unroll
        for (int e = 0; e < EPT; ++e) {
          const uint32_t dst = raw_s + (slot * (uint32_t)(EPT * 256) + (uint32_t)(e * 256)) * 8u;
          asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst),
                       "l"(__cvta_generic_to_global(src + goff[e]))
                       : "memory");
        }
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
    };
#pragma unroll
    for (int k = 0; k < RS - 1; ++k) issue(blockIdx.x + (uint64_t)k * g, (uint32_t)k);
    uint32_t it = 0;
    for (uint64_t bt = blockIdx.x; bt < nb; bt += g, ++it) {
      issue(bt + (uint64_t)(RS - 1) * g, (it + RS - 1) % RS);  // the slot tile it - 1 used
      asm volatile("cp.async.wait_group %0;" ::"n"(RS - 1) : "memory");  // this thread's tile `it`
      const float2* mine = raw + (it % RS) * (uint32_t)(EPT * 256) + tid;
      float2 v[EPT];
#pragma unroll
      for (int e = 0; e < EPT; ++e) v[e] = mine[e * 256];
      const uint32_t s2 = it % ST, ph = (it / ST) & 1u;
      const bool ok = mbar_wait_or_abort(smem_u32(&bar_empty[s2]), ph ^ 1u, &abort_all);
      if (!__all_sync(0xffffffffu, ok)) {  // the warp leaves together
        fail();
        break;
      }
      float* bh = Bop + s2 * NOP * B_FLOATS;
#pragma unroll
      for (int e = 0; e < EPT; ++e) {
        const float hr = tf32_rna(v[e].x), hi = tf32_rna(v[e].y);
        *reinterpret_cast<float2*>(bh + soff[e]) = make_float2(hr, hi);
        if (X3) *reinterpret_cast<float2*>(bh + B_FLOATS + soff[e]) = make_float2(v[e].x - hr, v[e].y - hi);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(smem_u32(&bar_full[s2]));
    }
    asm volatile("cp.async.wait_all;" ::: "memory");  // nothing in flight when the thread leaves
  } else if (BULK && warp < PW) {
    // ---- producers reading the raw ring ----
    uint32_t roff[EPT], soff[EPT];
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
      const int task = warp + PW * e;
      const int c = 8 * (task % (N / 8)) + (lane & 7), j = 4 * (task / (N / 8)) + (lane >> 3);
      roff[e] = (uint32_t)(j * RAW_PITCH + c);
      soff[e] = core_off((uint32_t)c, (uint32_t)(2 * j)) >> 2;
    }
    uint32_t it = 0;
    for (uint64_t bt = blockIdx.x; bt < nb; bt += gridDim.x, ++it) {
      const uint32_t r = it % RS, pr = (it / RS) & 1u, s = it % ST, ps = (it / ST) & 1u;
      bool ok = mbar_wait_or_abort(smem_u32(&bar_rfull[r]), pr, &abort_all);
      if (ok) ok = mbar_wait_or_abort(smem_u32(&bar_empty[s]), ps ^ 1u, &abort_all);
      if (!__all_sync(0xffffffffu, ok)) {  // the warp leaves together
        fail();
        break;
      }
      const float2* raw = Raw + r * RAW_STAGE;
      float2 v[EPT];
#pragma unroll
      for (int e = 0; e < EPT; ++e) v[e] = raw[roff[e]];
      mbar_arrive(smem_u32(&bar_rempty[r]));  // the raw stage is read
      float* bh = Bop + s * NOP * B_FLOATS;
#pragma unroll
      for (int e = 0; e < EPT; ++e) {
        const float hr = tf32_rna(v[e].x), hi = tf32_rna(v[e].y);
        *reinterpret_cast<float2*>(bh + soff[e]) = make_float2(hr, hi);
        if (X3) *reinterpret_cast<float2*>(bh + B_FLOATS + soff[e]) = make_float2(v[e].x - hr, v[e].y - hi);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(smem_u32(&bar_full[s]));
    }
  } else if (BULK && warp == PW + kDrainWarps + 1) {
    // ---- loader ----
    uint32_t it = 0;
    for (uint64_t bt = blockIdx.x; bt < nb; bt += gridDim.x, ++it) {
      const uint32_t r = it % RS, pr = (it / RS) & 1u;
      const bool ok = mbar_wait_or_abort(smem_u32(&bar_rempty[r]), pr ^ 1u, &abort_all);
      if (!__all_sync(0xffffffffu, ok)) {
        fail();
        break;
      }
      const uint32_t full = smem_u32(&bar_rfull[r]);
      if (lane == 0) mbar_expect_tx(full, (uint32_t)(kTcDim * N * 8));
      __syncwarp();
      const uint64_t base = tile_base(bt);
      const uint32_t dst = smem_u32(Raw + r * RAW_STAGE);
      for (int row = lane; row < kTcDim; row += 32)
        bulk_load(dst + (uint32_t)(row * RAW_PITCH * 8), P.psi + (base | rowoff[row]), (uint32_t)(N * 8), full);
    }
    // copies still in flight after an abort complete before the CTA exits
    if (lane == 0)
      for (uint32_t k = it > (uint32_t)RS ? it - RS : 0; k < it; ++k) {
        const uint32_t r = k % RS, pr = (k / RS) & 1u;
        const unsigned long long t0 = global_ns();
        for (;;) {
          uint32_t done;
          asm volatile(
              "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
              "selp.u32 %0, 1, 0, p;\n\t}\n"
              : "=r"(done)
              : "r"(smem_u32(&bar_rfull[r])), "r"(pr)
              : "memory");
          if (done || global_ns() - t0 > kWaitNs) break;
        }
      }
  } else if (!BULK && !CPA && warp < PW) {
    // ---- producers ----
    // NB register buffers rotate: while one tile is rounded and stored, the
    // loads of the next NB - 1 tiles are in flight
    float2 vb[NB][EPT];
    Off goff[EPT];       // element offsets inside a tile (the same for every tile)
    uint32_t soff[EPT];  // and their operand positions (floats)
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
      const int task = warp + PW * e;
      const int c = 8 * (task % (N / 8)) + (lane & 7), j = 4 * (task / (N / 8)) + (lane >> 3);
      goff[e] = (Off)(rowoff[j] | coloff[c]);
      soff[e] = core_off((uint32_t)c, (uint32_t)(2 * j)) >> 2;
    }
    auto load = [&](uint64_t bt, float2 (&v)[EPT]) {
      const float2* src = P.psi + tile_base(bt);
#pragma unroll
      for (int e = 0; e < EPT; ++e) v[e] = src[goff[e]];
    };
    // waits for stage `it`'s buffer, stores tile v into it; false to stop
    auto put = [&](uint32_t it, const float2 (&v)[EPT]) {
      const uint32_t s = it % ST, ph = (it / ST) & 1u;
      const bool ok = mbar_wait_or_abort(smem_u32(&bar_empty[s]), ph ^ 1u, &abort_all);
      if (!__all_sync(0xffffffffu, ok)) {  // the warp leaves together
        fail();
        return false;
      }
      float* bh = Bop + s * NOP * B_FLOATS;
#pragma unroll
      for (int e = 0; e < EPT; ++e) {
        const float hr = tf32_rna(v[e].x), hi = tf32_rna(v[e].y);
        *reinterpret_cast<float2*>(bh + soff[e]) = make_float2(hr, hi);
        if (X3) *reinterpret_cast<float2*>(bh + B_FLOATS + soff[e]) = make_float2(v[e].x - hr, v[e].y - hi);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(smem_u32(&bar_full[s]));
      return true;
    };
    const uint64_t g = gridDim.x;
    uint64_t bt = blockIdx.x;
    uint32_t it = 0;
#pragma unroll
    for (int k = 0; k < NB - 1; ++k)
      if (bt + (uint64_t)k * g < nb) load(bt + (uint64_t)k * g, vb[k]);
    bool go = bt < nb;
    while (go) {
#pragma unroll
      for (int k = 0; k < NB; ++k) {
        // tile bt is in vb[k]; the buffer of the tile before it is free
        const uint64_t ahead = bt + (uint64_t)(NB - 1) * g;
        if (ahead < nb) load(ahead, vb[(k + NB - 1) % NB]);
        if (!put(it, vb[k])) {
          go = false;
          break;
        }
        ++it;
        bt += g;
        if (bt >= nb) {
          go = false;
          break;
        }
      }
    }
  } else if (warp < PW + kDrainWarps) {
    // ---- drain ----
    const int q = warp & 3;  // TMEM lane quadrant of this warp
    const int jrow = 16 * q + (lane >> 1);
    const bool odd = lane & 1;
    uint32_t it = 0;
    for (uint64_t bt = blockIdx.x; bt < nb; bt += gridDim.x, ++it) {
      const uint32_t a = it & 1u, pa = (it >> 1) & 1u;
      const bool ok = mbar_wait_or_abort(smem_u32(&bar_accf[a]), pa, &abort_all);
      if (!__all_sync(0xffffffffu, ok)) {  // the warp leaves together
        fail();
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      uint32_t r[N];
#pragma unroll
      for (int cc = 0; cc < N; cc += 16) {
        uint32_t (&rr)[16] = *reinterpret_cast<uint32_t(*)[16]>(r + cc);
        tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + ACC0 + a * (uint32_t)N + (uint32_t)cc, rr);
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(smem_u32(&bar_acce[a]));
      const uint64_t rb = tile_base(bt) | rowoff[jrow];
      // columns 4g..4g+3: the even lane writes 4g, 4g+1 and the odd lane
      // 4g+2, 4g+3, each as (re, im) pairs; one shuffle per value moved
#pragma unroll
      for (int g = 0; g < N / 4; ++g) {
        const float s0 = __uint_as_float(odd ? r[4 * g] : r[4 * g + 2]);
        const float s1 = __uint_as_float(odd ? r[4 * g + 1] : r[4 * g + 3]);
        const float t0 = __shfl_xor_sync(0xffffffffu, s0, 1);
        const float t1 = __shfl_xor_sync(0xffffffffu, s1, 1);
        const int c = 4 * g + (odd ? 2 : 0);
        float2 x0, x1;
        if (!odd) {  // own: real parts; received: imaginary parts
          x0 = make_float2(__uint_as_float(r[4 * g]), t0);
          x1 = make_float2(__uint_as_float(r[4 * g + 1]), t1);
        } else {     // own: imaginary parts; received: real parts
          x0 = make_float2(t0, __uint_as_float(r[4 * g + 2]));
          x1 = make_float2(t1, __uint_as_float(r[4 * g + 3]));
        }
        if (P.contig) {
          *reinterpret_cast<float4*>(P.psi + (rb | (uint64_t)c)) = make_float4(x0.x, x0.y, x1.x, x1.y);
        } else {
          P.psi[rb | coloff[c]] = x0;
          P.psi[rb | coloff[c + 1]] = x1;
        }
      }
    }
  } else if (lane == 0) {
    // ---- MMA issue ----
    constexpr uint32_t ID = idesc_tf32<N>();
    uint32_t it = 0;
    uint64_t bt = blockIdx.x;
    if (P.stall_ns) {  // injected fault: no arrival ever completes this phase
      const unsigned long long t0 = global_ns();
      for (;;) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(smem_u32(&bar_never)), "r"(0u)
            : "memory");
        if (done) break;
        if (global_ns() - t0 > P.stall_ns) {
          fail();
          bt = nb;  // nothing is issued to the tensor pipe
          break;
        }
      }
    }
    for (; bt < nb; bt += gridDim.x, ++it) {
      const uint32_t s = it % ST, ph = (it / ST) & 1u, a = it & 1u, pa = (it >> 1) & 1u;
      if (!mbar_wait_or_abort(smem_u32(&bar_full[s]), ph, &abort_all) ||
          !mbar_wait_or_abort(smem_u32(&bar_acce[a]), pa ^ 1u, &abort_all)) {
        fail();
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t bh = smem_u32(Bop + s * NOP * B_FLOATS), bl = bh + B_FLOATS * 4u;
      const uint32_t d = tmem + ACC0 + a * (uint32_t)N;
      // a K step of 8: 8 TMEM columns of A; 256 bytes of B (+16 in the
      // descriptor's address field)
      const uint64_t dbh = smem_desc(bh), dbl = smem_desc(bl);
#pragma unroll 1
      for (int k = 0; k < kTcKR / 8; ++k) {
        const uint64_t ks = (uint64_t)k * 16u;
        const uint32_t ka = tmem + 8u * (uint32_t)k;
        mma_tf32_ta(d, ka, dbh + ks, ID, k > 0);
        if (X3) {
          mma_tf32_ta(d, ka, dbl + ks, ID, 1);
          mma_tf32_ta(d, ka + kTcKR, dbh + ks, ID, 1);
        }
      }
      mma_commit(smem_u32(&bar_empty[s]));
      mma_commit(smem_u32(&bar_accf[a]));
    }
    // every MMA issued above has completed before the accumulators are freed
    mma_commit(smem_u32(&bar_fin));
    if (!mbar_wait_or_abort(smem_u32(&bar_fin), 0, &abort_all)) {
      // aborting: still give the tensor pipe its bounded time to finish
      const unsigned long long t0 = global_ns();
      for (;;) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(smem_u32(&bar_fin)), "r"(0u)
            : "memory");
        if (done || global_ns() - t0 > kWaitNs) break;
      }
    }
  }
  __syncwarp();  // the MMA warp's other lanes wait here for lane 0
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS)
                 : "memory");
}

template <int CB, bool X3, int ST, bool BULK, int RS, bool CPA = false>
constexpr size_t tc_smem() {
  constexpr size_t N = size_t(1) << CB;
  // the operand ring (the unitary lives in TMEM), plus the raw ring with
  // BULK (padded rows) or CPA (a tile per slot)
  return (X3 ? 2 : 1) * ST * N * kTcKR * 4 + (BULK ? RS * size_t(kTcDim) * (N + 8) * 8 : 0) +
         (CPA ? RS * size_t(kTcDim) * N * 8 : 0);
}

template <int CB, bool X3, int ST, bool WIDE, bool BULK = false, int RS = 1, bool CPA = false, int PW = kProdWarps,
          int NB = 2>
int launch_tc(const TcParams& P, cudaStream_t s) {
  static std::atomic<unsigned> attr_done{0};  // one bit per device ordinal < 32
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  constexpr size_t smem = tc_smem<CB, X3, ST, BULK, RS, CPA>();
  static_assert(smem <= 227u * 1024u - 2048u, "tensor-core pipeline exceeds shared memory");
  if (dev >= 32 || !((attr_done.load() >> dev) & 1u)) {
    cudaError_t e = cudaFuncSetAttribute(fused_tc_kernel<CB, X3, ST, WIDE, BULK, RS, CPA, PW, NB>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_status(e);
    if (dev < 32) attr_done.fetch_or(1u << dev);
  }
  const uint64_t nb = 1ull << (P.n - kTcK - CB);
  const uint64_t grid = std::min<uint64_t>(nb, (uint64_t)sms);
  constexpr int threads = 32 * (PW + kDrainWarps + 1) + (BULK ? 32 : 0);
  fused_tc_kernel<CB, X3, ST, WIDE, BULK, RS, CPA, PW, NB><<<(unsigned)grid, threads, smem, s>>>(P);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_cuda_error("tensor-core fused kernel launch", e);
    return QS_ECUDA;
  }
  return QS_OK;
}

float tf32_round_host(float x) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  u += 0xFFFu + ((u >> 13) & 1u);
  u &= 0xFFFFE000u;
  float r;
  std::memcpy(&r, &u, 4);
  return r;
}

}  // namespace

// W for a 2^6 x 2^6 complex unitary (row-major complex64) as the kernel's
// tensor-memory A operand: 128 x 128 row-major, hi part, then (3xTF32) lo.
// out: tc_weight_floats(x3) floats.
void tc_prepare_weights_into(const float* u, bool x3, float* out) {
  const int D = kTcDim, R = kTcKR;
  for (int m = 0; m < R; ++m)
    for (int kk = 0; kk < R; ++kk) {
      // M index 2r + (0: real, 1: imaginary output part); K index 2c + (0:
      // real, 1: imaginary input part)
      const int r = m >> 1, c = kk >> 1;
      const float ur = u[2 * (r * D + c)], ui = u[2 * (r * D + c) + 1];
      float w;
      if (!(m & 1)) w = (kk & 1) ? -ui : ur;
      else w = (kk & 1) ? ur : ui;
      const float hi = tf32_round_host(w);
      const uint32_t o = (uint32_t)(m * R + kk);  // row-major: row m goes to TMEM lane m
      out[o] = hi;
      if (x3) out[R * R + o] = tf32_round_host(w - hi);
    }
}

void tc_prepare_weights(const float* u, bool x3, std::vector<float>* out) {
  out->assign(tc_weight_floats(x3), 0.0f);
  tc_prepare_weights_into(u, x3, out->data());
}

static std::atomic<uint64_t> g_tc_stall_ns{0};

void tc_set_stall(uint64_t ns) { g_tc_stall_ns.store(ns); }

// launches per load-path variant (TcVariant), for tests that must know which
// path ran
static std::atomic<uint64_t> g_tc_launches[kTcVariants];

void tc_launch_counts(uint64_t* out, int cap) {
  for (int v = 0; v < kTcVariants && v < cap; ++v) out[v] = g_tc_launches[v].load();
}

// Reads the device's expired-wait flag in stream order (after the work
// queued on s), clearing it when asked.  QS_ETIMEDOUT when it was set.
int tc_check_error(cudaStream_t s, bool clear) {
  int v = 0;
  cudaError_t e = cudaMemcpyFromSymbolAsync(&v, g_tc_error, sizeof(int), 0, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_status(e);
  if (v && clear) {
    const int z = 0;
    e = cudaMemcpyToSymbolAsync(g_tc_error, &z, sizeof(int), 0, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_status(e);
  }
  return v ? QS_ETIMEDOUT : QS_OK;
}

// Load form of the tiles away from the bulk and 64-bit cases: register
// gathers by eight producer warps with two buffers (default), sixteen warps
// with three buffers (QSIM_TC_LOAD=reg16), or cp.async into a raw ring
// (QSIM_TC_LOAD=cpasync).
// Measured at 30 qubits, every kernel of the 40-layer entangling circuit
// fused: register gathers 3.48 ms (TF32) / 3.87 ms (3xTF32) per launch,
// sixteen warps 4.24 / 4.42 ms, cp.async 4.53 / 4.78 ms.
static int tc_load_form() {
  static const int v = [] {
    const char* e = std::getenv("QSIM_TC_LOAD");
    if (e && std::strcmp(e, "cpasync") == 0) return 1;
    if (e && std::strcmp(e, "reg16") == 0) return 2;
    return 0;
  }();
  return v;
}

// a.u points at the prepared weights (tc_prepare_weights) in device memory
int launch_fused_tc(const FusedLaunch& a, cudaStream_t s) {
  if (a.k != kTcK) return QS_EUNSUPPORTED;
  if (a.n < kTcK + 5) return QS_EUNSUPPORTED;  // at least 32 columns per tile
  const bool x3 = a.precision == QS_PREC_TF32X3;
  TcParams P;
  P.psi = a.psi;
  P.w = reinterpret_cast<const float*>(a.u);
  P.n = a.n;
  P.stall_ns = g_tc_stall_ns.load();
  P.fixed = 0;
  for (int j = 0; j < kTcK; ++j) {
    P.targets[j] = (int8_t)a.targets[j];
    P.fixed |= 1ull << a.targets[j];
  }
  // columns: the 64 lowest non-target qubits (32 when n = 11)
  const int cb = std::min(6, a.n - kTcK);
  int got = 0;
  for (int q = 0; q < a.n && got < cb; ++q)
    if (!((P.fixed >> q) & 1ull)) P.cols[got++] = (int8_t)q;
  for (int j = got; j < 8; ++j) P.cols[j] = -1;
  P.contig = 1;
  for (int j = 0; j < cb; ++j) {
    P.fixed |= 1ull << P.cols[j];
    if (P.cols[j] != j) P.contig = 0;
  }
  int rc;
  TcVariant v;
  // Bulk-staged loads pay off only when a tile's rows lie in many different
  // 2 MiB pages (five or more targets at qubit 18 or above: 32-64 pages per
  // tile, beyond what the address translation caches hold), where they
  // measured 7.3 ms against 9.6 ms per 30-qubit launch; elsewhere the
  // register path is faster (3.1 against 4.0 ms).
  int high = 0;
  for (int j = 0; j < kTcK; ++j) high += a.targets[j] >= 18;
  if (a.n > 32) {  // amplitude offsets need 64 bits
    v = kTcWide;
    rc = x3 ? launch_tc<6, true, 3, true>(P, s) : launch_tc<6, false, 6, true>(P, s);
  } else if (P.contig && cb == 6 && high >= 5) {
    v = kTcBulk;
    rc = x3 ? launch_tc<6, true, 2, false, true, 2>(P, s) : launch_tc<6, false, 3, false, true, 3>(P, s);
  } else if (tc_load_form() == 2) {  // sixteen producer warps, three register buffers
    v = kTcRegister;
    if (x3)
      rc = cb == 5 ? launch_tc<5, true, 3, false, false, 1, false, 16, 3>(P, s)
                   : launch_tc<6, true, 3, false, false, 1, false, 16, 3>(P, s);
    else
      rc = cb == 5 ? launch_tc<5, false, 6, false, false, 1, false, 16, 3>(P, s)
                   : launch_tc<6, false, 6, false, false, 1, false, 16, 3>(P, s);
  } else if (tc_load_form() == 1) {
    v = kTcCpAsync;
    if (x3)
      rc = cb == 5 ? launch_tc<5, true, 2, false, false, 3, true>(P, s) : launch_tc<6, true, 2, false, false, 3, true>(P, s);
    else
      rc = cb == 5 ? launch_tc<5, false, 4, false, false, 3, true>(P, s) : launch_tc<6, false, 4, false, false, 3, true>(P, s);
  } else {
    v = kTcRegister;
    if (x3) rc = cb == 5 ? launch_tc<5, true, 3, false>(P, s) : launch_tc<6, true, 3, false>(P, s);
    else rc = cb == 5 ? launch_tc<5, false, 6, false>(P, s) : launch_tc<6, false, 6, false>(P, s);
  }
  if (rc == QS_OK) g_tc_launches[v].fetch_add(1);
  return rc;
}

}  // namespace qs
