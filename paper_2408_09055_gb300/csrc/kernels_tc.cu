// Fused kernels on the 5th-generation tensor cores (tcgen05, sm_103a):
// TF32 and split-precision 3xTF32 (Sec. 6.2 "Fusion" kernels: the product of
// a kernel's gates applied as one dense unitary).
//
// The complex 2^6 x 2^6 unitary U = Ur + i Ui becomes the real 128 x 128 block
// matrix W = [[Ur, -Ui], [Ui, Ur]] (the A operand).  A tile of the state --
// 64 target rows by N columns (the lowest non-target qubits) -- becomes the
// real 128 x N matrix [Re X; Im X] (the B operand), and D = W B lands in
// tensor memory as fp32.  For 3xTF32, W = Wh + Wl is split on the host and
// B = Bh + Bl on the device (Bh = B rounded to TF32, Bl = B - Bh), and
// D = Wh Bh + Wh Bl + Wl Bh recovers close to FP32 accuracy (Markidis et al.
// 2018; Ootomo and Yokota 2022).
//
// Shared-memory operands use the K-major, no-swizzle canonical layout: core
// matrices of 8 rows x 16 bytes (4 TF32), adjacent along K 128 B apart
// (leading byte offset) and along M/N (K/4)*128 B apart (stride byte offset).
// One thread issues the MMAs; completion is signalled by tcgen05.commit on an
// mbarrier whose wait is bounded in time (an expired wait sets an error flag,
// the CTA frees its tensor memory and returns).
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "internal.hpp"

namespace qs {

namespace {

constexpr int kTcK = 6;                // target qubits handled by the kernel
constexpr int kTcDim = 1 << kTcK;      // 64 complex rows
constexpr int kTcKR = 2 * kTcDim;      // 128: the real block's M = K
constexpr int kTcThreads = 256;
constexpr uint32_t kCoreStride = (kTcKR / 4) * 128;  // bytes between 8-row groups
constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s bound on an mbarrier wait

__device__ int g_tc_error;  // 1 after a bounded wait expired

struct TcParams {
  float2* psi;
  const float* w;  // W (hi, then lo for 3xTF32) in the core layout
  int n;
  uint64_t fixed;  // target and column qubits
  int8_t targets[kTcK];
  int8_t cols[8];
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

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n"
      :
      : "r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(acc)
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

// Waits for the mbarrier phase `parity`; false if the bound expired.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
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
    if (global_ns() - t0 > kWaitNs) return false;
  }
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

template <int CB, bool X3>
__global__ void __launch_bounds__(kTcThreads, X3 ? 1 : 2) fused_tc_kernel(const __grid_constant__ TcParams P) {
  constexpr int N = 1 << CB;
  constexpr uint32_t A_FLOATS = kTcKR * kTcKR;
  constexpr uint32_t B_FLOATS = N * kTcKR;
  constexpr int DP = N + 1;  // padded pitch of the output staging tile
  extern __shared__ __align__(1024) float smem[];
  float* Ah = smem;
  float* Al = smem + A_FLOATS;  // used with X3
  float* Bh = smem + (X3 ? 2 : 1) * A_FLOATS;
  float* Bl = Bh + B_FLOATS;    // used with X3
  float* Dsm = Bh;              // output staging reuses the B region
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_all;
  __shared__ unsigned long long rowoff[kTcDim];
  __shared__ unsigned long long coloff[N];
  const int tid = threadIdx.x, warp = tid >> 5;

  {  // unitary (host-arranged in the core layout) into shared memory
    const float4* src = reinterpret_cast<const float4*>(P.w);
    float4* dst = reinterpret_cast<float4*>(Ah);
    for (uint32_t i = tid; i < (X3 ? 2 : 1) * A_FLOATS / 4; i += kTcThreads) dst[i] = src[i];
  }
  for (int r = tid; r < kTcDim; r += kTcThreads) {
    unsigned long long o = 0;
    for (int j = 0; j < kTcK; ++j)
      if ((r >> j) & 1) o |= 1ull << P.targets[j];
    rowoff[r] = o;
  }
  for (int c = tid; c < N; c += kTcThreads) {
    unsigned long long o = 0;
    for (int j = 0; j < CB; ++j)
      if ((c >> j) & 1) o |= 1ull << P.cols[j];
    coloff[c] = o;
  }
  const uint32_t mb = smem_u32(&mbar);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb) : "memory");
    abort_all = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base)),
                 "r"((uint32_t)N)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  uint32_t parity = 0;
  const uint64_t nb = 1ull << (P.n - kTcK - CB);
  constexpr int E = kTcDim * N / kTcThreads;  // tile elements per thread
  const int lane = tid & 31;
  auto tile_base = [&](uint64_t bt) {
    uint64_t base = 0, x = bt;
    for (int q = 0; q < P.n && x; ++q)
      if (!((P.fixed >> q) & 1ull)) {
        base |= (x & 1ull) << q;
        x >>= 1;
      }
    return base;
  };
  // element i of this thread: column c, row j (8 consecutive columns x 4 rows
  // per warp access: 64-byte global runs, conflict-free operand stores)
  auto elem = [&](int i, int& c, int& j) {
    const int wq = (tid >> 5) + (kTcThreads / 32) * i;
    c = (lane & 7) + 8 * (wq % (N / 8));
    j = (lane >> 3) + 4 * (wq / (N / 8));
  };
  float2 v[E];
  auto load_tile = [&](uint64_t base) {
#pragma unroll
    for (int i = 0; i < E; ++i) {
      int c, j;
      elem(i, c, j);
      v[i] = P.psi[base | rowoff[j] | coloff[c]];
    }
  };
  // registers -> B operand (real block rows: Re 0..63, Im 64..127), then MMAs
  auto stage_and_issue = [&]() {
#pragma unroll
    for (int i = 0; i < E; ++i) {
      int c, j;
      elem(i, c, j);
      const uint32_t ore = core_off(c, j) >> 2, oim = core_off(c, j + kTcDim) >> 2;
      const float hr = tf32_rna(v[i].x), hi = tf32_rna(v[i].y);
      Bh[ore] = hr;
      Bh[oim] = hi;
      if (X3) {
        Bl[ore] = v[i].x - hr;
        Bl[oim] = v[i].y - hi;
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      constexpr uint32_t ID = idesc_tf32<N>();
      const uint32_t ah = smem_u32(Ah), al = smem_u32(Al), bh = smem_u32(Bh), bl = smem_u32(Bl);
#pragma unroll 1
      for (int s = 0; s < kTcKR / 8; ++s) {  // K = 8 per instruction: two core matrices
        const uint32_t ks = (uint32_t)s * 256u;
        mma_tf32(tmem, smem_desc(ah + ks), smem_desc(bh + ks), ID, s > 0);
        if (X3) {
          mma_tf32(tmem, smem_desc(ah + ks), smem_desc(bl + ks), ID, 1);
          mma_tf32(tmem, smem_desc(al + ks), smem_desc(bh + ks), ID, 1);
        }
      }
      mma_commit(mb);
    }
  };
  uint64_t bt = blockIdx.x;
  uint64_t base = 0;
  if (bt < nb) {
    base = tile_base(bt);
    load_tile(base);
    stage_and_issue();
  }
  for (; bt < nb; bt += gridDim.x) {
    // loads of the next tile are in flight while this tile's MMAs finish and
    // its accumulator drains
    const uint64_t nxt = bt + gridDim.x;
    uint64_t nbase = 0;
    if (nxt < nb) {
      nbase = tile_base(nxt);
      load_tile(nbase);
    }
    const bool ok = mbar_wait(mb, parity);
    parity ^= 1u;
    if (!ok) abort_all = 1;
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (abort_all) {
      if (tid == 0) atomicExch(&g_tc_error, 1);
      break;
    }
    {  // accumulator (row = TMEM lane) -> staging tile; warps w and w+4 share lanes
      const int lane_base = 32 * (warp & 3);
      const int row = lane_base + lane;
      const int c0 = (warp >> 2) * (N / 2);
#pragma unroll 1
      for (int cc = 0; cc < N / 2; cc += 16) {
        uint32_t r[16];
        tmem_ld16(tmem + ((uint32_t)lane_base << 16) + (uint32_t)(c0 + cc), r);
#pragma unroll
        for (int i = 0; i < 16; ++i) Dsm[row * DP + c0 + cc + i] = __uint_as_float(r[i]);
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    for (int e = tid; e < kTcDim * N; e += kTcThreads) {
      const int c = e & (N - 1), j = e >> CB;
      P.psi[base | rowoff[j] | coloff[c]] = make_float2(Dsm[j * DP + c], Dsm[(j + kTcDim) * DP + c]);
    }
    __syncthreads();  // the staging tile (B region) is free again
    if (nxt < nb) {
      base = nbase;
      stage_and_issue();
    }
  }
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)N)
                 : "memory");
}

template <int CB, bool X3>
constexpr size_t tc_smem() {
  constexpr size_t N = size_t(1) << CB;
  constexpr size_t a = (X3 ? 2 : 1) * size_t(kTcKR) * kTcKR * 4;
  constexpr size_t b = (X3 ? 2 : 1) * N * kTcKR * 4;
  constexpr size_t d = size_t(kTcKR) * (N + 1) * 4;
  return a + (b > d ? b : d);
}

template <int CB, bool X3>
int launch_tc(const TcParams& P, cudaStream_t s) {
  static unsigned attr_done = 0;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  constexpr size_t smem = tc_smem<CB, X3>();
  static_assert(smem <= 227u * 1024u - 4096u, "tensor-core tile exceeds shared memory");
  if (dev >= 32 || !((attr_done >> dev) & 1u)) {
    cudaError_t e = cudaFuncSetAttribute(fused_tc_kernel<CB, X3>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_status(e);
    if (dev < 32) attr_done |= 1u << dev;
  }
  const uint64_t nb = 1ull << (P.n - kTcK - CB);
  const int per_sm = (2 * (smem + 4096) <= 228u * 1024u) ? 2 : 1;
  const uint64_t grid = std::min<uint64_t>(nb, (uint64_t)sms * per_sm);
  fused_tc_kernel<CB, X3><<<(unsigned)grid, kTcThreads, smem, s>>>(P);
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

// W for a 2^6 x 2^6 complex unitary (row-major complex64), arranged in the
// kernel's shared-memory layout: hi part, then (3xTF32) lo part.
void tc_prepare_weights(const float* u, bool x3, std::vector<float>* out) {
  const int D = kTcDim, R = kTcKR;
  out->assign((x3 ? 2 : 1) * R * R, 0.0f);
  for (int m = 0; m < R; ++m)
    for (int kk = 0; kk < R; ++kk) {
      const int r = m & (D - 1), c = kk & (D - 1);
      const float ur = u[2 * (r * D + c)], ui = u[2 * (r * D + c) + 1];
      float w;
      if (m < D) w = kk < D ? ur : -ui;
      else w = kk < D ? ui : ur;
      const float hi = tf32_round_host(w);
      const uint32_t o = core_off((uint32_t)m, (uint32_t)kk) >> 2;
      (*out)[o] = hi;
      if (x3) (*out)[R * R + o] = tf32_round_host(w - hi);
    }
}

int tc_check_error(bool clear) {
  int v = 0;
  cudaError_t e = cudaMemcpyFromSymbol(&v, g_tc_error, sizeof(int));
  if (e != cudaSuccess) return cuda_status(e);
  if (v && clear) {
    int z = 0;
    cudaMemcpyToSymbol(g_tc_error, &z, sizeof(int));
  }
  return v ? QS_ETIMEDOUT : QS_OK;
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
  P.fixed = 0;
  for (int j = 0; j < kTcK; ++j) {
    P.targets[j] = (int8_t)a.targets[j];
    P.fixed |= 1ull << a.targets[j];
  }
  const int cb = std::min(6, a.n - kTcK);  // 64 columns per tile
  int got = 0;
  for (int q = 0; q < a.n && got < cb; ++q)
    if (!((P.fixed >> q) & 1ull)) P.cols[got++] = (int8_t)q;
  for (int j = got; j < 8; ++j) P.cols[j] = -1;
  for (int j = 0; j < cb; ++j) P.fixed |= 1ull << P.cols[j];
  if (x3) {
    if (cb == 5) return launch_tc<5, true>(P, s);
    return launch_tc<6, true>(P, s);
  }
  if (cb == 5) return launch_tc<5, false>(P, s);
  return launch_tc<6, false>(P, s);
}

}  // namespace qs
