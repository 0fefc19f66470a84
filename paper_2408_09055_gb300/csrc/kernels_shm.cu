// Shared-memory kernel (Sec. 5 "Cost Function in Kernelize", kernel type 2;
// Appendix A.2 "Insular qubits").
//
// One pass over the state: for every batch (fixed values of the n - m
// non-active qubits) the 2^m amplitudes of the active set A are gathered
// into shared memory, every gate of the kernel is applied there in order,
// and the tile is written back in place.  Gates whose non-active qubits are
// insular use the batch's known bit values: a control on a non-active qubit
// enables or skips the gate for the whole batch; a diagonal factor on a
// non-active qubit becomes a per-batch scalar.
#include <algorithm>

#include "internal.hpp"

namespace qs {

namespace {

constexpr int kThreads = 256;

struct ShmParams {
  float2* psi;
  const DevOp* ops;
  int nops;
  int n, m;
  uint64_t amask;  // active physical qubits
  int8_t act[kMaxShmActive];
};

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 c) {  // a*b + c
  return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, c.y)));
}

__global__ void __launch_bounds__(kThreads) shm_kernel_v1(ShmParams P) {
  extern __shared__ float2 tile[];
  __shared__ unsigned long long tab[3][32];  // local index 5-bit chunk -> physical offset
  const int tid = threadIdx.x;
  if (tid < 96) {
    int c = tid >> 5, e = tid & 31;
    unsigned long long off = 0;
    for (int b = 0; b < 5; ++b) {
      int j = 5 * c + b;
      if (j < P.m && ((e >> b) & 1)) off |= 1ull << P.act[j];
    }
    tab[c][e] = off;
  }
  __syncthreads();
  const int L = 1 << P.m;
  const uint64_t nb = 1ull << (P.n - P.m);
  for (uint64_t b = blockIdx.x; b < nb; b += gridDim.x) {
    // deposit the batch index into the non-active qubit positions
    uint64_t base = 0, x = b;
    for (int q = 0; q < P.n && x; ++q)
      if (!((P.amask >> q) & 1)) {
        base |= (x & 1ull) << q;
        x >>= 1;
      }
    for (int li = tid; li < L; li += kThreads)
      tile[li] = P.psi[base | tab[0][li & 31] | tab[1][(li >> 5) & 31] | tab[2][(li >> 10) & 31]];
    __syncthreads();
    for (int o = 0; o < P.nops; ++o) {
      const DevOp& op = P.ops[o];
      const uint64_t cg = op.cglob;
      if ((base & cg) != cg) continue;  // uniform over the block
      const uint8_t kind = op.kind;
      const uint32_t cl = op.cloc;
      if (kind == OP_DENSE1) {
        const int t = op.t0;
        const float2 u00 = make_float2(op.m[0], op.m[1]), u01 = make_float2(op.m[2], op.m[3]);
        const float2 u10 = make_float2(op.m[4], op.m[5]), u11 = make_float2(op.m[6], op.m[7]);
        for (int p = tid; p < (L >> 1); p += kThreads) {
          int i0 = ((p >> t) << (t + 1)) | (p & ((1 << t) - 1));
          if ((i0 & cl) != cl) continue;
          int i1 = i0 | (1 << t);
          float2 a = tile[i0], c = tile[i1];
          tile[i0] = cfma(u00, a, cmul(u01, c));
          tile[i1] = cfma(u10, a, cmul(u11, c));
        }
      } else if (kind == OP_DENSE2) {
        const int t0 = op.t0, t1 = op.t1;
        const int lo = min(t0, t1), hi = max(t0, t1);
        for (int p = tid; p < (L >> 2); p += kThreads) {
          int i = ((p >> lo) << (lo + 1)) | (p & ((1 << lo) - 1));
          i = ((i >> hi) << (hi + 1)) | (i & ((1 << hi) - 1));
          if ((i & cl) != cl) continue;
          int idx[4];
          float2 v[4];
#pragma unroll
          for (int s = 0; s < 4; ++s) {
            idx[s] = i | ((s & 1) << t0) | ((s >> 1) << t1);
            v[s] = tile[idx[s]];
          }
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll
            for (int s = 0; s < 4; ++s)
              acc = cfma(make_float2(op.m[2 * (4 * r + s)], op.m[2 * (4 * r + s) + 1]), v[s], acc);
            tile[idx[r]] = acc;
          }
        }
      } else {  // OP_DIAG
        const int t0 = op.t0, t1 = op.t1;
        const int gb0 = op.g0 >= 0 ? (int)((base >> op.g0) & 1) : 0;
        const int gb1 = op.g1 >= 0 ? (int)((base >> op.g1) & 1) : 0;
        float2 d[4];
#pragma unroll
        for (int s = 0; s < 4; ++s) d[s] = make_float2(op.m[2 * s], op.m[2 * s + 1]);
        for (int li = tid; li < L; li += kThreads) {
          if ((li & cl) != cl) continue;
          int b0 = t0 >= 0 ? ((li >> t0) & 1) : gb0;
          int b1 = t1 >= 0 ? ((li >> t1) & 1) : gb1;
          int s = b0 | (b1 << 1);
          float2 f = s == 0 ? d[0] : (s == 1 ? d[1] : (s == 2 ? d[2] : d[3]));
          tile[li] = cmul(tile[li], f);
        }
      }
      __syncthreads();
    }
    for (int li = tid; li < L; li += kThreads)
      P.psi[base | tab[0][li & 31] | tab[1][(li >> 5) & 31] | tab[2][(li >> 10) & 31]] = tile[li];
    __syncthreads();
  }
}

}  // namespace

int launch_shm(const ShmLaunch& a, cudaStream_t s) {
  if (a.m < 1 || a.m > kMaxShmActive || a.m > a.n) return QS_EINVAL;
  ShmParams P;
  P.psi = a.psi;
  P.ops = a.ops;
  P.nops = a.nops;
  P.n = a.n;
  P.m = a.m;
  P.amask = 0;
  for (int j = 0; j < kMaxShmActive; ++j) {
    P.act[j] = j < a.m ? (int8_t)a.act[j] : (int8_t)-1;
    if (j < a.m) P.amask |= 1ull << a.act[j];
  }
  const size_t smem = sizeof(float2) << a.m;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  static unsigned attr_done = 0;  // one bit per device ordinal < 32
  if (dev >= 32 || !((attr_done >> dev) & 1u)) {
    cudaFuncSetAttribute(shm_kernel_v1, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(sizeof(float2) << kMaxShmActive));
    if (dev < 32) attr_done |= 1u << dev;
  }
  const uint64_t nb = 1ull << (a.n - a.m);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int per_sm = std::max(1, (int)((200u << 10) / (smem + 1024)));
  const uint64_t grid = std::min<uint64_t>(nb, (uint64_t)sms * std::min(per_sm, 8));
  shm_kernel_v1<<<(unsigned)grid, kThreads, smem, s>>>(P);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_cuda_error("shm kernel launch", e);
    return QS_ECUDA;
  }
  return QS_OK;
}

}  // namespace qs

// ---------------------------------------------------------------------------
// Register-phased shared-memory kernel (program compiled by shm_program.cpp).
//
// Per batch: every thread loads its 32 amplitudes straight from HBM into
// registers (lane bits = the forced low qubits, so each warp access is two
// 128-byte runs), interprets the kernel's program -- gates as register
// arithmetic on register bits, controls and diagonal factors on thread or
// batch bits -- exchanging through a swizzled shared-memory tile only when
// the register bits change, and stores the registers back to HBM.
// ---------------------------------------------------------------------------
#include "shm_program.hpp"

namespace qs {

namespace {

struct V2Params {
  float2* psi;
  const uint32_t* prog;
  int n;
  uint64_t amask;
  uint32_t ld_er[kRegBits];
  uint32_t ld_tloc[kMaxThreadBits];
  uint32_t ld_tswz[kMaxThreadBits];
  uint64_t ld_preg[kRegBits], ld_pthr[kMaxThreadBits];
  uint64_t st_preg[kRegBits], st_pthr[kMaxThreadBits];
};

__host__ __device__ constexpr int ctz_c(int i) { return (i & 1) ? 0 : 1 + ctz_c(i >> 1); }

__device__ __forceinline__ float2 cmul2(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

__device__ __forceinline__ float ldf(const uint32_t* p) { return __uint_as_float(__ldg(p)); }

__device__ __forceinline__ uint32_t known_bit(uint32_t ref, uint32_t lt, uint64_t base) {
  return (ref & REF_GLOBAL) ? (uint32_t)((base >> (ref & 63u)) & 1ull) : ((lt >> (ref & 31u)) & 1u);
}

// mask over register index j of the pairs (or amplitudes) a control enables
__device__ __forceinline__ uint32_t control_mask(uint32_t ref, uint32_t lt, uint64_t base) {
  if (ref == REF_NONE) return 0xFFFFFFFFu;
  switch (ref) {  // register index j with bit `ref` set
    case 0: return 0xAAAAAAAAu;
    case 1: return 0xCCCCCCCCu;
    case 2: return 0xF0F0F0F0u;
    case 3: return 0xFF00FF00u;
    case 4: return 0xFFFF0000u;
    default: break;
  }
  return known_bit(ref, lt, base) ? 0xFFFFFFFFu : 0u;
}

template <int T>
__device__ __forceinline__ void op_g1(float2 (&a)[kRegAmps], const float* f, uint32_t pm) {
  const float2 u00 = make_float2(f[0], f[1]), u01 = make_float2(f[2], f[3]);
  const float2 u10 = make_float2(f[4], f[5]), u11 = make_float2(f[6], f[7]);
#pragma unroll
  for (int j = 0; j < kRegAmps; ++j) {
    if (j & (1 << T)) continue;
    if (!((pm >> j) & 1u)) continue;
    const int k = j | (1 << T);
    const float2 x = a[j], y = a[k];
    a[j] = make_float2(fmaf(u00.x, x.x, fmaf(-u00.y, x.y, fmaf(u01.x, y.x, -u01.y * y.y))),
                       fmaf(u00.x, x.y, fmaf(u00.y, x.x, fmaf(u01.x, y.y, u01.y * y.x))));
    a[k] = make_float2(fmaf(u10.x, x.x, fmaf(-u10.y, x.y, fmaf(u11.x, y.x, -u11.y * y.y))),
                       fmaf(u10.x, x.y, fmaf(u10.y, x.x, fmaf(u11.x, y.y, u11.y * y.x))));
  }
}

template <int T>
__device__ __forceinline__ void op_xg(float2 (&a)[kRegAmps], uint32_t pm) {
#pragma unroll
  for (int j = 0; j < kRegAmps; ++j) {
    if (j & (1 << T)) continue;
    if (!((pm >> j) & 1u)) continue;
    const int k = j | (1 << T);
    const float2 t = a[j];
    a[j] = a[k];
    a[k] = t;
  }
}

// diagonal on one register bit: factor e[bit]; unit[bit] skips the multiply
template <int S>
__device__ __forceinline__ void op_d1(float2 (&a)[kRegAmps], float2 e0, float2 e1, bool u0, bool u1) {
#pragma unroll
  for (int j = 0; j < kRegAmps; ++j) {
    if (j & (1 << S)) {
      if (!u1) a[j] = cmul2(a[j], e1);
    } else {
      if (!u0) a[j] = cmul2(a[j], e0);
    }
  }
}

template <int S0, int S1>
__device__ __forceinline__ void op_d2(float2 (&a)[kRegAmps], const float* f, uint32_t unit) {
#pragma unroll
  for (int j = 0; j < kRegAmps; ++j) {
    const int idx = ((j >> S0) & 1) | (((j >> S1) & 1) << 1);
    if ((unit >> idx) & 1u) continue;
    a[j] = cmul2(a[j], make_float2(f[2 * idx], f[2 * idx + 1]));
  }
}

template <int S0, int S1>
__device__ __forceinline__ void op_swapr(float2 (&a)[kRegAmps]) {
#pragma unroll
  for (int j = 0; j < kRegAmps; ++j) {
    if (!((j >> S0) & 1) || ((j >> S1) & 1)) continue;
    const int k = j ^ (1 << S0) ^ (1 << S1);
    const float2 t = a[j];
    a[j] = a[k];
    a[k] = t;
  }
}

template <int S0, int S1>
__device__ __forceinline__ void op_xx(float2 (&a)[kRegAmps], float c, float s) {
#pragma unroll
  for (int j = 0; j < kRegAmps; ++j) {
    if ((j >> S1) & 1) continue;
    const int k = j ^ (1 << S0) ^ (1 << S1);
    const float2 x = a[j], y = a[k];
    a[j] = make_float2(fmaf(c, x.x, s * y.y), fmaf(c, x.y, -s * y.x));
    a[k] = make_float2(fmaf(c, y.x, s * x.y), fmaf(c, y.y, -s * x.x));
  }
}

#define QS_PAIR_SWITCH(FN, S0, S1, ...)                                   \
  switch ((S0) * 5 + (S1)) {                                             \
    case 1: FN<0, 1>(__VA_ARGS__); break;                                \
    case 2: FN<0, 2>(__VA_ARGS__); break;                                \
    case 3: FN<0, 3>(__VA_ARGS__); break;                                \
    case 4: FN<0, 4>(__VA_ARGS__); break;                                \
    case 7: FN<1, 2>(__VA_ARGS__); break;                                \
    case 8: FN<1, 3>(__VA_ARGS__); break;                                \
    case 9: FN<1, 4>(__VA_ARGS__); break;                                \
    case 13: FN<2, 3>(__VA_ARGS__); break;                               \
    case 14: FN<2, 4>(__VA_ARGS__); break;                               \
    case 19: FN<3, 4>(__VA_ARGS__); break;                               \
    default: break;                                                      \
  }

#define QS_SLOT_SWITCH(FN, S, ...)          \
  switch (S) {                              \
    case 0: FN<0>(__VA_ARGS__); break;      \
    case 1: FN<1>(__VA_ARGS__); break;      \
    case 2: FN<2>(__VA_ARGS__); break;      \
    case 3: FN<3>(__VA_ARGS__); break;      \
    case 4: FN<4>(__VA_ARGS__); break;      \
    default: break;                         \
  }

template <int M>
__global__ void __launch_bounds__(1 << (M - kRegBits), 1 << (kMaxShmActive - M))
    shm_kernel_v2(const __grid_constant__ V2Params P) {
  extern __shared__ float2 tile[];
  const uint32_t tid = threadIdx.x;
  uint32_t lt0 = 0, st0 = 0;
  uint64_t ptl = 0, pts = 0;
#pragma unroll
  for (int k = 0; k < M - kRegBits; ++k)
    if ((tid >> k) & 1u) {
      lt0 |= P.ld_tloc[k];
      st0 ^= P.ld_tswz[k];
      ptl |= P.ld_pthr[k];
      pts |= P.st_pthr[k];
    }
  const uint64_t nb = 1ull << (P.n - M);
  for (uint64_t bt = blockIdx.x; bt < nb; bt += gridDim.x) {
    uint64_t base = 0, x = bt;
    for (int q = 0; q < P.n && x; ++q)
      if (!((P.amask >> q) & 1ull)) {
        base |= (x & 1ull) << q;
        x >>= 1;
      }
    float2 a[kRegAmps];
    {
      uint64_t p = base | ptl;
#pragma unroll
      for (int i = 0; i < kRegAmps; ++i) {
        if (i) p ^= P.ld_preg[ctz_c(i)];
        a[i ^ (i >> 1)] = P.psi[p];
      }
    }
    uint32_t lt = lt0, st = st0;
    uint32_t er[kRegBits];
#pragma unroll
    for (int i = 0; i < kRegBits; ++i) er[i] = P.ld_er[i];
    const uint32_t* pc = P.prog;
    for (;;) {
      const uint32_t w = __ldg(pc);
      const uint32_t op = w & 0xFFu, A = (w >> 8) & 0xFFu, B = (w >> 16) & 0xFFu, Cu = w >> 24;
      if (op == PK_END) break;
      if (op == PK_G1) {
        float f[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) f[i] = ldf(pc + 1 + i);
        const uint32_t pm = control_mask(B, lt, base);
        QS_SLOT_SWITCH(op_g1, A, a, f, pm)
        pc += 9;
      } else if (op == PK_XG) {
        const uint32_t pm = control_mask(B, lt, base);
        QS_SLOT_SWITCH(op_xg, A, a, pm)
        pc += 1;
      } else if (op == PK_D1) {
        const uint32_t kb = (B == REF_NONE) ? 0u : known_bit(B, lt, base);
        const float2 e0 = make_float2(ldf(pc + 1 + 4 * kb), ldf(pc + 2 + 4 * kb));
        const float2 e1 = make_float2(ldf(pc + 3 + 4 * kb), ldf(pc + 4 + 4 * kb));
        const bool u0 = (Cu >> (2 * kb)) & 1u, u1 = (Cu >> (2 * kb + 1)) & 1u;
        QS_SLOT_SWITCH(op_d1, A, a, e0, e1, u0, u1)
        pc += 9;
      } else if (op == PK_D2) {
        float f[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) f[i] = ldf(pc + 1 + i);
        QS_PAIR_SWITCH(op_d2, A, B, a, f, Cu)
        pc += 9;
      } else if (op == PK_D0) {
        const uint32_t k0 = known_bit(A, lt, base);
        const uint32_t k1 = (B == REF_NONE) ? 0u : known_bit(B, lt, base);
        const uint32_t idx = k0 | (k1 << 1);
        if (!((Cu >> idx) & 1u)) {
          const float2 e = make_float2(ldf(pc + 1 + 2 * idx), ldf(pc + 2 + 2 * idx));
#pragma unroll
          for (int j = 0; j < kRegAmps; ++j) a[j] = cmul2(a[j], e);
        }
        pc += 9;
      } else if (op == PK_SWAPR) {
        QS_PAIR_SWITCH(op_swapr, A, B, a)
        pc += 1;
      } else if (op == PK_XX) {
        const float c = ldf(pc + 1), s = ldf(pc + 2);
        QS_PAIR_SWITCH(op_xx, A, B, a, c, s)
        pc += 3;
      } else if (op == PK_XCHG) {
        __syncthreads();  // every thread has finished reading the previous exchange
        {
          uint32_t xs = st;
#pragma unroll
          for (int i = 0; i < kRegAmps; ++i) {
            if (i) xs ^= er[ctz_c(i)];
            tile[xs] = a[i ^ (i >> 1)];
          }
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < kRegBits; ++i) er[i] = __ldg(pc + 1 + i);
        lt = 0;
        st = 0;
#pragma unroll
        for (int k = 0; k < M - kRegBits; ++k) {
          const uint32_t v = __ldg(pc + 1 + kRegBits + k);
          if ((tid >> k) & 1u) {
            lt |= v & 0xFFFFu;
            st ^= v >> 16;
          }
        }
        {
          uint32_t xs = st;
#pragma unroll
          for (int i = 0; i < kRegAmps; ++i) {
            if (i) xs ^= er[ctz_c(i)];
            a[i ^ (i >> 1)] = tile[xs];
          }
        }
        pc += 1 + kRegBits + A;
      } else {
        break;  // unknown opcode: the host compiler never emits one
      }
    }
    {
      uint64_t p = base | pts;
#pragma unroll
      for (int i = 0; i < kRegAmps; ++i) {
        if (i) p ^= P.st_preg[ctz_c(i)];
        P.psi[p] = a[i ^ (i >> 1)];
      }
    }
  }
}

template <int M>
int launch_v2_m(const V2Params& P, int n, cudaStream_t s) {
  static int blocks_per_sm[64] = {0};
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t smem = sizeof(float2) << M;
  const int threads = 1 << (M - kRegBits);
  if (dev < 64 && blocks_per_sm[dev] == 0) {
    cudaFuncSetAttribute(shm_kernel_v2<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, shm_kernel_v2<M>, threads, smem);
    blocks_per_sm[dev] = std::max(1, b);
  }
  const int bps = dev < 64 ? blocks_per_sm[dev] : 1;
  const uint64_t nb = 1ull << (n - M);
  const uint64_t grid = std::min<uint64_t>(nb, (uint64_t)sms * bps);
  shm_kernel_v2<M><<<(unsigned)grid, threads, smem, s>>>(P);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_cuda_error("shm v2 kernel launch", e);
    return QS_ECUDA;
  }
  return QS_OK;
}

}  // namespace

int launch_shm_v2(const ShmV2Launch& a, cudaStream_t s) {
  const ShmProgramV2& pg = *a.pg;
  if (!pg.ok || pg.m < kMinPhasedM || pg.m > kMaxShmActive || pg.m > a.n) return QS_EINVAL;
  V2Params P;
  P.psi = a.psi;
  P.prog = a.prog;
  P.n = a.n;
  P.amask = a.amask;
  for (int i = 0; i < kRegBits; ++i) {
    P.ld_er[i] = pg.ld_er[i];
    P.ld_preg[i] = pg.ld_preg[i];
    P.st_preg[i] = pg.st_preg[i];
  }
  for (int k = 0; k < kMaxThreadBits; ++k) {
    P.ld_tloc[k] = pg.ld_tloc[k];
    P.ld_tswz[k] = pg.ld_tswz[k];
    P.ld_pthr[k] = pg.ld_pthr[k];
    P.st_pthr[k] = pg.st_pthr[k];
  }
  switch (pg.m) {
    case 10: return launch_v2_m<10>(P, a.n, s);
    case 11: return launch_v2_m<11>(P, a.n, s);
    case 12: return launch_v2_m<12>(P, a.n, s);
    case 13: return launch_v2_m<13>(P, a.n, s);
    case 14: return launch_v2_m<14>(P, a.n, s);
    default: return QS_EINVAL;
  }
}

}  // namespace qs
