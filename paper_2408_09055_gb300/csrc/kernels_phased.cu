// Register-phased shared-memory kernel: device interpreter of the programs
// compiled by shm_program.cpp (Sec. 5 "Cost Function in Kernelize", kernel
// type 2; Appendix A.2 "Insular qubits").
//
// Per batch (fixed values of the non-active qubits): every thread loads its
// 32 amplitudes straight from HBM into registers -- the lane bits are the
// forced low qubits, so each warp access is two 128-byte runs -- then runs
// the kernel's program: gates are register arithmetic on register bits,
// controls and diagonal factors on thread or batch bits use the known bit
// value, and an exchange through a swizzled shared-memory tile changes the
// register bits.  Finally the registers are stored back to HBM.
#include <atomic>
#include <algorithm>

#include "internal.hpp"
#include "shm_program.hpp"

namespace qs {

namespace {

struct V2Params {
  float2* psi;
  const uint32_t* prog;
  uint64_t hi;  // known bits of qubits outside the addressed state (chunked execution)
  int n, nruns;
  uint8_t run_src[16], run_len[16], run_dst[16];
  uint32_t ld_er[kRegBits];
  uint32_t ld_tloc[kMaxThreadBits], ld_tswz[kMaxThreadBits];
  uint32_t ld_preg[kRegBits], st_preg[kRegBits];
  uint32_t ld_pthr[kMaxThreadBits], st_pthr[kMaxThreadBits];
};

using Amps = float2[kRegAmps];

__host__ __device__ constexpr int ctz_c(int i) { return (i & 1) ? 0 : 1 + ctz_c(i >> 1); }

__device__ __forceinline__ float ldf(const uint32_t* p) { return __uint_as_float(__ldg(p)); }
__device__ __forceinline__ float2 ldc(const uint32_t* p) { return make_float2(ldf(p), ldf(p + 1)); }

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

__device__ __forceinline__ uint32_t known_bit(uint32_t ref, uint32_t lt, uint64_t base) {
  return (ref & REF_GLOBAL) ? (uint32_t)((base >> (ref & 63u)) & 1ull) : ((lt >> (ref & 31u)) & 1u);
}

// ---- one-slot matrices ------------------------------------------------------
template <int T>
__device__ __forceinline__ void k_g1(Amps& a, float2 u00, float2 u01, float2 u10, float2 u11) {
#pragma unroll
  for (int j = 0; j < kRegAmps; ++j) {
    if (j & (1 << T)) continue;
    const int k = j | (1 << T);
    const float2 x = a[j], y = a[k];
    a[j] = make_float2(fmaf(u00.x, x.x, fmaf(-u00.y, x.y, fmaf(u01.x, y.x, -u01.y * y.y))),
                       fmaf(u00.x, x.y, fmaf(u00.y, x.x, fmaf(u01.x, y.y, u01.y * y.x))));
    a[k] = make_float2(fmaf(u10.x, x.x, fmaf(-u10.y, x.y, fmaf(u11.x, y.x, -u11.y * y.y))),
                       fmaf(u10.x, x.y, fmaf(u10.y, x.x, fmaf(u11.x, y.y, u11.y * y.x))));
  }
}

template <int T>
__device__ __forceinline__ void k_g1c(Amps& a, float2 u00, float2 u01, float2 u10, float2 u11,
                                      uint32_t pm) {
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

template <int T>  // real 2x2
__device__ __forceinline__ void k_g1r(Amps& a, float r00, float r01, float r10, float r11) {
#pragma unroll
  for (int j = 0; j < kRegAmps; ++j) {
    if (j & (1 << T)) continue;
    const int k = j | (1 << T);
    const float2 x = a[j], y = a[k];
    a[j] = make_float2(fmaf(r00, x.x, r01 * y.x), fmaf(r00, x.y, r01 * y.y));
    a[k] = make_float2(fmaf(r10, x.x, r11 * y.x), fmaf(r10, x.y, r11 * y.y));
  }
}

template <int T>  // [[c0, i s1], [i s2, c3]]
__device__ __forceinline__ void k_g1x(Amps& a, float c0, float s1, float s2, float c3) {
#pragma unroll
  for (int j = 0; j < kRegAmps; ++j) {
    if (j & (1 << T)) continue;
    const int k = j | (1 << T);
    const float2 x = a[j], y = a[k];
    a[j] = make_float2(fmaf(c0, x.x, -s1 * y.y), fmaf(c0, x.y, s1 * y.x));
    a[k] = make_float2(fmaf(c3, y.x, -s2 * x.y), fmaf(c3, y.y, s2 * x.x));
  }
}

template <int T>
__device__ __forceinline__ void k_xg(Amps& a) {
#pragma unroll
  for (int j = 0; j < kRegAmps; ++j) {
    if (j & (1 << T)) continue;
    const int k = j | (1 << T);
    const float2 t = a[j];
    a[j] = a[k];
    a[k] = t;
  }
}

template <int T, int C>  // X on slot T where slot C is set
__device__ __forceinline__ void k_xgs(Amps& a) {
#pragma unroll
  for (int j = 0; j < kRegAmps; ++j) {
    if ((j & (1 << T)) || !(j & (1 << C))) continue;
    const int k = j | (1 << T);
    const float2 t = a[j];
    a[j] = a[k];
    a[k] = t;
  }
}

// diagonal factors on one slot: W selects the amplitudes (1: bit clear,
// 2: bit set, 3: both)
template <int S, int W>
__device__ __forceinline__ void k_d1(Amps& a, float2 e0, float2 e1) {
#pragma unroll
  for (int j = 0; j < kRegAmps; ++j) {
    if (j & (1 << S)) {
      if (W & 2) a[j] = cmul(a[j], e1);
    } else {
      if (W & 1) a[j] = cmul(a[j], e0);
    }
  }
}
template <int S> __device__ __forceinline__ void k_d1_all(Amps& a, float2 e0, float2 e1) { k_d1<S, 3>(a, e0, e1); }
template <int S> __device__ __forceinline__ void k_d1_lo(Amps& a, float2 e0, float2 e1) { k_d1<S, 1>(a, e0, e1); }
template <int S> __device__ __forceinline__ void k_d1_hi(Amps& a, float2 e0, float2 e1) { k_d1<S, 2>(a, e0, e1); }

template <int S0, int S1>
__device__ __forceinline__ void k_d2(Amps& a, const float2 (&d)[4]) {
#pragma unroll
  for (int j = 0; j < kRegAmps; ++j) {
    const int idx = ((j >> S0) & 1) | (((j >> S1) & 1) << 1);
    a[j] = cmul(a[j], d[idx]);
  }
}

template <int S0, int S1>
__device__ __forceinline__ void k_d2p(Amps& a, float2 e) {
#pragma unroll
  for (int j = 0; j < kRegAmps; ++j)
    if (((j >> S0) & 1) && ((j >> S1) & 1)) a[j] = cmul(a[j], e);
}

template <int S0, int S1>
__device__ __forceinline__ void k_swapr(Amps& a) {
#pragma unroll
  for (int j = 0; j < kRegAmps; ++j) {
    if (!((j >> S0) & 1) || ((j >> S1) & 1)) continue;
    const int k = j ^ (1 << S0) ^ (1 << S1);
    const float2 t = a[j];
    a[j] = a[k];
    a[k] = t;
  }
}

template <int S0, int S1>  // exp(-i t X(x)X / 2) = c I - i s X(x)X
__device__ __forceinline__ void k_xx(Amps& a, float c, float s) {
#pragma unroll
  for (int j = 0; j < kRegAmps; ++j) {
    if ((j >> S1) & 1) continue;
    const int k = j ^ (1 << S0) ^ (1 << S1);
    const float2 x = a[j], y = a[k];
    a[j] = make_float2(fmaf(c, x.x, s * y.y), fmaf(c, x.y, -s * y.x));
    a[k] = make_float2(fmaf(c, y.x, s * x.y), fmaf(c, y.y, -s * x.x));
  }
}

template <int S0, int S1>  // dense 4x4, index bit(S0) + 2 bit(S1), row-major in the program
__device__ __forceinline__ void k_g2(Amps& a, const uint32_t* g) {
#pragma unroll
  for (int j = 0; j < kRegAmps; ++j) {
    if (((j >> S0) & 1) || ((j >> S1) & 1)) continue;
    const int idx[4] = {j, j | (1 << S0), j | (1 << S1), j | (1 << S0) | (1 << S1)};
    const float2 x[4] = {a[idx[0]], a[idx[1]], a[idx[2]], a[idx[3]]};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      float re = 0.f, im = 0.f;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float ur = __uint_as_float(__ldg(g + 2 * (4 * i + k)));
        const float ui = __uint_as_float(__ldg(g + 2 * (4 * i + k) + 1));
        re = fmaf(ur, x[k].x, fmaf(-ui, x[k].y, re));
        im = fmaf(ur, x[k].y, fmaf(ui, x[k].x, im));
      }
      a[idx[i]] = make_float2(re, im);
    }
  }
}

__device__ __forceinline__ void k_scale(Amps& a, float2 e) {
#pragma unroll
  for (int j = 0; j < kRegAmps; ++j) a[j] = cmul(a[j], e);
}

#define QS_SLOT(FN, S, ...)                 \
  switch (S) {                              \
    case 0: FN<0>(__VA_ARGS__); break;      \
    case 1: FN<1>(__VA_ARGS__); break;      \
    case 2: FN<2>(__VA_ARGS__); break;      \
    case 3: FN<3>(__VA_ARGS__); break;      \
    case 4: FN<4>(__VA_ARGS__); break;      \
    default: break;                         \
  }

#define QS_PAIR(FN, S0, S1, ...)                \
  switch ((S0) * 5 + (S1)) {                    \
    case 1: FN<0, 1>(__VA_ARGS__); break;       \
    case 2: FN<0, 2>(__VA_ARGS__); break;       \
    case 3: FN<0, 3>(__VA_ARGS__); break;       \
    case 4: FN<0, 4>(__VA_ARGS__); break;       \
    case 7: FN<1, 2>(__VA_ARGS__); break;       \
    case 8: FN<1, 3>(__VA_ARGS__); break;       \
    case 9: FN<1, 4>(__VA_ARGS__); break;       \
    case 13: FN<2, 3>(__VA_ARGS__); break;      \
    case 14: FN<2, 4>(__VA_ARGS__); break;      \
    case 19: FN<3, 4>(__VA_ARGS__); break;      \
    default: break;                             \
  }

#define QS_OPAIR(FN, T, C, ...)                 \
  switch ((T) * 5 + (C)) {                      \
    case 1: FN<0, 1>(__VA_ARGS__); break;       \
    case 2: FN<0, 2>(__VA_ARGS__); break;       \
    case 3: FN<0, 3>(__VA_ARGS__); break;       \
    case 4: FN<0, 4>(__VA_ARGS__); break;       \
    case 5: FN<1, 0>(__VA_ARGS__); break;       \
    case 7: FN<1, 2>(__VA_ARGS__); break;       \
    case 8: FN<1, 3>(__VA_ARGS__); break;       \
    case 9: FN<1, 4>(__VA_ARGS__); break;       \
    case 10: FN<2, 0>(__VA_ARGS__); break;      \
    case 11: FN<2, 1>(__VA_ARGS__); break;      \
    case 13: FN<2, 3>(__VA_ARGS__); break;      \
    case 14: FN<2, 4>(__VA_ARGS__); break;      \
    case 15: FN<3, 0>(__VA_ARGS__); break;      \
    case 16: FN<3, 1>(__VA_ARGS__); break;      \
    case 17: FN<3, 2>(__VA_ARGS__); break;      \
    case 19: FN<3, 4>(__VA_ARGS__); break;      \
    case 20: FN<4, 0>(__VA_ARGS__); break;      \
    case 21: FN<4, 1>(__VA_ARGS__); break;      \
    case 22: FN<4, 2>(__VA_ARGS__); break;      \
    case 23: FN<4, 3>(__VA_ARGS__); break;      \
    default: break;                             \
  }

template <int M>
__global__ void __launch_bounds__(1 << (M - kRegBits), 1 << (kMaxShmActive - M))
    shm_kernel_v2(const __grid_constant__ V2Params P) {
  extern __shared__ float2 tile[];
  const uint32_t tid = threadIdx.x;
  uint32_t lt0 = 0, st0 = 0, ptl = 0, pts = 0;
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
    uint64_t base = 0;
    for (int r = 0; r < P.nruns; ++r)
      base |= ((bt >> P.run_src[r]) & ((1ull << P.run_len[r]) - 1ull)) << P.run_dst[r];
    const uint64_t kbase = base | P.hi;  // for known-bit references only
    Amps a;
    {
      const float2* tp = P.psi + (base | ptl);
      uint32_t off = 0;
#pragma unroll
      for (int i = 0; i < kRegAmps; ++i) {
        if (i) off ^= P.ld_preg[ctz_c(i)];
        a[i ^ (i >> 1)] = tp[off];
      }
    }
    uint32_t lt = lt0, st = st0;
    uint32_t er[kRegBits];
#pragma unroll
    for (int i = 0; i < kRegBits; ++i) er[i] = P.ld_er[i];
    const uint32_t* pc = P.prog;
    bool run = true;
    while (run) {
      const uint32_t w = __ldg(pc);
      const uint32_t A = (w >> 8) & 0xFFu, B = (w >> 16) & 0xFFu, Cu = w >> 24;
      switch (w & 0xFFu) {
        case PK_G1: {
          const float2 u00 = ldc(pc + 1), u01 = ldc(pc + 3), u10 = ldc(pc + 5), u11 = ldc(pc + 7);
          QS_SLOT(k_g1, A, a, u00, u01, u10, u11)
          pc += 9;
          break;
        }
        case PK_G1R: {
          const float r00 = ldf(pc + 1), r01 = ldf(pc + 2), r10 = ldf(pc + 3), r11 = ldf(pc + 4);
          QS_SLOT(k_g1r, A, a, r00, r01, r10, r11)
          pc += 5;
          break;
        }
        case PK_G1X: {
          const float c0 = ldf(pc + 1), s1 = ldf(pc + 2), s2 = ldf(pc + 3), c3 = ldf(pc + 4);
          QS_SLOT(k_g1x, A, a, c0, s1, s2, c3)
          pc += 5;
          break;
        }
        case PK_G1C: {
          const float2 u00 = ldc(pc + 1), u01 = ldc(pc + 3), u10 = ldc(pc + 5), u11 = ldc(pc + 7);
          uint32_t pm;
          if (B < (uint32_t)kRegBits) {
            pm = B == 0 ? 0xAAAAAAAAu : B == 1 ? 0xCCCCCCCCu : B == 2 ? 0xF0F0F0F0u
               : B == 3 ? 0xFF00FF00u : 0xFFFF0000u;
          } else {
            pm = known_bit(B, lt, kbase) ? 0xFFFFFFFFu : 0u;
          }
          QS_SLOT(k_g1c, A, a, u00, u01, u10, u11, pm)
          pc += 9;
          break;
        }
        case PK_XG:
          QS_SLOT(k_xg, A, a)
          pc += 1;
          break;
        case PK_XGS:
          QS_OPAIR(k_xgs, A, B, a)
          pc += 1;
          break;
        case PK_XGK:
          if (known_bit(B, lt, kbase)) {
            QS_SLOT(k_xg, A, a)
          }
          pc += 1;
          break;
        case PK_D1B: {
          const float2 e1 = ldc(pc + 1);
          QS_SLOT(k_d1_hi, A, a, e1, e1)
          pc += 3;
          break;
        }
        case PK_D1: {
          const float2 e0 = ldc(pc + 1), e1 = ldc(pc + 3);
          QS_SLOT(k_d1_all, A, a, e0, e1)
          pc += 5;
          break;
        }
        case PK_D1K: {
          const uint32_t kb = known_bit(B, lt, kbase);
          const float2 e0 = ldc(pc + 1 + 4 * kb), e1 = ldc(pc + 3 + 4 * kb);
          const uint32_t u = (Cu >> (2 * kb)) & 3u;  // bit0: e0 is 1, bit1: e1 is 1
          if (u == 0) {
            QS_SLOT(k_d1_all, A, a, e0, e1)
          } else if (u == 1) {
            QS_SLOT(k_d1_hi, A, a, e0, e1)
          } else if (u == 2) {
            QS_SLOT(k_d1_lo, A, a, e0, e1)
          }
          pc += 9;
          break;
        }
        case PK_D2: {
          const float2 d[4] = {ldc(pc + 1), ldc(pc + 3), ldc(pc + 5), ldc(pc + 7)};
          QS_PAIR(k_d2, A, B, a, d)
          pc += 9;
          break;
        }
        case PK_D2P: {
          const float2 e = ldc(pc + 1);
          QS_PAIR(k_d2p, A, B, a, e)
          pc += 3;
          break;
        }
        case PK_D0: {
          const uint32_t k0 = known_bit(A, lt, kbase);
          const uint32_t k1 = (B == REF_NONE) ? 0u : known_bit(B, lt, kbase);
          const uint32_t idx = k0 | (k1 << 1);
          if (!((Cu >> idx) & 1u)) k_scale(a, ldc(pc + 1 + 2 * idx));
          pc += 9;
          break;
        }
        case PK_SWAPR:
          QS_PAIR(k_swapr, A, B, a)
          pc += 1;
          break;
        case PK_XX: {
          const float c = ldf(pc + 1), s = ldf(pc + 2);
          QS_PAIR(k_xx, A, B, a, c, s)
          pc += 3;
          break;
        }
        case PK_SCALE:
          k_scale(a, ldc(pc + 1));
          pc += 3;
          break;
        case PK_G2:
          QS_PAIR(k_g2, A, B, a, pc + 1)
          pc += 33;
          break;
        case PK_XCHG: {
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
          break;
        }
        default:  // PK_END (the host compiler emits no other opcode)
          run = false;
          break;
      }
    }
    {
      float2* tp = P.psi + (base | pts);
      uint32_t off = 0;
#pragma unroll
      for (int i = 0; i < kRegAmps; ++i) {
        if (i) off ^= P.st_preg[ctz_c(i)];
        tp[off] = a[i ^ (i >> 1)];
      }
    }
  }
}

template <int M>
int launch_m(const V2Params& P, int n, cudaStream_t s) {
  static std::atomic<int> blocks_per_sm[64];  // per device ordinal; 0: not yet set up
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t smem = sizeof(float2) << M;
  const int threads = 1 << (M - kRegBits);
  int bps = dev < 64 ? blocks_per_sm[dev].load() : 0;
  if (bps == 0) {
    cudaFuncSetAttribute(shm_kernel_v2<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, shm_kernel_v2<M>, threads, smem);
    bps = std::max(1, b);
    if (dev < 64) blocks_per_sm[dev].store(bps);
  }
  const uint64_t nb = 1ull << (n - M);
  const uint64_t grid = std::min<uint64_t>(nb, (uint64_t)sms * bps);
  shm_kernel_v2<M><<<(unsigned)grid, threads, smem, s>>>(P);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_cuda_error("phased shm kernel launch", e);
    return QS_ECUDA;
  }
  return QS_OK;
}

}  // namespace

int launch_jit(cudaKernel_t k, const ShmProgramV2& pg, int blocks_per_sm, float2* psi, int n, uint64_t hi,
               cudaStream_t s) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int m = pg.m;
  const size_t smem = (size_t)pg.jit_smem;
  const int threads = 1 << (m - kRegBits);
  const int bps = std::max(1, blocks_per_sm);
  unsigned long long nb = 1ull << (n - m);
  const uint64_t grid = std::min<uint64_t>(nb, (uint64_t)sms * bps);
  unsigned long long hiv = hi;
  void* args[] = {&psi, &nb, &hiv};
  cudaError_t e = cudaLaunchKernel((const void*)k, dim3((unsigned)grid), dim3(threads), args, smem, s);
  if (e != cudaSuccess) {
    set_cuda_error("specialised shm kernel launch", e);
    return QS_ECUDA;
  }
  return QS_OK;
}

int launch_shm_v2(const ShmV2Launch& a, cudaStream_t s) {
  const ShmProgramV2& pg = *a.pg;
  if (!pg.ok || pg.m < kMinPhasedM || pg.m > kMaxShmActive || pg.m > a.n) return QS_EINVAL;
  V2Params P;
  P.psi = a.psi;
  P.prog = a.prog;
  P.hi = a.hi;
  P.n = a.n;
  P.nruns = pg.nruns;
  for (int r = 0; r < 16; ++r) {
    P.run_src[r] = r < pg.nruns ? pg.run_src[r] : 0;
    P.run_len[r] = r < pg.nruns ? pg.run_len[r] : 0;
    P.run_dst[r] = r < pg.nruns ? pg.run_dst[r] : 0;
  }
  for (int i = 0; i < kRegBits; ++i) {
    P.ld_er[i] = pg.ld_er[i];
    P.ld_preg[i] = (uint32_t)pg.ld_preg[i];
    P.st_preg[i] = (uint32_t)pg.st_preg[i];
  }
  for (int k = 0; k < kMaxThreadBits; ++k) {
    P.ld_tloc[k] = pg.ld_tloc[k];
    P.ld_tswz[k] = pg.ld_tswz[k];
    P.ld_pthr[k] = (uint32_t)pg.ld_pthr[k];
    P.st_pthr[k] = (uint32_t)pg.st_pthr[k];
  }
  switch (pg.m) {
    case 10: return launch_m<10>(P, a.n, s);
    case 11: return launch_m<11>(P, a.n, s);
    case 12: return launch_m<12>(P, a.n, s);
    case 13: return launch_m<13>(P, a.n, s);
    case 14: return launch_m<14>(P, a.n, s);
    default: return QS_EINVAL;
  }
}

}  // namespace qs
