// Fused kernels (Sec. 5 "Cost Function in Kernelize", kernel type 1): the
// product of a kernel's gates is one dense 2^k x 2^k unitary U applied to
// every group of 2^k amplitudes that share the non-target bits.  Viewing the
// state as a 2^k x 2^(n-k) matrix over the target qubits, this is the
// batched complex matrix product psi <- U psi.
//
// FP32 CUDA-core path.  A CTA stages a tile of 2^k rows (target index) by
// 2^cb columns (the cb lowest non-target qubits, so that each row of the tile
// is a contiguous run in memory when the targets are high qubits) in shared
// memory with U^T, and every thread accumulates a 4 x 4 block of outputs
// in registers.
#include <atomic>
#include <algorithm>

#include "internal.hpp"

namespace qs {

int launch_fused_tc(const FusedLaunch& a, cudaStream_t s);  // kernels_tc.cu

namespace {

constexpr int kThreads = 256;
constexpr int kTileLog = 12;  // 4096 amplitudes (32 KiB) per tile
constexpr int kMaxCols = 7;   // at most 128 columns per tile

struct FusedParams {
  float2* psi;
  const float2* u;
  int n, k, cb;
  uint64_t fixed;  // target and column qubits
  int8_t targets[kMaxFuse];
  int8_t cols[kTileLog];
};

__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 c) {
  return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, c.y)));
}

__global__ void __launch_bounds__(kThreads) fused_fp32_kernel(FusedParams P) {
  extern __shared__ float2 sm[];
  const int R = 1 << P.k, NC = 1 << P.cb, T = R * NC;
  float2* ut = sm;          // ut[j * R + r] = U[r][j]
  float2* tile = sm + R * R;  // tile[r * NC + c]
  __shared__ unsigned long long rowoff[1 << kMaxFuse];
  __shared__ unsigned long long coloff[1 << kMaxCols];
  const int tid = threadIdx.x;
  for (int i = tid; i < R * R; i += kThreads) {
    int r = i / R, j = i % R;
    ut[j * R + r] = P.u[i];
  }
  for (int r = tid; r < R; r += kThreads) {
    unsigned long long off = 0;
    for (int j = 0; j < P.k; ++j)
      if ((r >> j) & 1) off |= 1ull << P.targets[j];
    rowoff[r] = off;
  }
  for (int c = tid; c < NC; c += kThreads) {
    unsigned long long off = 0;
    for (int j = 0; j < P.cb; ++j)
      if ((c >> j) & 1) off |= 1ull << P.cols[j];
    coloff[c] = off;
  }
  __syncthreads();
  const uint64_t nb = 1ull << (P.n - P.k - P.cb);
  const bool blocked = (T == kThreads * 16) && R >= 4 && NC >= 4;
  const int TR = R / 4, TC = NC / 4;  // blocked: TR * TC == 256
  const int tr = tid / max(TC, 1), tc = tid % max(TC, 1);
  for (uint64_t b = blockIdx.x; b < nb; b += gridDim.x) {
    uint64_t base = 0, x = b;
    for (int q = 0; q < P.n && x; ++q)
      if (!((P.fixed >> q) & 1)) {
        base |= (x & 1ull) << q;
        x >>= 1;
      }
    for (int idx = tid; idx < T; idx += kThreads) {
      int r = idx >> P.cb, c = idx & (NC - 1);
      tile[idx] = P.psi[base | rowoff[r] | coloff[c]];
    }
    __syncthreads();
    if (blocked) {
      float2 acc[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);
      for (int j = 0; j < R; ++j) {
        float2 uv[4], tv[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) uv[i] = ut[j * R + tr + TR * i];
#pragma unroll
        for (int i = 0; i < 4; ++i) tv[i] = tile[j * NC + tc + TC * i];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[i][c] = cfma(uv[i], tv[c], acc[i][c]);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int c = 0; c < 4; ++c)
          P.psi[base | rowoff[tr + TR * i] | coloff[tc + TC * c]] = acc[i][c];
    } else {
      float2 acc[16];
#pragma unroll
      for (int s = 0; s < 16; ++s) {
        int idx = tid + kThreads * s;
        acc[s] = make_float2(0.f, 0.f);
        if (idx < T) {
          int r = idx >> P.cb, c = idx & (NC - 1);
          for (int j = 0; j < R; ++j) acc[s] = cfma(ut[j * R + r], tile[j * NC + c], acc[s]);
        }
      }
#pragma unroll
      for (int s = 0; s < 16; ++s) {
        int idx = tid + kThreads * s;
        if (idx < T) {
          int r = idx >> P.cb, c = idx & (NC - 1);
          P.psi[base | rowoff[r] | coloff[c]] = acc[s];
        }
      }
    }
    __syncthreads();
  }
}

}  // namespace

int launch_fused(const FusedLaunch& a, cudaStream_t s) {
  if (a.k < 1 || a.k > kMaxFuse || a.k > a.n) return QS_EINVAL;
  if (a.precision != QS_PREC_FP32) return launch_fused_tc(a, s);
  FusedParams P;
  P.psi = a.psi;
  P.u = a.u;
  P.n = a.n;
  P.k = a.k;
  P.fixed = 0;
  for (int j = 0; j < kMaxFuse; ++j) {
    P.targets[j] = j < a.k ? (int8_t)a.targets[j] : (int8_t)-1;
    if (j < a.k) P.fixed |= 1ull << a.targets[j];
  }
  const int cb = std::min(std::min(kMaxCols, kTileLog - a.k), a.n - a.k);
  P.cb = 0;
  for (int q = 0; q < a.n && P.cb < cb; ++q)
    if (!((P.fixed >> q) & 1)) P.cols[P.cb++] = (int8_t)q;
  for (int j = 0; j < P.cb; ++j) P.fixed |= 1ull << P.cols[j];
  for (int j = P.cb; j < kTileLog; ++j) P.cols[j] = -1;
  const size_t smem = sizeof(float2) * ((size_t(1) << (2 * a.k)) + (size_t(1) << (a.k + P.cb)));
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  static std::atomic<unsigned> attr_done{0};  // one bit per device ordinal < 32
  if (dev >= 32 || !((attr_done.load() >> dev) & 1u)) {
    cudaFuncSetAttribute(fused_fp32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(sizeof(float2) * ((1 << (2 * kMaxFuse)) + (1 << kTileLog))));
    if (dev < 32) attr_done.fetch_or(1u << dev);
  }
  const uint64_t nb = 1ull << (a.n - a.k - P.cb);
  const int per_sm = std::max(1, (int)((200u << 10) / (smem + 2048)));
  const uint64_t grid = std::min<uint64_t>(nb, (uint64_t)sms * std::min(per_sm, 8));
  fused_fp32_kernel<<<(unsigned)grid, kThreads, smem, s>>>(P);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_cuda_error("fused kernel launch", e);
    return QS_ECUDA;
  }
  return QS_OK;
}

}  // namespace qs
