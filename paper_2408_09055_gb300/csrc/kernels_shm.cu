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
#include <atomic>
#include <algorithm>

#include "internal.hpp"

namespace qs {

namespace {

constexpr int kThreads = 256;

struct ShmParams {
  float2* psi;
  uint64_t hi;  // known bits of qubits outside the addressed state
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
    const uint64_t kbase = base | P.hi;  // for known-bit references only
    for (int o = 0; o < P.nops; ++o) {
      const DevOp& op = P.ops[o];
      const uint64_t cg = op.cglob;
      if ((kbase & cg) != cg) continue;  // uniform over the block
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
        const int gb0 = op.g0 >= 0 ? (int)((kbase >> op.g0) & 1) : 0;
        const int gb1 = op.g1 >= 0 ? (int)((kbase >> op.g1) & 1) : 0;
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
  P.hi = a.hi;
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
  static std::atomic<unsigned> attr_done{0};  // one bit per device ordinal < 32
  if (dev >= 32 || !((attr_done.load() >> dev) & 1u)) {
    cudaFuncSetAttribute(shm_kernel_v1, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(sizeof(float2) << kMaxShmActive));
    if (dev < 32) attr_done.fetch_or(1u << dev);
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

