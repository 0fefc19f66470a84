// State initialisation, FP64 reductions (norm, fidelity, max-abs error) and
// the qubit-remap permutation (Alg. 1 "Shard": the state is permuted so that
// a stage's qubits occupy the low physical bits, Fig. 2).
#include <algorithm>
#include <vector>

#include "internal.hpp"

namespace qs {

namespace {

constexpr int kRedThreads = 512;

__global__ void set_first_kernel(float2* psi) { psi[0] = make_float2(1.f, 0.f); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Per-block partial sums of |psi_i|^2 in FP64 (one value per block).
__global__ void __launch_bounds__(kRedThreads) norm2_kernel(const float4* psi, uint64_t n4,
                                                            double* part) {
  double s = 0;
  for (uint64_t i = blockIdx.x * (uint64_t)kRedThreads + threadIdx.x; i < n4;
       i += (uint64_t)gridDim.x * kRedThreads) {
    float4 v = psi[i];
    s += (double)v.x * v.x + (double)v.y * v.y + (double)v.z * v.z + (double)v.w * v.w;
  }
  __shared__ double red[kRedThreads / 32];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < kRedThreads / 32 ? red[threadIdx.x] : 0.0;
    t = warp_sum(t);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
  }
}

// Per-block partials: Re/Im <ref|psi>, <ref|ref>, <psi|psi>, max |ref - psi|.
__global__ void __launch_bounds__(kRedThreads) compare_kernel(const float2* psi, const double2* ref,
                                                              uint64_t len, double* part) {
  double ir = 0, ii = 0, rr = 0, pp = 0, mx = 0;
  for (uint64_t i = blockIdx.x * (uint64_t)kRedThreads + threadIdx.x; i < len;
       i += (uint64_t)gridDim.x * kRedThreads) {
    float2 p = psi[i];
    double2 r = ref[i];
    double px = p.x, py = p.y;
    ir += r.x * px + r.y * py;  // conj(r) * p
    ii += r.x * py - r.y * px;
    rr += r.x * r.x + r.y * r.y;
    pp += px * px + py * py;
    double dx = r.x - px, dy = r.y - py;
    mx = fmax(mx, sqrt(dx * dx + dy * dy));
  }
  __shared__ double red[5][kRedThreads / 32];
  double v[5] = {ir, ii, rr, pp, mx};
#pragma unroll
  for (int k = 0; k < 4; ++k) v[k] = warp_sum(v[k]);
  v[4] = warp_max(v[4]);
  if ((threadIdx.x & 31) == 0)
    for (int k = 0; k < 5; ++k) red[k][threadIdx.x >> 5] = v[k];
  __syncthreads();
  if (threadIdx.x < 32) {
    for (int k = 0; k < 5; ++k) {
      double t = threadIdx.x < kRedThreads / 32 ? red[k][threadIdx.x] : (k == 4 ? 0.0 : 0.0);
      t = k == 4 ? warp_max(t) : warp_sum(t);
      if (threadIdx.x == 0) part[5 * blockIdx.x + k] = t;
    }
  }
}

struct Perm {
  int8_t to[kMaxQubits];
};

// out[pi(i)] = in[i]: reads coalesced, writes scattered at the granularity
// of the longest run of low bits that pi keeps in place.
__global__ void remap_kernel(const float2* in, float2* out, int n, Perm p, uint64_t len) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < len;
       i += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t j = 0;
    for (int b = 0; b < n; ++b) j |= ((i >> b) & 1ull) << p.to[b];
    out[j] = in[i];
  }
}

// Tiled bit permutation for n >= 10 (a generalised transpose).  A tile is the
// set of amplitudes that differ only in the tile bits T: the 5 lowest input
// bits, the input bits that land on the 5 lowest output bits, and further low
// input bits up to |T| = 10 (1024 amplitudes, four per thread in flight).  It is
// read in runs of 32 consecutive input amplitudes into shared memory (padded
// one slot per 32) and written in runs of 32 consecutive output amplitudes.
// Index deposits use tables of 5-bit chunks:
//   t_in[c][v]  tile position t (chunk c of its bits) -> input offset
//   u_out[c][v] output-ordered tile position u -> output offset
//   u_t[c][v]   u -> t
//   g_in/g_out  tile number -> input / output base offset
struct RemapTables {
  uint64_t t_in[2][32], u_out[2][32], g_in[6][32], g_out[6][32];
  uint32_t u_t[2][32];
};
constexpr int kRemapThreads = 256;
constexpr int kRemapTile = 1024;  // 2^10 amplitudes

__global__ void __launch_bounds__(kRemapThreads) remap_tiled_kernel(const float2* __restrict__ in,
                                                                    float2* __restrict__ out,
                                                                    const RemapTables* __restrict__ tabs,
                                                                    uint64_t ntiles) {
  __shared__ RemapTables T;
  __shared__ float2 tile[kRemapTile + kRemapTile / 32];
  {
    const uint32_t* src = reinterpret_cast<const uint32_t*>(tabs);
    uint32_t* dst = reinterpret_cast<uint32_t*>(&T);
    for (uint32_t i = threadIdx.x; i < sizeof(RemapTables) / 4; i += kRemapThreads) dst[i] = src[i];
  }
  __syncthreads();
  constexpr int kPer = kRemapTile / kRemapThreads;
  for (uint64_t g = blockIdx.x; g < ntiles; g += gridDim.x) {
    uint64_t bin = 0, bout = 0;
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      const uint32_t v = (uint32_t)(g >> (5 * c)) & 31u;
      bin |= T.g_in[c][v];
      bout |= T.g_out[c][v];
    }
    float2 v[kPer];
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const uint32_t t = threadIdx.x + k * kRemapThreads;
      v[k] = in[bin | T.t_in[0][t & 31u] | T.t_in[1][t >> 5]];
    }
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const uint32_t t = threadIdx.x + k * kRemapThreads;
      tile[t + (t >> 5)] = v[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const uint32_t u = threadIdx.x + k * kRemapThreads;
      const uint32_t t = T.u_t[0][u & 31u] | T.u_t[1][u >> 5];
      v[k] = tile[t + (t >> 5)];
    }
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const uint32_t u = threadIdx.x + k * kRemapThreads;
      out[bout | T.u_out[0][u & 31u] | T.u_out[1][u >> 5]] = v[k];
    }
    __syncthreads();
  }
}

int reduction_grid(uint64_t work) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  uint64_t want = (work + kRedThreads - 1) / kRedThreads;
  return (int)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)sms * 4));
}

}  // namespace

int launch_set_zero(float2* psi, int n, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(psi, 0, sizeof(float2) << n, s);
  if (e != cudaSuccess) return cuda_status(e);
  set_first_kernel<<<1, 1, 0, s>>>(psi);
  return cuda_status(cudaGetLastError());
}

int launch_norm2(const float2* psi, int n, double* out, cudaStream_t s) {
  const uint64_t len = 1ull << n;
  if (n < 1) return QS_EINVAL;
  const uint64_t n4 = len / 2;  // float4 = two amplitudes
  const int grid = reduction_grid(n4);
  double* part = nullptr;
  cudaError_t e = cudaMallocAsync(&part, sizeof(double) * grid, s);
  if (e != cudaSuccess) return cuda_status(e);
  norm2_kernel<<<grid, kRedThreads, 0, s>>>(reinterpret_cast<const float4*>(psi), n4, part);
  std::vector<double> h(grid);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), part, sizeof(double) * grid, cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(part, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_status(e);
  double t = 0;
  for (double v : h) t += v;
  *out = t;
  return QS_OK;
}

int launch_compare(const float2* psi, const double2* ref, int n, double* fid, double* maxabs,
                   cudaStream_t s) {
  const uint64_t len = 1ull << n;
  const int grid = reduction_grid(len);
  double* part = nullptr;
  cudaError_t e = cudaMallocAsync(&part, sizeof(double) * 5 * grid, s);
  if (e != cudaSuccess) return cuda_status(e);
  compare_kernel<<<grid, kRedThreads, 0, s>>>(psi, ref, len, part);
  std::vector<double> h(5 * grid);
  e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h.data(), part, sizeof(double) * 5 * grid, cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(part, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_status(e);
  double ir = 0, ii = 0, rr = 0, pp = 0, mx = 0;
  for (int b = 0; b < grid; ++b) {
    ir += h[5 * b];
    ii += h[5 * b + 1];
    rr += h[5 * b + 2];
    pp += h[5 * b + 3];
    mx = std::max(mx, h[5 * b + 4]);
  }
  *fid = (rr > 0 && pp > 0) ? (ir * ir + ii * ii) / (rr * pp) : 0.0;
  *maxabs = mx;
  return QS_OK;
}

int launch_remap(const float2* in, float2* out, int n, const int32_t* perm, cudaStream_t s) {
  Perm p;
  for (int b = 0; b < kMaxQubits; ++b) p.to[b] = b < n ? (int8_t)perm[b] : (int8_t)0;
  const uint64_t len = 1ull << n;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (n < 10) {
    const uint64_t grid = std::max<uint64_t>(1, std::min<uint64_t>((len + 255) / 256, (uint64_t)sms * 16));
    remap_kernel<<<(unsigned)grid, 256, 0, s>>>(in, out, n, p, len);
    return cuda_status(cudaGetLastError());
  }
  // tile bits (input positions): 0..4, the preimages of output bits 0..4,
  // then further low bits up to 8 tile bits
  int inv[kMaxQubits];
  for (int b = 0; b < n; ++b) inv[perm[b]] = b;
  std::vector<int> tpos;
  uint64_t in_t = 0;
  auto add = [&](int b) {
    if (!((in_t >> b) & 1)) {
      in_t |= 1ull << b;
      tpos.push_back(b);
    }
  };
  for (int b = 0; b < 5; ++b) add(b);
  for (int o = 0; o < 5; ++o) add(inv[o]);
  for (int b = 5; b < n && (int)tpos.size() < 10; ++b) add(b);
  const int tb = (int)tpos.size();  // 10: n >= 10
  if (tb != 10) return QS_EINVAL;
  std::vector<int> upos;  // output position of u's bits
  for (int o = 0; o < 5; ++o) upos.push_back(o);
  for (int x : tpos)
    if (perm[x] >= 5) upos.push_back(perm[x]);
  std::vector<int> tindex(n, -1);
  for (int i = 0; i < tb; ++i) tindex[tpos[i]] = i;
  std::vector<int> gpos;
  for (int b = 0; b < n; ++b)
    if (!((in_t >> b) & 1)) gpos.push_back(b);
  RemapTables h{};
  for (int c = 0; c < 2; ++c)
    for (uint32_t v = 0; v < 32; ++v)
      for (int j = 0; j < 5; ++j) {
        const int i = 5 * c + j;
        if (i >= tb || !((v >> j) & 1)) continue;
        h.t_in[c][v] |= 1ull << tpos[i];
        h.u_out[c][v] |= 1ull << upos[i];
        h.u_t[c][v] |= 1u << tindex[inv[upos[i]]];
      }
  for (int c = 0; c < 6; ++c)
    for (uint32_t v = 0; v < 32; ++v)
      for (int j = 0; j < 5; ++j) {
        const int i = 5 * c + j;
        if (i >= (int)gpos.size() || !((v >> j) & 1)) continue;
        h.g_in[c][v] |= 1ull << gpos[i];
        h.g_out[c][v] |= 1ull << perm[gpos[i]];
      }
  // the tables travel in a small per-call device buffer, freed stream-ordered
  void* dt = nullptr;
  cudaError_t e = cudaMallocAsync(&dt, sizeof(RemapTables), s);
  if (e != cudaSuccess) return cuda_status(e);
  e = cudaMemcpyAsync(dt, &h, sizeof(RemapTables), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) {
    cudaFreeAsync(dt, s);
    return cuda_status(e);
  }
  const uint64_t ntiles = 1ull << (n - tb);
  const uint64_t grid = std::max<uint64_t>(1, std::min<uint64_t>(ntiles, (uint64_t)sms * 8));
  remap_tiled_kernel<<<(unsigned)grid, kRemapThreads, 0, s>>>(in, out, static_cast<const RemapTables*>(dt),
                                                                ntiles);
  e = cudaGetLastError();
  cudaFreeAsync(dt, s);
  return cuda_status(e);
}

}  // namespace qs
