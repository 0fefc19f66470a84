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
  const uint64_t grid = std::max<uint64_t>(1, std::min<uint64_t>((len + 255) / 256, (uint64_t)sms * 16));
  remap_kernel<<<(unsigned)grid, 256, 0, s>>>(in, out, n, p, len);
  return cuda_status(cudaGetLastError());
}

}  // namespace qs
