// Allocation-free variant of qs_apply_fused (see include/qsim.h).
//
// qs_apply_fused stages the caller's unitary in device memory it allocates
// per call (cudaMallocAsync).  This entry point stages it instead in a fixed
// file-scope device array, so it never allocates.  Host code cannot use the
// array's name as a device address: the address is looked up once per device
// with cudaGetSymbolAddress and cached.
#include <mutex>

#include "internal.hpp"

namespace qs {

namespace {

constexpr int kStaticFuseMax = 7;  // widest unitary accepted: 2^7 x 2^7
constexpr size_t kStaticUElems = size_t(1) << (2 * kStaticFuseMax);  // 128 KiB of complex64

// Staging buffer for the unitary, shared by every call on a device; it keeps
// the last call's matrix.
static __device__ __align__(256) float2 g_static_u[kStaticUElems];

std::mutex g_static_mu;
float2* g_static_addr[64] = {nullptr};  // device address of g_static_u, per device

// Set-up, once per device with that device current: the device address of
// the staging array.
int static_u_address(float2** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_status(e);
  if (dev < 0 || dev >= 64) return QS_EUNSUPPORTED;
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_u);
    if (e != cudaSuccess) return cuda_status(e);
    g_static_addr[dev] = static_cast<float2*>(p);
  }
  *out = g_static_addr[dev];
  return QS_OK;
}

}  // namespace

}  // namespace qs

using namespace qs;

extern "C" int qs_apply_fused_static(float* state, int32_t n, const int32_t* targets, int32_t k,
                                     const float* u_host, int32_t precision, void* stream) {
  if (!state || !targets || !u_host || k < 1 || n < k || n > 34) return QS_EINVAL;
  if (k > kStaticFuseMax) return QS_EINVAL;  // the matrix would not fit the static buffer
  if (precision < QS_PREC_FP32 || precision > QS_PREC_TF32X3) return QS_EINVAL;
  uint64_t seen = 0;
  for (int j = 0; j < k; ++j) {
    if (targets[j] < 0 || targets[j] >= n || ((seen >> targets[j]) & 1)) return QS_EINVAL;
    seen |= 1ull << targets[j];
  }
  float2* u_dev = nullptr;
  int rc = static_u_address(&u_dev);
  if (rc != QS_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = sizeof(float2) << (2 * k);
  cudaError_t e = cudaMemcpyAsync(u_dev, u_host, bytes, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_status(e);
  FusedLaunch a;
  a.psi = reinterpret_cast<float2*>(state);
  a.n = n;
  a.k = k;
  for (int j = 0; j < kMaxFuse; ++j) a.targets[j] = j < k ? targets[j] : -1;
  a.u = u_dev;
  a.precision = precision;
  rc = launch_fused(a, s);
  if (rc == QS_OK) rc = cuda_status(cudaStreamSynchronize(s));
  return rc;
}
