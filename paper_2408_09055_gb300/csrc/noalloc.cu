// Allocation-free variant of qs_apply_fused (see include/qsim.h).
//
// qs_apply_fused stages what the fused kernel reads -- the caller's unitary
// (FP32) or the tensor-core weights prepared from it (TF32, 3xTF32) -- in
// device memory it allocates per call (cudaMallocAsync).  This entry point
// stages it instead in a fixed file-scope device array, so it never
// allocates device memory.  Host code cannot use the array's name as a
// device address: the address is looked up once per device with
// cudaGetSymbolAddress and cached.
#include <mutex>

#include "internal.hpp"

namespace qs {

namespace {

constexpr int kStaticFuseMax = 7;  // widest unitary accepted: 2^7 x 2^7
constexpr size_t kStaticUElems = size_t(1) << (2 * kStaticFuseMax);  // 128 KiB of complex64
// the 3xTF32 weights (hi and lo parts of the 128 x 128 real block) fill it exactly
static_assert(tc_weight_floats(true) * sizeof(float) <= kStaticUElems * sizeof(float2),
              "tensor-core weights exceed the static staging array");

// Staging buffer for the unitary, shared by every call on a device; it keeps
// the last call's matrix.
static __device__ __align__(256) float2 g_static_u[kStaticUElems];

std::mutex g_static_mu;
float2* g_static_addr[64] = {nullptr};  // device address of g_static_u, per device
// host-side scratch for the widened unitary and its tensor-core weights
// (guarded by g_static_mu): static, so a call allocates no host memory either
float g_static_uw[2 << (2 * kTcTargets)];
float g_static_w[tc_weight_floats(true)];

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
  FusedLaunch a;
  a.psi = reinterpret_cast<float2*>(state);
  a.n = n;
  a.k = k;
  for (int j = 0; j < kMaxFuse; ++j) a.targets[j] = j < k ? targets[j] : -1;
  a.u = u_dev;
  a.precision = precision;
  {
    // the host scratch is released once the copy has read it: a copy from
    // pageable memory returns after the source has been consumed
    std::lock_guard<std::mutex> lk(g_static_mu);
    const float* src = u_host;
    size_t bytes = sizeof(float2) << (2 * k);
    if (precision != QS_PREC_FP32) {
      // as qs_apply_fused: widen to the kernel's 6 targets with the lowest
      // unused qubits (U (x) I), then the TF32 hi (and lo) weights
      if (k > kTcTargets || n < kTcTargets + 5) return QS_EUNSUPPORTED;
      widen_unitary(u_host, k, kTcTargets, g_static_uw);
      widen_targets(n, k, kTcTargets, a.targets);
      a.k = kTcTargets;
      const bool x3 = precision == QS_PREC_TF32X3;
      tc_prepare_weights_into(g_static_uw, x3, g_static_w);
      src = g_static_w;
      bytes = tc_weight_floats(x3) * sizeof(float);
    }
    cudaError_t e = cudaMemcpyAsync(u_dev, src, bytes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_status(e);
  }
  rc = launch_fused(a, s);
  if (rc == QS_OK) rc = cuda_status(cudaStreamSynchronize(s));
  if (rc == QS_OK) rc = tc_check_error(s, true);
  return rc;
}
