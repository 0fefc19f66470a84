// Host stand-ins for the CUDA names a plan-specialised kernel's source uses,
// so that the generated source compiles as C++ and runs on the CPU with one
// host thread per CUDA thread (tests/test_jit_host.py).  Only the default
// load form is covered: its source has no inline assembly.  fmaf is the C
// library's fused multiply-add, which rounds once, as the GPU's FFMA does.
#include <barrier>
#include <cmath>
#include <cstdint>
#include <thread>
#include <vector>

struct float2 {
  float x, y;
};
static inline float2 make_float2(float a, float b) { return float2{a, b}; }
struct HostDim3 {
  unsigned x = 0, y = 0, z = 0;
};
static thread_local HostDim3 threadIdx;
static HostDim3 blockIdx, gridDim;
static std::barrier<>* host_barrier = nullptr;
static inline void __syncthreads() { host_barrier->arrive_and_wait(); }
float2 host_tile[1 << 16];  // >= the padded tile of 2^14 amplitudes

#define __global__
#define __device__
#define __forceinline__ inline
#define __restrict__
#define __launch_bounds__(...)
#define __shared__
#define tile host_tile

typedef void (*host_kernel)(float2*, unsigned long long, unsigned long long);

// one block that walks every batch (the kernels loop over batches with a
// stride of gridDim.x), nthr host threads
static void host_launch(host_kernel k, float* psi, unsigned long long nb, unsigned long long hi, unsigned nthr) {
  std::barrier<> bar((std::ptrdiff_t)nthr);
  host_barrier = &bar;
  gridDim.x = 1;
  blockIdx.x = 0;
  std::vector<std::thread> th;
  for (unsigned t = 0; t < nthr; ++t)
    th.emplace_back([=] {
      threadIdx.x = t;
      k(reinterpret_cast<float2*>(psi), nb, hi);
    });
  for (auto& x : th) x.join();
  host_barrier = nullptr;
}
