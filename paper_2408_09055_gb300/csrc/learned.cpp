// Learned kernel cost inside the planners: the features of the kernel as it
// will execute (its qubit set widened exactly as the program compiler widens
// it), the network's BF16 prediction of ln(microseconds on a 30-qubit state),
// scaled by 2^(n-30).  Predictions are memoised by feature key and computed
// in batches on the GPU (a private stream, pinned staging buffers).
#include <bit>
#include <cmath>
#include <cstring>
#include <string>
#include <unordered_map>

#include "internal.hpp"

namespace qs {

constexpr int kRefQubits = 30;  // the state size the timings are taken on

void kernel_features(int n, const KStat& s, bool fusion, uint64_t exec_mask, float* f) {
  (void)n;
  std::memset(f, 0, sizeof(float) * QS_MLP_FEATURES);
  for (int q = 0; q < kRefQubits; ++q) f[q] = (float)((exec_mask >> q) & 1ull);
  for (int t = 0; t < QS_NUM_GATE_TYPES; ++t) f[30 + t] = s.cnt[t] / 16.0f;
  f[40] = s.nins / 16.0f;
  f[41] = fusion ? 1.0f : 0.0f;
  f[42] = std::popcount(exec_mask) / 16.0f;
  f[43] = s.ng / 64.0f;
}

struct LearnedCost {
  const PlanImpl* p = nullptr;
  qs_mlp* mlp = nullptr;
  int n = 0;
  uint64_t low = 0;
  int fuse_kmin = 1;
  std::unordered_map<std::string, double> memo;
  cudaStream_t stream = nullptr;
  float* dx = nullptr;
  float* dy = nullptr;
  float* hx = nullptr;
  float* hy = nullptr;
  int cap = 0;
  int status = QS_OK;  // first failure of an inference call
};

namespace {

uint64_t exec_mask(const LearnedCost* lc, const KStat& s, bool fusion) {
  if (fusion) {
    int k = std::popcount(s.q);
    return widen_mask(s.q, lc->n, std::max(k, std::min(lc->fuse_kmin, lc->n)));
  }
  uint64_t a = s.ni | lc->low;
  return widen_mask(a, lc->n, std::min(lc->n, std::max(std::popcount(a), 10)));
}

std::string key_of(const KStat& s, bool fusion, uint64_t mask) {
  std::string k(1 + 8 + 2 * (QS_NUM_GATE_TYPES + 2), '\0');
  char* w = k.data();
  w[0] = fusion ? 1 : 0;
  std::memcpy(w + 1, &mask, 8);
  std::memcpy(w + 9, s.cnt, 2 * QS_NUM_GATE_TYPES);
  std::memcpy(w + 9 + 2 * QS_NUM_GATE_TYPES, &s.nins, 2);
  std::memcpy(w + 11 + 2 * QS_NUM_GATE_TYPES, &s.ng, 2);
  return k;
}

int ensure_cap(LearnedCost* lc, int B) {
  if (B <= lc->cap) return QS_OK;
  if (lc->dx) cudaFree(lc->dx);
  if (lc->dy) cudaFree(lc->dy);
  if (lc->hx) cudaFreeHost(lc->hx);
  if (lc->hy) cudaFreeHost(lc->hy);
  lc->dx = lc->dy = lc->hx = lc->hy = nullptr;
  int cap = std::max(B, 1024);
  cudaError_t e = cudaMalloc(&lc->dx, sizeof(float) * cap * QS_MLP_FEATURES);
  if (e == cudaSuccess) e = cudaMalloc(&lc->dy, sizeof(float) * cap);
  if (e == cudaSuccess) e = cudaMallocHost(&lc->hx, sizeof(float) * cap * QS_MLP_FEATURES);
  if (e == cudaSuccess) e = cudaMallocHost(&lc->hy, sizeof(float) * cap);
  if (e != cudaSuccess) {
    lc->cap = 0;
    return cuda_status(e);
  }
  lc->cap = cap;
  return QS_OK;
}

// predicts the given feature rows (already in lc->hx) into lc->hy
int infer(LearnedCost* lc, int B) {
  cudaError_t e = cudaMemcpyAsync(lc->dx, lc->hx, sizeof(float) * B * QS_MLP_FEATURES,
                                  cudaMemcpyHostToDevice, lc->stream);
  if (e != cudaSuccess) return cuda_status(e);
  int rc = qs_mlp_forward(lc->mlp, lc->dx, B, lc->dy, 1, lc->stream);
  if (rc != QS_OK) return rc;
  e = cudaMemcpyAsync(lc->hy, lc->dy, sizeof(float) * B, cudaMemcpyDeviceToHost, lc->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(lc->stream);
  return cuda_status(e);
}

double to_cost(const LearnedCost* lc, float y) {
  // clamp the exponent so an untrained network cannot overflow the DP
  double v = std::exp(std::min(std::max((double)y, -20.0), 30.0));
  return v * std::ldexp(1.0, lc->n - kRefQubits);
}

}  // namespace

LearnedCost* learned_create(const PlanImpl* p, qs_mlp* mlp, int* status) {
  int32_t F = 0, H = 0;
  if (!mlp || qs_mlp_shape(mlp, &F, &H) != QS_OK || F != QS_MLP_FEATURES) {
    *status = QS_EINVAL;
    return nullptr;
  }
  LearnedCost* lc = new (std::nothrow) LearnedCost();
  if (!lc) {
    *status = QS_ENOMEM;
    return nullptr;
  }
  lc->p = p;
  lc->mlp = mlp;
  lc->n = p->n;
  const int fl = std::min(p->opts.forced_low, p->n);
  lc->low = fl <= 0 ? 0ull : ((1ull << fl) - 1);
  lc->fuse_kmin = p->opts.precision != QS_PREC_FP32 ? std::max(p->opts.fuse_kmin, kTcTargets)
                                                    : p->opts.fuse_kmin;
  cudaError_t e = cudaStreamCreateWithFlags(&lc->stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    *status = cuda_status(e);
    delete lc;
    return nullptr;
  }
  *status = ensure_cap(lc, 1024);
  if (*status != QS_OK) {
    learned_destroy(lc);
    return nullptr;
  }
  return lc;
}

int learned_status(const LearnedCost* lc) { return lc ? lc->status : QS_OK; }

void learned_destroy(LearnedCost* lc) {
  if (!lc) return;
  if (lc->dx) cudaFree(lc->dx);
  if (lc->dy) cudaFree(lc->dy);
  if (lc->hx) cudaFreeHost(lc->hx);
  if (lc->hy) cudaFreeHost(lc->hy);
  if (lc->stream) cudaStreamDestroy(lc->stream);
  delete lc;
}

void learned_prefetch(LearnedCost* lc, const std::vector<std::pair<KStat, bool>>& ks) {
  std::vector<std::string> keys;
  std::unordered_map<std::string, int> pending;
  for (const auto& [s, fusion] : ks) {
    uint64_t m = exec_mask(lc, s, fusion);
    std::string k = key_of(s, fusion, m);
    if (lc->memo.count(k) || pending.count(k)) continue;
    if (ensure_cap(lc, (int)keys.size() + 1) != QS_OK) break;
    pending.emplace(k, (int)keys.size());
    kernel_features(lc->n, s, fusion, m, lc->hx + keys.size() * QS_MLP_FEATURES);
    keys.push_back(std::move(k));
  }
  if (keys.empty()) return;
  int rc = infer(lc, (int)keys.size());
  if (rc != QS_OK) {
    if (lc->status == QS_OK) lc->status = rc;
    return;
  }
  for (size_t i = 0; i < keys.size(); ++i) lc->memo.emplace(keys[i], to_cost(lc, lc->hy[i]));
}

double learned_cost(LearnedCost* lc, const KStat& s, bool fusion) {
  uint64_t m = exec_mask(lc, s, fusion);
  std::string k = key_of(s, fusion, m);
  auto it = lc->memo.find(k);
  if (it != lc->memo.end()) return it->second;
  kernel_features(lc->n, s, fusion, m, lc->hx);
  int rc = infer(lc, 1);
  if (rc != QS_OK) {
    if (lc->status == QS_OK) lc->status = rc;
    return 1e30;
  }
  double v = to_cost(lc, lc->hy[0]);
  lc->memo.emplace(std::move(k), v);
  return v;
}

}  // namespace qs

extern "C" int qs_kernel_features(int32_t n, const qs_gate* gates, uint64_t ngates, int32_t kernel_type,
                                  uint64_t qubit_mask, float* out) {
  using namespace qs;
  if (!out || n < 1 || n > kMaxQubits || (ngates && !gates)) return QS_EINVAL;
  if (kernel_type != QS_KERNEL_SHM && kernel_type != QS_KERNEL_FUSED) return QS_EINVAL;
  KStat s;
  for (uint64_t i = 0; i < ngates; ++i) {
    Gate g;
    int rc = make_gate(gates[i], n, &g);
    if (rc != QS_OK) return rc;
    s.add(g, 0.0);
  }
  kernel_features(n, s, kernel_type == QS_KERNEL_FUSED, qubit_mask, out);
  return QS_OK;
}
