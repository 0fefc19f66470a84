// Learned kernel cost inside the planners: the features of the kernel as it
// will execute (its qubit set widened exactly as the program compiler widens
// it), the network's BF16 prediction of ln(microseconds on a 30-qubit state),
// scaled by 2^(n-30).  Predictions are memoised by feature key and computed
// in batches on the GPU (a private stream, pinned staging buffers).
#include <bit>
#include <cmath>
#include <cstring>
#include <limits>
#include <vector>

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

// What a prediction depends on, packed into five words: the executed qubit
// mask, the per-type gate counts, the insular and total gate counts, and the
// kernel type.
struct LKey {
  uint64_t w[5];
  bool operator==(const LKey& o) const { return std::memcmp(w, o.w, sizeof w) == 0; }
};
static_assert(QS_NUM_GATE_TYPES == 10, "key layout holds ten gate counts");

// Memo of predictions: open addressing with linear probing, power-of-two
// capacity, at most half full.  A NaN value marks a key whose prediction is
// queued in the current batch.
struct Memo {
  std::vector<LKey> keys;
  std::vector<double> vals;
  std::vector<uint8_t> used;
  size_t count = 0;
  static uint64_t hash(const LKey& k) {
    uint64_t h = 0x9E3779B97F4A7C15ull;
    for (uint64_t x : k.w) {
      h ^= x + 0x9E3779B97F4A7C15ull + (h << 6) + (h >> 2);
      h ^= h >> 31;
      h *= 0xBF58476D1CE4E5B9ull;
    }
    return h ^ (h >> 29);
  }
  void grow() {
    const size_t cap = keys.empty() ? 1024 : 2 * keys.size();
    std::vector<LKey> ok;
    std::vector<double> ov;
    std::vector<uint8_t> ou;
    ok.swap(keys);
    ov.swap(vals);
    ou.swap(used);
    keys.assign(cap, LKey{});
    vals.assign(cap, 0.0);
    used.assign(cap, 0);
    count = 0;
    for (size_t i = 0; i < ok.size(); ++i)
      if (ou[i]) *slot(ok[i], nullptr) = ov[i];
  }
  // room for `extra` more keys without growing: slot pointers taken after
  // this stay valid for the next `extra` insertions
  void reserve(size_t extra) {
    while (2 * (count + extra) > keys.size()) grow();
  }
  // the value slot of k, inserting it (value NaN) when absent; *inserted
  // tells which
  double* slot(const LKey& k, bool* inserted) {
    if (2 * (count + 1) > keys.size()) grow();
    const size_t mask = keys.size() - 1;
    for (size_t i = hash(k) & mask;; i = (i + 1) & mask) {
      if (!used[i]) {
        used[i] = 1;
        keys[i] = k;
        vals[i] = std::numeric_limits<double>::quiet_NaN();
        ++count;
        if (inserted) *inserted = true;
        return &vals[i];
      }
      if (keys[i] == k) {
        if (inserted) *inserted = false;
        return &vals[i];
      }
    }
  }
};

struct LearnedCost {
  const PlanImpl* p = nullptr;
  qs_mlp* mlp = nullptr;
  int n = 0;
  uint64_t low = 0;
  int fuse_kmin = 1;
  Memo memo;
  // discovery mode: a miss records the kernel (for one batched inference)
  // and reads as infeasible instead of running an inference of its own
  bool collect = false;
  std::vector<std::pair<KStat, bool>> want;
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

LKey key_of(const KStat& s, bool fusion, uint64_t mask) {
  LKey k{};
  k.w[0] = mask;
  std::memcpy(&k.w[1], s.cnt, 16);  // counts of types 0..7
  k.w[3] = (uint64_t)s.cnt[8] | ((uint64_t)s.cnt[9] << 16) | ((uint64_t)s.nins << 32) | ((uint64_t)s.ng << 48);
  k.w[4] = fusion ? 1 : 0;
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
  // keys new to the memo get a NaN slot (so a repeat in this batch is
  // skipped) and a feature row; one inference fills them
  std::vector<double*> pending;
  lc->memo.reserve(ks.size());  // no growth below: the queued slot pointers stay valid
  for (const auto& [s, fusion] : ks) {
    const uint64_t m = exec_mask(lc, s, fusion);
    bool fresh = false;
    double* v = lc->memo.slot(key_of(s, fusion, m), &fresh);
    if (!fresh && !std::isnan(*v)) continue;  // known (a NaN slot was queued by discovery)
    *v = 0.0;  // claimed by this batch: a repeat below is skipped
    if (ensure_cap(lc, (int)pending.size() + 1) != QS_OK) {
      *v = 1e30;  // never left unfilled; the status below fails the plan
      if (lc->status == QS_OK) lc->status = QS_ENOMEM;
      break;
    }
    kernel_features(lc->n, s, fusion, m, lc->hx + pending.size() * QS_MLP_FEATURES);
    pending.push_back(v);
  }
  if (pending.empty()) return;
  int rc = infer(lc, (int)pending.size());
  if (rc != QS_OK && lc->status == QS_OK) lc->status = rc;
  for (size_t i = 0; i < pending.size(); ++i) *pending[i] = rc == QS_OK ? to_cost(lc, lc->hy[i]) : 1e30;
}

void learned_collect_begin(LearnedCost* lc) {
  lc->collect = true;
  lc->want.clear();
}

bool learned_collect_end(LearnedCost* lc) {
  lc->collect = false;
  if (lc->want.empty()) return false;
  std::vector<std::pair<KStat, bool>> w;
  w.swap(lc->want);
  learned_prefetch(lc, w);
  return true;
}

double learned_cost(LearnedCost* lc, const KStat& s, bool fusion) {
  const uint64_t m = exec_mask(lc, s, fusion);
  const LKey key = key_of(s, fusion, m);
  if (lc->collect) {
    bool fresh = false;
    double* v = lc->memo.slot(key, &fresh);
    if (!fresh && !std::isnan(*v)) return *v;
    if (fresh) lc->want.push_back({s, fusion});  // NaN until the batch fills it
    return 1e30;
  }
  bool fresh = false;
  double* v = lc->memo.slot(key, &fresh);
  if (!fresh && !std::isnan(*v)) return *v;
  kernel_features(lc->n, s, fusion, m, lc->hx);
  int rc = infer(lc, 1);
  if (rc != QS_OK) {
    if (lc->status == QS_OK) lc->status = rc;
    *v = 1e30;
    return 1e30;
  }
  *v = to_cost(lc, lc->hy[0]);
  return *v;
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
