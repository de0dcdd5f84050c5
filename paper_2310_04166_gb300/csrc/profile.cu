// Launch counter and optional CUDA-event timing of the library's kernels.
// Events are recorded on the stream each kernel is launched on; reading the
// totals waits for them.  Off by default; not meant for use under stream
// capture.
#include <atomic>
#include <mutex>
#include <vector>

#include "common.cuh"

namespace anqs {
namespace {

std::atomic<uint64_t> g_launches{0};
std::atomic<int> g_prof_on{0};
std::mutex g_mu;

struct Pending {
  int id;
  cudaEvent_t a, b;
};
std::vector<Pending> g_pending;
std::vector<cudaEvent_t> g_pool;
double g_ms[PROF_COUNT];
uint64_t g_count[PROF_COUNT];

const char* kNames[PROF_COUNT] = {
    "connected_kernel",       "diagonal_kernel",      "mlp_fp32_logpsi_kernel", "mlp_fp32_slot_logits_kernel",
    "mlp_fp32_grad_kernel",   "table_kernels",        "eloc_sum_kernel",        "stats_kernel",
    "cotangent_kernel",       "sampler_draw_kernels", "mlp_tc_parent_kernel",   "mlp_tc_suffix_kernel",
    "tc_sort_kernels",        "eloc_assemble_kernel", "mlp_tc_slot_kernel",     "tf_fp32_kernel",
    "finalize_kernel",        "grad_partial_sum_kernel", "unused",              "tf_fp32_grad_kernels",
    "tf_tc_parent_kernel",    "tf_tc_suffix_kernel",  "tf_tc_slot_kernel",
    "nade_logpsi_kernel", "nade_grad_kernel", "nade_slot_kernel",
    "nade_parent_kernel",    "nade_suffix_kernel",   "mlp_tc_grad_kernel"};

cudaEvent_t get_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

}  // namespace

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

ProfScope::ProfScope(int id_, cudaStream_t s) : id(id_), stream(s), start(nullptr) {
  if (!g_prof_on.load(std::memory_order_relaxed)) return;
  std::lock_guard<std::mutex> lk(g_mu);
  start = get_event();
  if (start && cudaEventRecord(start, stream) != cudaSuccess) {
    cudaGetLastError();
    g_pool.push_back(start);
    start = nullptr;
  }
}

ProfScope::~ProfScope() {
  if (!start) return;
  std::lock_guard<std::mutex> lk(g_mu);
  cudaEvent_t stop = get_event();
  if (stop && cudaEventRecord(stop, stream) == cudaSuccess) {
    g_pending.push_back({id, start, stop});
  } else {
    cudaGetLastError();
    g_pool.push_back(start);
    if (stop) g_pool.push_back(stop);
  }
}

static int drain() {
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto& p : g_pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(p.b) != cudaSuccess || cudaEventElapsedTime(&ms, p.a, p.b) != cudaSuccess) {
      cudaGetLastError();
    } else {
      g_ms[p.id] += ms;
      g_count[p.id] += 1;
    }
    g_pool.push_back(p.a);
    g_pool.push_back(p.b);
  }
  g_pending.clear();
  return ANQS_OK;
}

}  // namespace anqs

using namespace anqs;

extern "C" {

int anqs_launch_count(uint64_t* n) {
  if (!n) return set_error(ANQS_ERR_ARG, "null output");
  *n = g_launches.load();
  return ANQS_OK;
}

int anqs_profile_enable(int on) {
  drain();
  {
    std::lock_guard<std::mutex> lk(g_mu);
    for (int i = 0; i < PROF_COUNT; ++i) {
      g_ms[i] = 0.0;
      g_count[i] = 0;
    }
  }
  g_prof_on.store(on ? 1 : 0);
  return ANQS_OK;
}

int anqs_profile_read(int id, const char** name, uint64_t* launches, double* total_ms) {
  if (id < 0 || id >= PROF_COUNT) return set_error(ANQS_ERR_ARG, "profile id %d outside 0..%d", id, PROF_COUNT - 1);
  drain();
  std::lock_guard<std::mutex> lk(g_mu);
  if (name) *name = kNames[id];
  if (launches) *launches = g_count[id];
  if (total_ms) *total_ms = g_ms[id];
  return ANQS_OK;
}

}  // extern "C"
