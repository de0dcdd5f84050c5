// anqs_local_energy_static: the FP32-form local energy with its scratch
// memory in a fixed array that the library itself holds, for callers that
// cannot allocate device memory at run time.
//
// Some callers have no way to hand the library a workspace: code running as
// a plug-in inside a host application that owns every device allocation
// through its own pool and offers no hook for scratch memory, or latency-
// critical loops where a cudaMalloc (which may synchronise the whole device)
// is not allowed after start-up.  For them this entry point takes only the
// inputs and the outputs and uses a file-scope __device__ array as scratch.
//
// The array has a fixed size (kStaticScratchBytes) and exists once on every
// GPU that loads the library, for as long as the process runs.  All calls on
// one device share it: two calls that can run at the same time on the GPU
// (issued to different streams, or from different threads without ordering)
// race on it, so the caller must order them.  The array keeps whatever the
// last call left in it; this call writes every scratch element before it
// reads it, so nothing has to start at zero.
#include <mutex>

#include "common.cuh"

namespace anqs {
namespace {

// 16 MiB: enough for n_x * n_connected up to about 690k (for example 441
// samples with 140 connected determinants each needs 1.5 MiB).
constexpr size_t kStaticScratchBytes = size_t(16) << 20;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {nullptr};
unsigned long long g_scratch_ctx[kMaxDevices] = {0};

// Identifier of the current CUDA context (the driver's cuCtxGetCurrent and
// cuCtxGetId, reached through the runtime's entry-point query so that the
// library does not link the driver library); 0 when unavailable.
unsigned long long current_context_id() {
  using GetCurrent = int (*)(void**);
  using GetId = int (*)(void*, unsigned long long*);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static bool looked_up = false;
  if (!looked_up) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<GetCurrent>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<GetId>(f);
    cudaGetLastError();
    looked_up = true;
  }
  void* ctx = nullptr;
  unsigned long long id = 0;
  if (get_current && get_id && get_current(&ctx) == 0 && ctx && get_id(ctx, &id) == 0) return id;
  return 0;
}

// Device address of the array in the current context, looked up once per
// (device, context) (the host-side symbol is only a stand-in and must never
// be passed to a kernel).  A context made anew on a device (for example
// after cudaDeviceReset) loads the module again and may place the array
// elsewhere, so a new context id triggers a new lookup.
int scratch_address(int device, void** out) {
  if (device < 0 || device >= kMaxDevices)
    return set_error(ANQS_ERR_UNSUPPORTED, "device ordinal %d beyond %d", device, kMaxDevices);
  std::lock_guard<std::mutex> lk(g_mu);
  const unsigned long long ctx = current_context_id();
  if (!g_scratch_ptr[device] || ctx != g_scratch_ctx[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(g_static_scratch)", __FILE__, __LINE__);
    g_scratch_ptr[device] = p;
    g_scratch_ctx[device] = ctx;
  }
  *out = g_scratch_ptr[device];
  return ANQS_OK;
}

}  // namespace
}  // namespace anqs

using namespace anqs;

extern "C" int anqs_local_energy_static(const anqs_model* M, const anqs_ham* H, const uint64_t* x,
                                        const uint64_t* counts, uint64_t n_x, double* ere, double* eim,
                                        double* stats, void* stream) {
  if (!M || !H) return set_error(ANQS_ERR_ARG, "null model or Hamiltonian");
  if (M->d.n_orb != H->v.n) return set_error(ANQS_ERR_ARG, "model and Hamiltonian sizes differ");
  if (M->d.form != ANQS_FORM_FP32)
    return set_error(ANQS_ERR_UNSUPPORTED, "the static-scratch local energy serves FP32-form models");
  if (n_x == 0) return set_error(ANQS_ERR_ARG, "n_x must be >= 1");
  if (!x || !ere || !eim) return set_error(ANQS_ERR_ARG, "null array argument");
  if (counts && !stats) return set_error(ANQS_ERR_ARG, "counts given without stats output");
  int dev = -1;
  ANQS_CUDA(cudaGetDevice(&dev));
  if (dev != M->device || dev != H->device)
    return set_error(ANQS_ERR_ARG, "model/Hamiltonian belong to another device than the current one");

  // scratch layout (same arrays as the workspace form)
  const uint64_t K = H->v.K;
  if (K && n_x > (uint64_t(1) << 40) / K) return set_error(ANQS_ERR_CAPACITY, "n_x * n_connected overflows");
  Arena A(nullptr, kStaticScratchBytes);
  const uint64_t m = n_x * K;
  A.take<uint64_t>(m);
  A.take<double>(m);
  A.take<double>(n_x);
  A.take<float>(n_x);
  A.take<float>(n_x);
  A.take<float>(m);
  A.take<float>(m);
  if (!A.fits())
    return set_error(ANQS_ERR_CAPACITY,
                     "static scratch of %zu bytes is too small: n_x=%llu with %llu connected each needs %zu bytes",
                     kStaticScratchBytes, (unsigned long long)n_x, (unsigned long long)K, A.off);

  void* base = nullptr;
  ANQS_TRY(scratch_address(dev, &base));
  Arena S(base, kStaticScratchBytes);
  uint64_t* xp = S.take<uint64_t>(m);
  double* hv = S.take<double>(m);
  double* hd = S.take<double>(n_x);
  float* la_x = S.take<float>(n_x);
  float* ph_x = S.take<float>(n_x);
  float* la_p = S.take<float>(m);
  float* ph_p = S.take<float>(m);
  cudaStream_t s = (cudaStream_t)stream;
  const Count nc = host_count(n_x);
  ANQS_TRY(launch_connected(H->v, x, nc, xp, hv, nullptr, hd, s));
  ANQS_TRY(logpsi_dispatch(M, H, x, nc, la_x, ph_x, s));
  ANQS_TRY(logpsi_dispatch(M, H, xp, host_count(m), la_p, ph_p, s));
  ANQS_TRY(launch_eloc_sum(H->v, nc, hv, hd, la_x, ph_x, la_p, ph_p, ere, eim, s));
  if (counts) ANQS_TRY(launch_stats(ere, eim, counts, nc, stats, s));
  return ANQS_OK;
}
