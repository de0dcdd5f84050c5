// BF16 tensor-core form of the per-slot MLP (tcgen05 / TMEM): not yet built.
#include "common.cuh"

namespace anqs {
int mlp_tc_pack_alloc(anqs_model*) {
  return set_error(ANQS_ERR_UNSUPPORTED, "BF16 tensor-core form not available in this build");
}
int mlp_tc_pack(anqs_model*, cudaStream_t) {
  return set_error(ANQS_ERR_UNSUPPORTED, "BF16 tensor-core form not available in this build");
}
size_t eloc_tc_workspace(const anqs_model*, const anqs_ham*, uint64_t) { return 0; }
int run_eloc_tc(const anqs_model*, const anqs_ham*, const uint64_t*, uint64_t, double*, double*, void*, size_t,
                cudaStream_t) {
  return set_error(ANQS_ERR_UNSUPPORTED, "BF16 tensor-core form not available in this build");
}
}  // namespace anqs
