// Tabular ansatz: slot p's eight outputs are read from a table indexed by
// the prefix v_<p (the prefix bits x & (4^p - 1)).  Used to inject given
// conditionals, e.g. those of an exact eigenvector (Eq. anqs_def with the
// marginals of |c_x|^2 as conditionals).
#include <cmath>

#include "common.cuh"

namespace anqs {
namespace {

__device__ __forceinline__ const float* table_row(const float* params, int p, uint64_t x) {
  uint64_t off = 8ull * (((1ull << (2 * p)) - 1ull) / 3ull);
  uint64_t row = x & ((1ull << (2 * p)) - 1ull);
  return params + off + 8ull * row;
}

__global__ void table_logpsi_kernel(const float* __restrict__ params, int n, HamView hv,
                                    const uint64_t* __restrict__ xs, Count n_x_, float* __restrict__ la_out,
                                    float* __restrict__ ph_out) {
  ANQS_PDL_ENTRY();
  const uint64_t n_x = n_x_.get();
  for (uint64_t l = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; l < n_x; l += uint64_t(gridDim.x) * blockDim.x) {
    uint64_t x = xs[l];
    float la = 0.f, ph = 0.f;
    bool dead = (x >> (2 * n)) != 0;
    int a = 0, b = 0;
    for (int p = 0; p < n && !dead; ++p) {
      const float* o8 = table_row(params, p, x);
      int v = int((x >> (2 * p)) & 3ull);
      const unsigned pm = slot_mask(hv, p, a, b, x), mk = norm_mask(hv, p, pm);
      if (!((pm >> v) & 1u)) {
        dead = true;
        break;
      }
      float mx = -INFINITY;
      for (int u = 0; u < 4; ++u)
        if ((mk >> u) & 1u) mx = fmaxf(mx, o8[u]);
      float s = 0.f;
      for (int u = 0; u < 4; ++u)
        if ((mk >> u) & 1u) s += expf(o8[u] - mx);
      la += 0.5f * (o8[v] - mx - logf(s));
      ph += o8[4 + v];
      a += v & 1;
      b += v >> 1;
    }
    la_out[l] = dead ? -INFINITY : la;
    ph_out[l] = ph;
  }
}

__global__ void table_logits_kernel(const float* __restrict__ params, int p, const uint64_t* __restrict__ pre,
                                    const uint64_t* __restrict__ n_rows_dev, float* __restrict__ out) {
  ANQS_PDL_ENTRY();
  const uint64_t n = *n_rows_dev;
  for (uint64_t t = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; t < n * 8; t += uint64_t(gridDim.x) * blockDim.x)
    out[t] = table_row(params, p, pre[t / 8])[t % 8];
}

}  // namespace

int launch_table_logpsi(const anqs_model* md, const HamView& hv, const uint64_t* x, Count n_x, float* la,
                        float* ph, cudaStream_t s) {
  uint64_t blocks = (n_x.n + 255) / 256;
  if (blocks == 0) blocks = 1;
  if (blocks > 152 * 16) blocks = 152 * 16;
  ProfScope ps(PROF_TABLE, s);
  ANQS_CUDA_LAUNCH("table_logpsi_kernel", launch_k(table_logpsi_kernel, dim3(unsigned(blocks)), dim3(256), 0, s, md->params, md->d.n_orb, hv, x, n_x, la, ph));
  return ANQS_OK;
}

int launch_table_slot_logits(const anqs_model* md, int p, const uint64_t* pre, const uint64_t* nr,
                             uint64_t max_rows, float* out, cudaStream_t s) {
  uint64_t blocks = (max_rows * 8 + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  ProfScope ps(PROF_TABLE, s);
  ANQS_CUDA_LAUNCH("table_logits_kernel", launch_k(table_logits_kernel, dim3(unsigned(blocks ? blocks : 1)), dim3(256), 0, s, md->params, p, pre, nr, out));
  return ANQS_OK;
}

}  // namespace anqs
