// Local-energy accumulation and count-weighted statistics in FP64
// (Eq. local_energy_def, Eq. energy_est), and the per-sample cotangents of
// the VMC gradient (Eq. grad_def).
#include <cmath>

#include "common.cuh"

namespace anqs {
namespace {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// one warp per determinant: eloc = H_xx + sum_k H_k exp(dlog|psi| + i dphase).
// The ratio psi(x')/psi(x) comes from float32 log-amplitudes, so it is formed
// in float32 (expf, sincosf of the differences); the products with H and
// their sum over the connected set are accumulated in FP64.
__global__ void eloc_sum_kernel(uint32_t K, Count n_x_, const double* __restrict__ hval,
                                const double* __restrict__ hdiag, const float* __restrict__ la_x,
                                const float* __restrict__ ph_x, const float* __restrict__ la_p,
                                const float* __restrict__ ph_p, double* __restrict__ ere,
                                double* __restrict__ eim) {
  ANQS_PDL_ENTRY();
  const int lane = threadIdx.x & 31;
  const uint64_t n_x = n_x_.get();
  const uint64_t warps = uint64_t(gridDim.x) * (blockDim.x >> 5);
  for (uint64_t l = blockIdx.x * uint64_t(blockDim.x >> 5) + (threadIdx.x >> 5); l < n_x; l += warps) {
    const float lx = la_x[l], px = ph_x[l];
    double re = 0.0, im = 0.0;
    const uint64_t base = l * K;
    for (uint32_t k = lane; k < K; k += 32) {
      const double h = hval[base + k];
      const float r = expf(la_p[base + k] - lx);
      float s, c;
      sincosf(ph_p[base + k] - px, &s, &c);
      const double hr = h * double(r);
      re = fma(hr, double(c), re);
      im = fma(hr, double(s), im);
    }
    re = warp_sum(re);
    im = warp_sum(im);
    if (lane == 0) {
      ere[l] = hdiag[l] + re;
      eim[l] = im;
    }
  }
}

// single CTA of STATS_T threads: S, E (complex) and Var in one shifted pass
// (cta_energy_stats).  Few warps on purpose: a warp-wide FP64 add is slow on
// this GPU, so the shuffle trees of many warps would cost more than the rows.
constexpr int STATS_T = 256;
__global__ void __launch_bounds__(STATS_T) stats_kernel(const double* __restrict__ ere, const double* __restrict__ eim,
                                                        const uint64_t* __restrict__ counts, Count n_x_,
                                                        double* __restrict__ stats) {
  ANQS_PDL_ENTRY();
  cta_energy_stats<STATS_T>(ere, eim, counts, n_x_.get(), stats);
}

// cot_la = 2 w Re(eloc - E), cot_ph = 2 w Im(eloc - E), w = n / S
__global__ void cotangent_kernel(const double* __restrict__ ere, const double* __restrict__ eim,
                                 const uint64_t* __restrict__ counts, const double* __restrict__ stats,
                                 Count n_x_, float* __restrict__ cl, float* __restrict__ cp) {
  ANQS_PDL_ENTRY();
  const double Er = stats[0], Ei = stats[1], S = stats[3];
  const uint64_t n_x = n_x_.get();
  for (uint64_t l = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; l < n_x; l += uint64_t(gridDim.x) * blockDim.x) {
    double w = double(counts[l]) / S;
    cl[l] = float(2.0 * w * (ere[l] - Er));
    cp[l] = float(2.0 * w * (eim[l] - Ei));
  }
}

// statistics of the union of `world` disjoint sample sets (law of total
// variance); one thread, world is small.  Empty sets (S_r = 0, whose E_r is
// 0/0) are skipped.
__global__ void stats_combine_kernel(const double* __restrict__ in, int world, double* __restrict__ out) {
  ANQS_PDL_ENTRY();
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s = 0.0, sr = 0.0, si = 0.0;
  for (int r = 0; r < world; ++r) {
    const double w = in[4 * r + 3];
    if (!(w > 0.0)) continue;
    s += w;
    sr = fma(w, in[4 * r + 0], sr);
    si = fma(w, in[4 * r + 1], si);
  }
  const double Er = sr / s, Ei = si / s;
  double v = 0.0;
  for (int r = 0; r < world; ++r) {
    if (!(in[4 * r + 3] > 0.0)) continue;
    const double dr = in[4 * r + 0] - Er, di = in[4 * r + 1] - Ei;
    v = fma(in[4 * r + 3], in[4 * r + 2] + dr * dr + di * di, v);
  }
  out[0] = Er;
  out[1] = Ei;
  out[2] = v / s;
  out[3] = s;
}

}  // namespace

int launch_stats_combine(const double* in, int world, double* out, cudaStream_t s) {
  ProfScope ps(PROF_STATS, s);
  ANQS_CUDA_LAUNCH("stats_combine_kernel", launch_k(stats_combine_kernel, dim3(1), dim3(32), 0, s, in, world, out));
  return ANQS_OK;
}

int launch_eloc_sum(const HamView& hv, Count n_x, const double* hval, const double* hdiag, const float* la_x,
                    const float* ph_x, const float* la_p, const float* ph_p, double* ere, double* eim,
                    cudaStream_t s) {
  uint64_t blocks = (n_x.n + 7) / 8;  // 8 warps per CTA
  if (blocks == 0) blocks = 1;
  if (blocks > 152 * 16) blocks = 152 * 16;
  ProfScope ps(PROF_ELOC_SUM, s);
  ANQS_CUDA_LAUNCH("eloc_sum_kernel", launch_k(eloc_sum_kernel, dim3(unsigned(blocks)), dim3(256), 0, s, hv.K, n_x, hval, hdiag, la_x, ph_x, la_p, ph_p, ere, eim));
  return ANQS_OK;
}

int launch_stats(const double* ere, const double* eim, const uint64_t* counts, Count n_x, double* stats,
                 cudaStream_t s) {
  ProfScope ps(PROF_STATS, s);
  ANQS_CUDA_LAUNCH("stats_kernel", launch_k(stats_kernel, dim3(1), dim3(STATS_T), 0, s, ere, eim, counts, n_x, stats));
  return ANQS_OK;
}

int launch_grad_cotangents(const double* ere, const double* eim, const uint64_t* counts, const double* stats,
                           Count n_x, float* cl, float* cp, cudaStream_t s) {
  uint64_t blocks = (n_x.n + 255) / 256;
  if (blocks == 0) blocks = 1;
  if (blocks > 152 * 8) blocks = 152 * 8;
  ProfScope ps(PROF_COTANGENT, s);
  ANQS_CUDA_LAUNCH("cotangent_kernel", launch_k(cotangent_kernel, dim3(unsigned(blocks)), dim3(256), 0, s, ere, eim, counts, stats, n_x, cl, cp));
  return ANQS_OK;
}

}  // namespace anqs
