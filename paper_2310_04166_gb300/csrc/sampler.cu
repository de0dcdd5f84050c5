// Masked autoregressive statistics sampling (Sec. II.C; MU, Sec. III.C).
//
// Breadth-first over the slot tree.  Level p holds the frontier of prefixes
// (slots < p) with their sample counts.  Per level:
//   1. the network's slot-p outputs for every frontier prefix;
//   2. per node: allowed outcomes from the IsPhys slot mask, the masked
//      conditional and its running sums C_v (float32 in a fixed order of IEEE
//      operations, see split_thresholds);
//   3. the node's n_in uniforms (Philox4x64-10, one block of four per
//      thread; counter (prefix, i >> 2, p, counter), key (seed, 0)) are
//      compared with C_v and the outcome counts are aggregated per warp
//      segment before one atomic per (node, outcome);
//   4. children with nonzero counts are compacted, in (node, outcome)
//      order, into the next frontier (the last level writes the output).
// Grids are sized from host-side bounds on the frontier (the number of
// physical prefixes of each level, capped by N_s); the actual sizes stay on
// the device so that the whole sequence can be captured in a CUDA graph.
#include <cmath>

#include "common.cuh"

namespace anqs {

int logits_dispatch(const anqs_model* M, const anqs_ham* H, int p, const uint64_t* pre, const uint64_t* n_dev,
                    uint64_t max_rows, float* out8, cudaStream_t s);

namespace {

constexpr int SCAN_T = 1024;      // threads per scan CTA
constexpr int SCAN_ITEMS = 4;     // elements per thread
constexpr int SCAN_CHUNK = SCAN_T * SCAN_ITEMS;

struct Philox {
  __device__ static void block(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3, uint64_t k0, uint64_t k1,
                               uint64_t out[4]) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
      if (r) {
        k0 += W0;
        k1 += W1;
      }
      uint64_t hi0 = __umul64hi(M0, c0), lo0 = M0 * c0;
      uint64_t hi1 = __umul64hi(M1, c2), lo1 = M1 * c2;
      uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
      c0 = n0;
      c1 = lo1;
      c2 = n2;
      c3 = lo0;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
  }
};

// Grid barrier of the persistent launch: one arrival counter per level
// (zeroed by the kernel launched just before it, never reset within a pass),
// so a level's barrier is one reduction per CTA and a poll until the count
// reaches the grid size.
struct GridBarrier {
  unsigned arrive[ANQS_MAX_ORB + 1];
  int err;  // a CTA gave up waiting
  int pad[2];
};
constexpr int kBarrierWords = int(sizeof(GridBarrier) / 4);

__global__ void init_kernel(uint64_t* pre, uint64_t* cnt, uint64_t* n_front, uint64_t n_samples, unsigned* done,
                            uint64_t* child, uint32_t* idx0, int* barrier) {
  ANQS_PDL_ENTRY();
  if (idx0) idx0[0] = 0;  // prefix-table mode: the root is table row 0
  if (barrier)            // the persistent launch's grid barrier: arrivals per level, error
    for (int k = 0; k < kBarrierWords; ++k) barrier[k] = 0;
  pre[0] = 0;
  cnt[0] = n_samples;
  n_front[0] = 1;
  *done = 0;
  for (int v = 0; v < 4; ++v) child[v] = 0;
}

// ---- the split conditional, reproducible bit for bit -------------------------
// exp(x) for x <= 0 in float32 from IEEE operations only, in a fixed order
// and without fused multiply-adds: Cody-Waite reduction x = k ln2 + r (ln2
// split into a 16-bit head and a tail) and the degree-7 Taylor polynomial of
// e^r, |r| <= ln2/2 (truncation below 6e-9 relative).  The oracle evaluates
// the same sequence with numpy float32.
__device__ __forceinline__ float exp_det(float x) {
  if (x < -80.f) return 0.f;
  const float k = floorf(__fadd_rn(__fmul_rn(x, 1.44269502162933349609375f), 0.5f));
  const float r = __fsub_rn(__fsub_rn(x, __fmul_rn(k, 0.693145751953125f)), __fmul_rn(k, 1.428606765330187045e-06f));
  float q = 1.f / 5040.f;
  q = __fadd_rn(__fmul_rn(q, r), 1.f / 720.f);
  q = __fadd_rn(__fmul_rn(q, r), 1.f / 120.f);
  q = __fadd_rn(__fmul_rn(q, r), 1.f / 24.f);
  q = __fadd_rn(__fmul_rn(q, r), 1.f / 6.f);
  q = __fadd_rn(__fmul_rn(q, r), 0.5f);
  q = __fadd_rn(__fmul_rn(q, r), 1.f);
  q = __fadd_rn(__fmul_rn(q, r), 1.f);
  return ldexpf(q, int(k));
}

// ceil(C 2^53) for a float32 C in [0, 1], from its bits
__device__ __forceinline__ uint64_t thr_from_float(float C) {
  const uint32_t b = __float_as_uint(C);
  const uint32_t e = (b >> 23) & 0xFFu, mant = b & 0x7FFFFFu;
  if (e == 0) return mant ? 1ull : 0ull;  // subnormal: 0 < C 2^53 < 1
  const uint64_t m24 = uint64_t(mant | 0x800000u);
  if (e >= 97) return m24 << (e - 97);
  const uint32_t sh = 97 - e;
  if (sh >= 25) return 1ull;
  return (m24 + (1ull << sh) - 1ull) >> sh;
}

// Thresholds T_v of one node: running sums C_v of the softmax of the
// allowed logits (float32, fixed order), T_v = ceil(C_v 2^53), so that a
// draw with word w goes to the first allowed v with (w >> 11) < T_v, i.e.
// u = (w >> 11) 2^-53 < C_v.
__device__ __forceinline__ void split_thresholds(const float* l, unsigned mk, uint64_t T[4]) {
  float m = -INFINITY;
  for (int v = 0; v < 4; ++v)
    if ((mk >> v) & 1u) m = fmaxf(m, l[v]);
  float e[4], s = 0.f;
  for (int v = 0; v < 4; ++v) {
    e[v] = ((mk >> v) & 1u) ? exp_det(__fsub_rn(l[v], m)) : 0.f;
    if ((mk >> v) & 1u) s = __fadd_rn(s, e[v]);
  }
  float run = 0.f;
  for (int v = 0; v < 4; ++v) {
    if ((mk >> v) & 1u) run = __fadd_rn(run, __fdiv_rn(e[v], s));
    T[v] = thr_from_float(run);
  }
}

__device__ __forceinline__ int popc_alpha(uint64_t x, int p) {
  uint64_t m = (p >= 32) ? ~0ull : ((1ull << (2 * p)) - 1ull);
  return __popcll(x & m & 0x5555555555555555ull);
}
__device__ __forceinline__ int popc_beta(uint64_t x, int p) {
  uint64_t m = (p >= 32) ? ~0ull : ((1ull << (2 * p)) - 1ull);
  return __popcll(x & m & 0xAAAAAAAAAAAAAAAAull);
}

// per node: running sums of the masked conditional, draw-block counts
__global__ void prep_kernel(HamView hv, int p, const uint64_t* __restrict__ pre, const uint64_t* __restrict__ cnt,
                            const uint64_t* __restrict__ n_front, const float* __restrict__ logits,
                            uint64_t* __restrict__ thr, uint8_t* __restrict__ allowed, uint64_t* __restrict__ nblk,
                            uint64_t* __restrict__ child) {
  ANQS_PDL_ENTRY();
  const uint64_t nf = *n_front;
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < nf; i += uint64_t(gridDim.x) * blockDim.x) {
    uint64_t x = pre[i];
    const unsigned pm = slot_mask(hv, p, popc_alpha(x, p), popc_beta(x, p), x), mk = norm_mask(hv, p, pm);
    uint64_t T[4];
    split_thresholds(logits + i * 8, mk, T);
    for (int v = 0; v < 4; ++v) {
      thr[i * 4 + v] = T[v];
      child[i * 4 + v] = 0;
    }
    allowed[i] = uint8_t(mk | (pm << 4));  // low: normalised outcomes, high: physical ones
    nblk[i] = (cnt[i] + 3) / 4;
  }
}

__device__ __forceinline__ int draw_outcome(uint64_t word, const uint64_t* thr, unsigned mk, int last) {
  const uint64_t m = word >> 11;
  for (int v = 0; v < 4; ++v)
    if (((mk >> v) & 1u) && m < thr[v]) return v;
  return last;
}

// ---- exclusive scan of uint64 over a device-sized array -------------------
__device__ __forceinline__ uint64_t warp_incl_scan(uint64_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint64_t t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// returns the exclusive prefix of v within the CTA, total in *tot
__device__ uint64_t block_excl_scan(uint64_t v, uint64_t* sh, uint64_t* tot) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint64_t inc = warp_incl_scan(v);
  __syncthreads();
  if (lane == 31) sh[w] = inc;
  __syncthreads();
  if (w == 0) {
    uint64_t t = lane < int(blockDim.x >> 5) ? sh[lane] : 0;
    uint64_t ti = warp_incl_scan(t);
    sh[lane] = ti - t;
    if (lane == 31) sh[32] = ti;
  }
  __syncthreads();
  *tot = sh[32];
  return sh[w] + inc - v;
}

// in[i] for i < n (n = *n_dev * mult), partial sums per chunk
__global__ void scan_reduce_kernel(const uint64_t* __restrict__ in, const uint64_t* __restrict__ n_dev,
                                   uint64_t mult, uint64_t* __restrict__ partial) {
  ANQS_PDL_ENTRY();
  __shared__ uint64_t sh[33];
  const uint64_t n = *n_dev * mult;
  const uint64_t base = uint64_t(blockIdx.x) * SCAN_CHUNK;
  uint64_t v = 0;
  if (base < n)
    for (int k = 0; k < SCAN_ITEMS; ++k) {
      uint64_t i = base + uint64_t(k) * SCAN_T + threadIdx.x;
      if (i < n) v += in[i];
    }
  uint64_t tot;
  block_excl_scan(v, sh, &tot);
  if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

__global__ void scan_partials_kernel(uint64_t* __restrict__ partial, uint64_t n_part) {
  ANQS_PDL_ENTRY();
  __shared__ uint64_t sh[33];
  uint64_t carry = 0;
  for (uint64_t b = 0; b < n_part; b += SCAN_T) {
    uint64_t i = b + threadIdx.x;
    uint64_t v = i < n_part ? partial[i] : 0;
    uint64_t tot;
    uint64_t ex = block_excl_scan(v, sh, &tot);
    if (i < n_part) partial[i] = carry + ex;
    carry += tot;
    __syncthreads();
  }
}

// out[i] = exclusive prefix; out[n] = total; total also to *total_dev
__global__ void scan_apply_kernel(const uint64_t* __restrict__ in, const uint64_t* __restrict__ n_dev,
                                  uint64_t mult, const uint64_t* __restrict__ partial, uint64_t* __restrict__ out,
                                  uint64_t* __restrict__ total_dev) {
  ANQS_PDL_ENTRY();
  __shared__ uint64_t sh[33];
  const uint64_t n = *n_dev * mult;
  const uint64_t base = uint64_t(blockIdx.x) * SCAN_CHUNK;
  if (base > n) return;
  // each thread owns SCAN_ITEMS consecutive elements
  uint64_t loc[SCAN_ITEMS], s = 0;
  const uint64_t first = base + uint64_t(threadIdx.x) * SCAN_ITEMS;
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    uint64_t i = first + k;
    loc[k] = i < n ? in[i] : 0;
    s += loc[k];
  }
  uint64_t tot;
  uint64_t ex = block_excl_scan(s, sh, &tot) + partial[blockIdx.x];
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    uint64_t i = first + k;
    if (i < n) out[i] = ex;
    if (i == n) {
      out[n] = ex;
      if (total_dev) *total_dev = ex;
    }
    ex += loc[k];
  }
}

// ---- draws -----------------------------------------------------------------
__global__ void draw_kernel(int p, uint64_t seed, uint64_t counter0, const uint64_t* __restrict__ counter_dev,
                            const uint64_t* __restrict__ pre,
                            const uint64_t* __restrict__ cnt, const uint64_t* __restrict__ n_front,
                            const uint64_t* __restrict__ nblk_scan, const uint64_t* __restrict__ thr,
                            const uint8_t* __restrict__ allowed, uint64_t* __restrict__ child,
                            uint64_t max_threads) {
  ANQS_PDL_ENTRY();
  const uint64_t nf = *n_front;
  const uint64_t total = nblk_scan[nf];
  const uint64_t counter = counter0 + (counter_dev ? *counter_dev : 0ull);
  const int lane = threadIdx.x & 31;
  for (uint64_t t0 = blockIdx.x * uint64_t(blockDim.x); t0 < max_threads; t0 += uint64_t(gridDim.x) * blockDim.x) {
    if (t0 >= total) break;
    const uint64_t t = t0 + threadIdx.x;
    int64_t node = -1;
    uint32_t packed = 0;
    if (t < total) {
      // largest i with nblk_scan[i] <= t
      uint64_t lo = 0, hi = nf - 1;
      while (lo < hi) {
        uint64_t mid = (lo + hi + 1) >> 1;
        if (nblk_scan[mid] <= t) lo = mid;
        else hi = mid - 1;
      }
      node = int64_t(lo);
      const uint64_t ib = t - nblk_scan[lo];
      const uint64_t c = cnt[lo];
      const uint64_t x = pre[lo];
      uint64_t w[4];
      Philox::block(x, ib, uint64_t(p), counter, seed, 0ull, w);
      const unsigned mk = allowed[lo] & 0xFu, pm = allowed[lo] >> 4;
      uint64_t T[4];
      for (int v = 0; v < 4; ++v) T[v] = thr[lo * 4 + v];
      int last = 3;
      while (last > 0 && !((mk >> last) & 1u)) --last;
      for (int k = 0; k < 4; ++k) {
        if (ib * 4 + k >= c) break;
        const int v = draw_outcome(w[k], T, mk, last);
        if ((pm >> v) & 1u) packed += 1u << (8 * v);  // DU levels: a draw to an unphysical child is lost
      }
    }
    // segmented sum over lanes with the same node (nodes are non-decreasing in t)
    int64_t prev = __shfl_up_sync(0xffffffffu, node, 1);
    unsigned heads = __ballot_sync(0xffffffffu, lane == 0 || prev != node);
    int seg_start = 31 - __clz(heads & ((2u << lane) - 1u));
    uint32_t v = packed;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t other = __shfl_up_sync(0xffffffffu, v, o);
      if (lane - o >= seg_start) v += other;
    }
    bool tail = (lane == 31) || ((heads >> (lane + 1)) & 1u);
    if (tail && node >= 0)
      for (int k = 0; k < 4; ++k) {
        uint32_t ck = (v >> (8 * k)) & 0xffu;
        if (ck) atomicAdd(reinterpret_cast<unsigned long long*>(child + node * 4 + k), (unsigned long long)ck);
      }
  }
}

// ---- binomial statistics sampling (Sec. II.C) ---------------------------------
// A node's n_in samples are split among its allowed outcomes by chained
// binomials: k_v ~ B(rest, p_v / (p_v + ... + p_last)) in ascending v, the
// last allowed outcome takes the rest; the cost per node does not depend on
// n_in.  p is the node's masked conditional (the same float32 softmax as the
// multinomial split).  Each binomial draws uniforms from its own Philox
// stream: counter (prefix, (v << 32) | block, level, counter), key (seed, 1).
struct Uniforms {
  uint64_t x, v, p, counter, seed, blk;
  uint64_t w[4];
  int used;
  __device__ double next() {
    if (used == 4) {
      Philox::block(x, (v << 32) | blk, p, counter, seed, 1ull, w);
      ++blk;
      used = 0;
    }
    return double(w[used++] >> 11) * 0x1.0p-53;
  }
};

// log Gamma(x) for x >= 1 by the Stirling series, the argument shifted to
// at least 10 (truncation below 1e-13 there)
__device__ __forceinline__ double lgamma_stirling(double x) {
  double shift = 0.0;
  while (x < 10.0) {
    shift -= log(x);
    x += 1.0;
  }
  const double r = 1.0 / x, r2 = r * r;
  const double series = r * (1.0 / 12 - r2 * (1.0 / 360 - r2 * (1.0 / 1260 - r2 * (1.0 / 1680))));
  return shift + (x - 0.5) * log(x) - x + 0.91893853320467274178 + series;
}

// one draw of B(n, q)
// Sets bit 1 of *events when an inversion walk stops at k = 4096 and bit 0
// when the BTRS loop gives up after 256 rejections (returning the mode); both
// have negligible probability, and either makes that draw biased.
__device__ uint64_t binomial(uint64_t n, double q, Uniforms& U, unsigned* events) {
  if (n == 0 || !(q > 0.0)) return 0;
  if (q >= 1.0) return n;
  const bool flip = q > 0.5;
  const double p = flip ? 1.0 - q : q, qq = 1.0 - p, nd = double(n);
  uint64_t k = 0;
  if (nd * p < 10.0) {
    // inversion: walk the pmf from 0, P(k+1) = P(k) (n - k) p / ((k + 1) q)
    double u = U.next(), r = exp(nd * log1p(-p));
    const double s = p / qq, a = (nd + 1.0) * s;
    while (u > r && k < n && k < 4096) {
      u -= r;
      ++k;
      r *= a / double(k) - s;
    }
    if (u > r && k < n) *events |= 2u;
  } else {
    // BTRS: transformed rejection with squeeze (Hormann 1993)
    const double spq = sqrt(nd * p * qq);
    const double b = 1.15 + 2.53 * spq, a = -0.0873 + 0.0248 * b + 0.01 * p, c = nd * p + 0.5;
    const double vr = 0.92 - 4.2 / b, alpha = (2.83 + 5.1 / b) * spq, lpq = log(p / qq);
    const double m = floor((nd + 1.0) * p);
    const double h = lgamma_stirling(m + 1.0) + lgamma_stirling(nd - m + 1.0);
    k = uint64_t(m);
    bool accepted = false;
    for (int it = 0; it < 256 && !accepted; ++it) {  // acceptance is above 0.8 per iteration
      const double u = U.next() - 0.5, v = U.next();
      const double us = 0.5 - fabs(u);
      const double kf = floor((2.0 * a / us + b) * u + c);
      if (kf < 0.0 || kf > nd) continue;
      if (us >= 0.07 && v <= vr) {
        k = uint64_t(kf);
        accepted = true;
        continue;
      }
      const double lv = log(v * alpha / (a / (us * us) + b));
      if (lv <= h - lgamma_stirling(kf + 1.0) - lgamma_stirling(nd - kf + 1.0) + (kf - m) * lpq) {
        k = uint64_t(kf);
        accepted = true;
      }
    }
    if (!accepted) *events |= 1u;
  }
  return flip ? n - k : k;
}

__global__ void binom_kernel(HamView hv, int p, uint64_t seed, uint64_t counter0,
                             const uint64_t* __restrict__ counter_dev, const uint64_t* __restrict__ pre,
                             const uint64_t* __restrict__ cnt, const uint64_t* __restrict__ n_front,
                             const float* __restrict__ logits, uint64_t* __restrict__ child) {
  ANQS_PDL_ENTRY();
  unsigned events = 0;
  const uint64_t nf = *n_front;
  const uint64_t counter = counter0 + (counter_dev ? *counter_dev : 0ull);
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < nf; i += uint64_t(gridDim.x) * blockDim.x) {
    const uint64_t x = pre[i];
    const unsigned pm = slot_mask(hv, p, popc_alpha(x, p), popc_beta(x, p), x), mk = norm_mask(hv, p, pm);
    const float* l = logits + i * 8;
    float m = -INFINITY;
    for (int v = 0; v < 4; ++v)
      if ((mk >> v) & 1u) m = fmaxf(m, l[v]);
    float e[4], s = 0.f;
    for (int v = 0; v < 4; ++v) {
      e[v] = ((mk >> v) & 1u) ? exp_det(__fsub_rn(l[v], m)) : 0.f;
      if ((mk >> v) & 1u) s = __fadd_rn(s, e[v]);
    }
    int last = 3;
    while (last > 0 && !((mk >> last) & 1u)) --last;
    uint64_t rest = cnt[i];
    double tail = 1.0;  // probability mass of the outcomes not split off yet
    for (int v = 0; v < 4; ++v) {
      uint64_t k = 0;
      if ((mk >> v) & 1u) {
        if (v == last) {
          k = rest;
        } else {
          const double pv = double(__fdiv_rn(e[v], s));
          Uniforms U{x, uint64_t(v), uint64_t(p), counter, seed, 0, {0, 0, 0, 0}, 4};
          k = binomial(rest, tail > 0.0 ? fmin(pv / tail, 1.0) : 1.0, U, &events);
          tail -= pv;
        }
      }
      child[i * 4 + v] = ((pm >> v) & 1u) ? k : 0ull;  // DU levels: samples of unphysical children are lost
      rest -= k;
    }
  }
  if (events && hv.status) atomicOr(hv.status, events);
}

__global__ void flag_kernel(const uint64_t* __restrict__ child, const uint64_t* __restrict__ n_front,
                            uint64_t* __restrict__ flags) {
  ANQS_PDL_ENTRY();
  const uint64_t n4 = *n_front * 4;
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < n4; i += uint64_t(gridDim.x) * blockDim.x)
    flags[i] = child[i] ? 1ull : 0ull;
}

__global__ void scatter_kernel(int p, const uint64_t* __restrict__ pre, const uint64_t* __restrict__ child,
                               const uint64_t* __restrict__ n_front, const uint64_t* __restrict__ pos,
                               uint64_t* __restrict__ pre_out, uint64_t* __restrict__ cnt_out) {
  ANQS_PDL_ENTRY();
  const uint64_t n4 = *n_front * 4;
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < n4; i += uint64_t(gridDim.x) * blockDim.x) {
    uint64_t c = child[i];
    if (c) {
      uint64_t j = pos[i];
      pre_out[j] = pre[i >> 2] | (uint64_t(i & 3) << (2 * p));
      cnt_out[j] = c;
    }
  }
}

// ---- one CTA per level for small frontiers ------------------------------------
// Everything after the network evaluation of a level in a single CTA of
// SMALL_T threads: per-node running sums, scan of the draw blocks, draws with
// warp-segment aggregation into shared counters, compaction of the children.
constexpr int SMALL_T = 256;
constexpr int SMALL_F = 2048;  // largest frontier handled this way
constexpr int RUN = 8;         // consecutive nodes or counters per thread in the scans
constexpr size_t SMALL_DYN = size_t(SMALL_T) * 48;  // thresholds and window counts

__device__ __forceinline__ uint32_t block_excl_scan_u32(uint32_t v, uint32_t* sh, uint32_t* tot) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  __syncthreads();
  if (lane == 31) sh[w] = inc;
  __syncthreads();
  if (w == 0) {
    uint32_t t = lane < int(blockDim.x >> 5) ? sh[lane] : 0;
    uint32_t ti = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t u = __shfl_up_sync(0xffffffffu, ti, o);
      if (lane >= o) ti += u;
    }
    sh[lane] = ti - t;
    if (lane == 31) sh[32] = ti;
  }
  __syncthreads();
  *tot = sh[32];
  return sh[w] + inc - v;
}

// One level of the sampler for frontiers of at most SMALL_F nodes (after the
// network has written the slot logits of every frontier prefix):
//   - every CTA scans the per-node draw-block counts in its own shared memory;
//   - for each window of SMALL_T draw blocks the CTA computes, for the nodes
//     the window touches, the masked conditional (split_thresholds) and the
//     integer thresholds T_v = ceil(C_v 2^53) (u < C_v <=> (word >> 11) < T_v);
//   - the draws compare Philox words with the thresholds and add
//     warp-segment sums of the outcome counts to the children;
//   - the last CTA to finish compacts the children, in (node, outcome)
//     order, into the next frontier and clears the counters it used.
// No CTA waits on another.
__global__ void __launch_bounds__(SMALL_T) draw_small_kernel(HamView hv, int p, uint64_t seed, uint64_t counter0,
                                                             const uint64_t* __restrict__ counter_dev,
                                                             const uint64_t* pre, const uint64_t* cnt,
                                                             const uint64_t* n_front,
                                                             const float* __restrict__ logits,
                                                             uint64_t* __restrict__ child, unsigned* __restrict__ done,
                                                             uint64_t* __restrict__ pre_out,
                                                             uint64_t* __restrict__ cnt_out,
                                                             uint64_t* __restrict__ n_out,
                                                             const uint32_t* idx_in,
                                                             uint32_t* __restrict__ idx_out,
                                                             const int32_t* __restrict__ pt_child, int early) {
  __shared__ uint32_t s_scan[SMALL_F + 1];
  extern __shared__ __align__(16) unsigned char s_dyn[];
  uint64_t(*s_thr)[4] = reinterpret_cast<uint64_t(*)[4]>(s_dyn);                  // SMALL_T x 4
  uint32_t(*s_cnt)[4] = reinterpret_cast<uint32_t(*)[4]>(s_dyn + SMALL_T * 32);   // window outcome counts
  __shared__ uint8_t s_mk[SMALL_T];
  __shared__ uint32_t s_red[33];
  __shared__ bool s_last;
  // Prologue (before the wait on the slot-logits kernel, with `early`): the
  // frontier and its counts were written two kernels back (the previous
  // level's split, or the initial/shard kernel), so the node offsets can be
  // scanned while the logits kernel finishes.  Without `early` (prefix-table
  // mode, where the previous kernel is the previous level's split itself)
  // the scan waits for the previous kernel first.
  // The frontier is read through L2 (__ldcg), never through the read-only
  // cache: in prefix-table mode it was written by the kernel just before
  // this one, which may still have been running when this grid started.
  if (!early) ANQS_PDL_WAIT();
  const int nf = int(__ldcg(n_front));
  const int lane = threadIdx.x & 31;
  // draw-block offsets of the nodes: each thread scans a run of RUN
  // consecutive nodes (their counts loaded together), one block scan per
  // RUN * SMALL_T nodes
  uint32_t carry = 0;
  for (int base = 0; base < nf; base += RUN * SMALL_T) {
    const int i0 = base + RUN * threadIdx.x;
    uint32_t nb[RUN], mine = 0;
#pragma unroll
    for (int e = 0; e < RUN; ++e) {
      nb[e] = i0 + e < nf ? uint32_t((__ldcg(cnt + i0 + e) + 3) / 4) : 0u;
      mine += nb[e];
    }
    uint32_t tot;
    uint32_t off = carry + block_excl_scan_u32(mine, s_red, &tot);
#pragma unroll
    for (int e = 0; e < RUN; ++e)
      if (i0 + e < nf) {
        s_scan[i0 + e] = off;
        off += nb[e];
      }
    carry += tot;
  }
  if (threadIdx.x == 0) s_scan[nf] = carry;
  ANQS_PDL_WAIT();
  ANQS_PDL_TRIGGER();
  const uint64_t counter = counter0 + (counter_dev ? *counter_dev : 0ull);
  __syncthreads();
  const uint32_t total = carry;
  auto node_of = [&](uint32_t t) {
    int lo = 0, hi = nf - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (s_scan[mid] <= t) lo = mid;
      else hi = mid - 1;
    }
    return lo;
  };
  for (uint32_t t0 = blockIdx.x * SMALL_T; t0 < total; t0 += gridDim.x * SMALL_T) {
    const uint32_t t_end = min(total, t0 + SMALL_T);
    const int n_lo = node_of(t0), n_hi = node_of(t_end - 1);
    __syncthreads();  // previous window's thresholds are no longer read
    if (threadIdx.x <= n_hi - n_lo) {
      const int i = n_lo + threadIdx.x;
      for (int v = 0; v < 4; ++v) s_cnt[threadIdx.x][v] = 0;
      const uint64_t x = __ldcg(pre + i);
      const unsigned pm = slot_mask(hv, p, popc_alpha(x, p), popc_beta(x, p), x), mk = norm_mask(hv, p, pm);
      // prefix-table mode: the node's logits sit at its table row
      const uint64_t row = idx_in ? uint64_t(__ldcg(idx_in + i)) : uint64_t(i);
      split_thresholds(logits + row * 8, mk, s_thr[threadIdx.x]);
      s_mk[threadIdx.x] = uint8_t(mk | (pm << 4));
    }
    __syncthreads();
    const uint32_t t = t0 + threadIdx.x;
    int node = -1;
    uint32_t packed = 0;
    if (t < t_end) {
      node = node_of(t);
      const int li = node - n_lo;
      const uint64_t ib = t - s_scan[node];
      const uint64_t c = __ldcg(cnt + node);
      uint64_t w[4];
      Philox::block(__ldcg(pre + node), ib, uint64_t(p), counter, seed, 0ull, w);
      const unsigned mk = s_mk[li] & 0xFu, pm = s_mk[li] >> 4;
      int last = 3;
      while (last > 0 && !((mk >> last) & 1u)) --last;
      for (int k = 0; k < 4; ++k) {
        if (ib * 4 + k >= c) break;
        const int v = draw_outcome(w[k], s_thr[li], mk, last);
        if ((pm >> v) & 1u) packed += 1u << (8 * v);
      }
    }
    const int prev = __shfl_up_sync(0xffffffffu, node, 1);
    const unsigned heads = __ballot_sync(0xffffffffu, lane == 0 || prev != node);
    const int seg_start = 31 - __clz(heads & ((2u << lane) - 1u));
    uint32_t v = packed;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t other = __shfl_up_sync(0xffffffffu, v, o);
      if (lane - o >= seg_start) v += other;
    }
    const bool tail = (lane == 31) || ((heads >> (lane + 1)) & 1u);
    if (tail && node >= 0)
      for (int k = 0; k < 4; ++k) {
        const uint32_t ck = (v >> (8 * k)) & 0xffu;
        if (ck) atomicAdd(&s_cnt[node - n_lo][k], ck);
      }
    __syncthreads();
    // one global atomic per (node, outcome) and window
    if (threadIdx.x <= n_hi - n_lo)
      for (int k = 0; k < 4; ++k) {
        const uint32_t ck = s_cnt[threadIdx.x][k];
        if (ck)
          atomicAdd(reinterpret_cast<unsigned long long*>(child + uint64_t(n_lo + threadIdx.x) * 4 + k),
                    (unsigned long long)ck);
      }
  }
  // last CTA: compaction (the other CTAs' counts are visible after their fence)
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = (atomicAdd(done, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // children in (node, outcome) order: runs of RUN consecutive counters per
  // thread, loaded together, one block scan per RUN * SMALL_T counters
  carry = 0;
  for (int base = 0; base < 4 * nf; base += RUN * SMALL_T) {
    const int i0 = base + RUN * threadIdx.x;
    uint64_t c[RUN];
    uint32_t mine = 0;
#pragma unroll
    for (int e = 0; e < RUN; ++e) {
      c[e] = i0 + e < 4 * nf ? __ldcg(child + i0 + e) : 0ull;
      mine += c[e] ? 1u : 0u;
    }
    uint32_t tot;
    uint32_t off = carry + block_excl_scan_u32(mine, s_red, &tot);
#pragma unroll
    for (int e = 0; e < RUN; ++e)
      if (c[e]) {
        const int i = i0 + e;
        pre_out[off] = __ldcg(pre + (i >> 2)) | (uint64_t(i & 3) << (2 * p));
        cnt_out[off] = c[e];
        if (idx_out) idx_out[off] = uint32_t(pt_child[uint64_t(__ldcg(idx_in + (i >> 2))) * 4 + (i & 3)]);
        ++off;
      }
    carry += tot;
  }
  __syncthreads();
  // clear the counters of the next level's nodes
  for (uint32_t i = threadIdx.x; i < 4 * carry; i += SMALL_T) child[i] = 0;
  if (threadIdx.x == 0) {
    *n_out = carry;
    *done = 0;
  }
}

// ---- every level in one persistent launch (prefix-table mode) -----------------
// The grid is co-resident (cooperative launch) and passes one grid-wide
// barrier per level.  Each CTA keeps its own copy of the frontier (prefix,
// count, table row) in shared memory: after the barrier of level p every CTA
// reads the child counters of level p and compacts them into its copy of
// the level-(p+1) frontier, so no frontier goes through global memory and no
// CTA waits for another's compaction.  The child counters rotate over three
// buffers: level p adds into buffer p % 3 and, before its barrier, the grid
// clears buffer (p + 1) % 3, which every CTA finished reading before the
// barrier of level p - 1 (level 0's counters and the barrier are cleared by
// the prefix-table slot launch before this one).  The draws and their order
// are those of draw_small_kernel, so the samples are the same bit for bit.
//
// When the table has at most kStageRows rows, every CTA first stages, for
// every row, the split thresholds of its conditional, its outcome masks and
// its children's rows in shared memory (the masks and children before the
// programmatic-dependency wait, the thresholds from the slot outputs after
// it), so that a level reads nothing from global memory but the child counts
// after its barrier.
constexpr int PER_F = 2048;                          // largest frontier (the prefix table's level bound)
constexpr size_t PER_DYN = size_t(2) * PER_F * (8 + 4 + 4)   // frontier copies: prefix, count, table row
                           + size_t(PER_F + 1) * 4            // draw-block offsets
                           + size_t(SMALL_T) * (32 + 16);     // window thresholds and counts
constexpr int kStageRows = 1024;
constexpr size_t STAGE_DYN = size_t(kStageRows) * (32 + 16 + 1);  // thresholds, child rows, masks
constexpr uint64_t kBarrierNs = 2000000000ull;

// The grid barrier's arrival target (gridDim.x + extra) and time limit.  extra
// is 0 and the limit kBarrierNs except under anqs_test_sampler_barrier, which
// makes every barrier wait for an arrival that never comes.
struct BarrierCfg {
  unsigned extra;
  uint64_t limit_ns;
};
BarrierCfg g_barrier_cfg{0u, kBarrierNs};

struct LevelOffsets {
  uint32_t off[ANQS_MAX_ORB + 1];  // table rows of level p: [off[p], off[p + 1])
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Barrier of level p over the co-resident grid: thread 0 of every CTA makes
// the CTA's writes visible and adds one to the level's arrival counter, then
// polls it until every CTA has arrived (bounded by kBarrierNs, after which it
// sets the error word and every CTA leaves).  Writes before the barrier are
// visible to every CTA after it.
__device__ bool level_barrier(GridBarrier* gb, int p, int* s_ok, const BarrierCfg& bc) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    asm volatile("red.relaxed.gpu.global.add.u32 [%0], 1;" ::"l"(&gb->arrive[p]) : "memory");
    int ok = 1;
    const unsigned target = gridDim.x + bc.extra;
    if (ld_acquire_u32(&gb->arrive[p]) < target) {
      const uint64_t t0 = gtimer();
      while (ld_acquire_u32(&gb->arrive[p]) < target) {
        if (*reinterpret_cast<volatile int*>(&gb->err) || gtimer() - t0 > bc.limit_ns) {
          atomicExch(&gb->err, 1);
          ok = 0;
          break;
        }
        __nanosleep(32);
      }
    }
    *s_ok = ok && !*reinterpret_cast<volatile int*>(&gb->err);
  }
  __syncthreads();
  return *s_ok != 0;
}

__global__ void __launch_bounds__(SMALL_T) sample_levels_kernel(HamView hv, int n, uint64_t n_samples, uint64_t seed,
                                                                uint64_t counter0, const uint64_t* counter_dev,
                                                                const float* logits, const uint64_t* pt_x,
                                                                const int32_t* pt_child, LevelOffsets lvo,
                                                                int staged, uint64_t* child, uint64_t child_stride,
                                                                GridBarrier* gb, uint64_t* __restrict__ x_out,
                                                                uint64_t* __restrict__ n_out,
                                                                uint64_t* __restrict__ n_unique, int* status,
                                                                BarrierCfg bc) {
  extern __shared__ __align__(16) unsigned char s_dyn[];
  uint64_t* fr_pre = reinterpret_cast<uint64_t*>(s_dyn);                        // [2][PER_F]
  uint32_t* fr_cnt = reinterpret_cast<uint32_t*>(fr_pre + 2 * PER_F);            // [2][PER_F]
  uint32_t* fr_idx = fr_cnt + 2 * PER_F;                                         // [2][PER_F]
  uint32_t* s_scan = fr_idx + 2 * PER_F;                                         // [PER_F + 1]
  uint64_t(*s_thr)[4] = reinterpret_cast<uint64_t(*)[4]>(s_scan + PER_F + 4);    // [SMALL_T][4]
  uint32_t(*s_cnt)[4] = reinterpret_cast<uint32_t(*)[4]>(s_thr + SMALL_T);       // [SMALL_T][4]
  uint64_t(*st_thr)[4] = reinterpret_cast<uint64_t(*)[4]>(s_cnt + SMALL_T);      // staged: [kStageRows][4]
  int32_t(*st_child)[4] = reinterpret_cast<int32_t(*)[4]>(st_thr + kStageRows);  // staged: [kStageRows][4]
  uint8_t* st_mk = reinterpret_cast<uint8_t*>(st_child + kStageRows);           // staged: [kStageRows]
  __shared__ uint8_t s_mk[SMALL_T];
  __shared__ uint32_t s_red[33];
  __shared__ int s_ok;
  __shared__ uint32_t s_off[ANQS_MAX_ORB + 1];
  if (threadIdx.x <= n) s_off[threadIdx.x] = lvo.off[threadIdx.x];
  __syncthreads();
  const int n_rows = int(s_off[n]);
  if (staged) {  // rows' masks and children: fixed by the Hamiltonian
    for (int r = threadIdx.x; r < n_rows; r += SMALL_T) {
      int p = 0;
      while (p + 1 < n && uint32_t(r) >= s_off[p + 1]) ++p;
      const uint64_t x = pt_x[r];
      const unsigned pm = slot_mask(hv, p, popc_alpha(x, p), popc_beta(x, p), x), mk = norm_mask(hv, p, pm);
      st_mk[r] = uint8_t(mk | (pm << 4));
      for (int v = 0; v < 4; ++v) st_child[r][v] = pt_child[uint64_t(r) * 4 + v];
    }
  }
  ANQS_PDL_WAIT();  // the prefix table's logits and the cleared counters come from the kernels before
  if (staged) {  // rows' split thresholds from the slot outputs just written
    __syncthreads();
    // all of a thread's rows' outputs are loaded before any is used (one L2
    // round trip instead of one per row): at most kStageRows / SMALL_T rows
    constexpr int RPT = kStageRows / SMALL_T;
    float4 l4[RPT];
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
      const int r = threadIdx.x + k * SMALL_T;
      l4[k] = r < n_rows ? __ldcg(reinterpret_cast<const float4*>(logits + uint64_t(r) * 8)) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
      const int r = threadIdx.x + k * SMALL_T;
      if (r < n_rows) {
        const float l[4] = {l4[k].x, l4[k].y, l4[k].z, l4[k].w};
        split_thresholds(l, st_mk[r] & 0xFu, st_thr[r]);
      }
    }
  }
  const int lane = threadIdx.x & 31;
  const uint64_t counter = counter0 + (counter_dev ? *counter_dev : 0ull);
  if (threadIdx.x == 0) {
    fr_pre[0] = 0;
    fr_cnt[0] = uint32_t(n_samples);
    fr_idx[0] = 0;
  }
  int nf = 1;
  bool ok = true;
  for (int p = 0; p < n && ok; ++p) {
    const int cur = p & 1, nxt = cur ^ 1;
    const uint64_t* pre = fr_pre + cur * PER_F;
    const uint32_t* cnt = fr_cnt + cur * PER_F;
    const uint32_t* idx = fr_idx + cur * PER_F;
    uint64_t* ch = child + uint64_t(p % 3) * child_stride;
    // clear the counters of level p + 1 (last read before the barrier of level p - 1)
    {
      uint64_t* nc = child + uint64_t((p + 1) % 3) * child_stride;
      for (uint64_t i = blockIdx.x * uint64_t(SMALL_T) + threadIdx.x; i < child_stride;
           i += uint64_t(gridDim.x) * SMALL_T)
        nc[i] = 0;
    }
    __syncthreads();  // this level's frontier copy is complete
    if (p == n - 1) {
      // The last slot: where every node has a single allowed outcome (always
      // so under MU masking, the electron counts fix the last orbital) every
      // draw goes to it, so the children are the nodes with that outcome and
      // their counts: written without draws or a barrier, in the order the
      // split would emit them.
      bool forced = true;
      for (int i = threadIdx.x; i < nf; i += SMALL_T) {
        unsigned mkb;
        if (staged) {
          mkb = st_mk[idx[i]];
        } else {
          const uint64_t x = pre[i];
          const unsigned pm = slot_mask(hv, p, popc_alpha(x, p), popc_beta(x, p), x);
          mkb = norm_mask(hv, p, pm) | (pm << 4);
        }
        if (__popc(mkb & 0xFu) != 1 || !((mkb >> 4) & mkb & 0xFu)) forced = false;
      }
      if (__syncthreads_and(forced)) {
        if (blockIdx.x == 0) {
          for (int i = threadIdx.x; i < nf; i += SMALL_T) {
            const unsigned mk = staged ? st_mk[idx[i]] & 0xFu
                                       : norm_mask(hv, p, slot_mask(hv, p, popc_alpha(pre[i], p),
                                                                    popc_beta(pre[i], p), pre[i]));
            x_out[i] = pre[i] | (uint64_t(__ffs(mk) - 1) << (2 * p));
            n_out[i] = cnt[i];
          }
          if (threadIdx.x == 0) *n_unique = uint64_t(nf);
        }
        break;
      }
    }
    // draw-block offsets of the nodes
    uint32_t carry = 0;
    for (int base = 0; base < nf; base += RUN * SMALL_T) {
      const int i0 = base + RUN * threadIdx.x;
      uint32_t nb[RUN], mine = 0;
#pragma unroll
      for (int e = 0; e < RUN; ++e) {
        nb[e] = i0 + e < nf ? (cnt[i0 + e] + 3u) / 4u : 0u;
        mine += nb[e];
      }
      uint32_t tot;
      uint32_t off = carry + block_excl_scan_u32(mine, s_red, &tot);
#pragma unroll
      for (int e = 0; e < RUN; ++e)
        if (i0 + e < nf) {
          s_scan[i0 + e] = off;
          off += nb[e];
        }
      carry += tot;
    }
    if (threadIdx.x == 0) s_scan[nf] = carry;
    __syncthreads();
    const uint32_t total = carry;
    auto node_of = [&](uint32_t t) {
      int lo = 0, hi = nf - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (s_scan[mid] <= t) lo = mid;
        else hi = mid - 1;
      }
      return lo;
    };
    for (uint32_t t0 = blockIdx.x * SMALL_T; t0 < total; t0 += gridDim.x * SMALL_T) {
      const uint32_t t_end = min(total, t0 + SMALL_T);
      const int n_lo = node_of(t0), n_hi = node_of(t_end - 1);
      __syncthreads();  // previous window's thresholds are no longer read
      if (threadIdx.x <= n_hi - n_lo) {
        const int i = n_lo + threadIdx.x;
        for (int v = 0; v < 4; ++v) s_cnt[threadIdx.x][v] = 0;
        if (!staged) {
          const uint64_t x = pre[i];
          const unsigned pm = slot_mask(hv, p, popc_alpha(x, p), popc_beta(x, p), x), mk = norm_mask(hv, p, pm);
          float l[4];
          for (int v = 0; v < 4; ++v) l[v] = __ldcg(logits + uint64_t(idx[i]) * 8 + v);
          split_thresholds(l, mk, s_thr[threadIdx.x]);
          s_mk[threadIdx.x] = uint8_t(mk | (pm << 4));
        }
      }
      __syncthreads();
      const uint32_t t = t0 + threadIdx.x;
      int node = -1;
      uint32_t packed = 0;
      if (t < t_end) {
        node = node_of(t);
        const int li = node - n_lo;
        const uint64_t ib = t - s_scan[node];
        const uint64_t c = cnt[node];
        uint64_t w[4];
        Philox::block(pre[node], ib, uint64_t(p), counter, seed, 0ull, w);
        const uint32_t row = idx[node];
        const unsigned mkb = staged ? st_mk[row] : s_mk[li];
        const uint64_t* thr = staged ? st_thr[row] : s_thr[li];
        const unsigned mk = mkb & 0xFu, pm = mkb >> 4;
        int last = 3;
        while (last > 0 && !((mk >> last) & 1u)) --last;
        for (int k = 0; k < 4; ++k) {
          if (ib * 4 + k >= c) break;
          const int v = draw_outcome(w[k], thr, mk, last);
          if ((pm >> v) & 1u) packed += 1u << (8 * v);
        }
      }
      const int prev = __shfl_up_sync(0xffffffffu, node, 1);
      const unsigned heads = __ballot_sync(0xffffffffu, lane == 0 || prev != node);
      const int seg_start = 31 - __clz(heads & ((2u << lane) - 1u));
      uint32_t v = packed;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t other = __shfl_up_sync(0xffffffffu, v, o);
        if (lane - o >= seg_start) v += other;
      }
      const bool tail = (lane == 31) || ((heads >> (lane + 1)) & 1u);
      if (tail && node >= 0)
        for (int k = 0; k < 4; ++k) {
          const uint32_t ck = (v >> (8 * k)) & 0xffu;
          if (ck) atomicAdd(&s_cnt[node - n_lo][k], ck);
        }
      __syncthreads();
      if (threadIdx.x <= n_hi - n_lo)
        for (int k = 0; k < 4; ++k) {
          const uint32_t ck = s_cnt[threadIdx.x][k];
          if (ck)
            atomicAdd(reinterpret_cast<unsigned long long*>(ch + uint64_t(n_lo + threadIdx.x) * 4 + k),
                      (unsigned long long)ck);
        }
    }
    // every CTA's counts of level p are in `ch`
    ok = level_barrier(gb, p, &s_ok, bc);
    if (!ok) break;
    // children in (node, outcome) order -> this CTA's copy of the next frontier
    // (the last level: the output, written by CTA 0)
    const bool last = (p == n - 1);
    carry = 0;
    for (int base = 0; base < 4 * nf; base += RUN * SMALL_T) {
      const int i0 = base + RUN * threadIdx.x;
      uint64_t c[RUN];
      uint32_t mine = 0;
#pragma unroll
      for (int e = 0; e < RUN; ++e) {
        c[e] = i0 + e < 4 * nf ? __ldcg(ch + i0 + e) : 0ull;
        mine += c[e] ? 1u : 0u;
      }
      uint32_t tot;
      uint32_t off = carry + block_excl_scan_u32(mine, s_red, &tot);
#pragma unroll
      for (int e = 0; e < RUN; ++e)
        if (c[e]) {
          const int i = i0 + e;
          const uint64_t xc = pre[i >> 2] | (uint64_t(i & 3) << (2 * p));
          if (!last) {
            if (off < uint32_t(PER_F)) {
              fr_pre[nxt * PER_F + off] = xc;
              fr_cnt[nxt * PER_F + off] = uint32_t(c[e]);
              fr_idx[nxt * PER_F + off] =
                  uint32_t(staged ? st_child[idx[i >> 2]][i & 3] : pt_child[uint64_t(idx[i >> 2]) * 4 + (i & 3)]);
            }
          } else if (blockIdx.x == 0) {
            x_out[off] = xc;
            n_out[off] = c[e];
          }
          ++off;
        }
      carry += tot;
    }
    if (last && blockIdx.x == 0 && threadIdx.x == 0) *n_unique = carry;
    if (!last && carry > uint32_t(PER_F)) {  // cannot happen with the prefix table's level bound
      if (threadIdx.x == 0) atomicExch(&gb->err, 1);
      ok = false;
    }
    nf = int(carry);
  }
  if (threadIdx.x == 0 && *reinterpret_cast<volatile int*>(&gb->err)) {
    atomicExch(status, 1);
    if (blockIdx.x == 0) *n_unique = 0;  // a pass that gave up returns no samples
  }
}


// and in place (one CTA, chunk by chunk: each chunk is read before any of
// its compacted entries is written).
__global__ void __launch_bounds__(SMALL_T) shard_kernel(uint64_t* __restrict__ pre, uint64_t* __restrict__ cnt,
                                                        uint64_t* __restrict__ n_list, int rank, int world) {
  ANQS_PDL_ENTRY();
  __shared__ uint32_t s_red[33];
  const uint64_t nf = *n_list;
  uint64_t carry = 0;
  for (uint64_t base = 0; base < nf; base += SMALL_T) {
    const uint64_t i = base + threadIdx.x;
    const bool keep = i < nf && (i % uint64_t(world)) == uint64_t(rank);
    const uint64_t x = keep ? pre[i] : 0ull, c = keep ? cnt[i] : 0ull;
    uint32_t tot;
    const uint32_t ex = block_excl_scan_u32(keep ? 1u : 0u, s_red, &tot);  // synchronises the CTA
    if (keep) {
      pre[carry + ex] = x;
      cnt[carry + ex] = c;
    }
    carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) *n_list = carry;
}

struct Plan {
  uint64_t F;  // max frontier
  uint64_t *pre[2], *cnt[2], *nblk, *nblk_scan, *child, *flags, *pos, *partial, *n_front;
  float* logits;
  float* plog;         // prefix-table mode: slot outputs of every table row [rows][8]
  uint32_t* idx[2];    // prefix-table mode: table row of each frontier node
  GridBarrier* barrier;  // prefix-table mode: the persistent launch's grid barrier
  uint64_t* thr;
  uint8_t* allowed;
  unsigned* done;
};

uint64_t level_cap(const anqs_ham* H, uint64_t n_samples, int p) {
  uint64_t c = H->phys_prefix[p];
  return c < n_samples ? c : n_samples;
}

void plan_ws(const anqs_ham* H, uint64_t n_samples, Arena& A, Plan& P) {
  uint64_t F = 1;
  for (int p = 0; p <= H->v.n; ++p) F = std::max(F, level_cap(H, n_samples, p));
  P.F = F;
  for (int b = 0; b < 2; ++b) {
    P.pre[b] = A.take<uint64_t>(F);
    P.cnt[b] = A.take<uint64_t>(F);
  }
  P.logits = A.take<float>(F * 8);
  P.thr = A.take<uint64_t>(F * 4);
  P.allowed = A.take<uint8_t>(F);
  P.nblk = A.take<uint64_t>(F);
  P.nblk_scan = A.take<uint64_t>(F + 1);
  P.child = A.take<uint64_t>(F * 4 * (H->pt_x.empty() ? 1 : 3));  // prefix-table mode: three rotating buffers
  P.flags = A.take<uint64_t>(F * 4);
  P.pos = A.take<uint64_t>(F * 4 + 1);
  P.partial = A.take<uint64_t>((F * 4 + 1) / SCAN_CHUNK + 2);
  P.n_front = A.take<uint64_t>(2);
  P.done = A.take<unsigned>(1);
  const uint64_t rows = H->pt_x.size();
  P.plog = rows ? A.take<float>(rows * 8) : nullptr;
  for (int b = 0; b < 2; ++b) P.idx[b] = rows ? A.take<uint32_t>(F) : nullptr;
  P.barrier = rows ? A.take<GridBarrier>(1) : nullptr;
}

int scan(const uint64_t* in, const uint64_t* n_dev, uint64_t mult, uint64_t max_n, uint64_t* partial,
         uint64_t* out, uint64_t* total_dev, cudaStream_t s) {
  uint64_t chunks = max_n / SCAN_CHUNK + 1;  // covers index max_n (the total)
  ANQS_CUDA_LAUNCH("scan_reduce_kernel", launch_k(scan_reduce_kernel, dim3(unsigned(chunks)), dim3(SCAN_T), 0, s, in, n_dev, mult, partial));
  ANQS_CUDA_LAUNCH("scan_partials_kernel", launch_k(scan_partials_kernel, dim3(1), dim3(SCAN_T), 0, s, partial, chunks));
  ANQS_CUDA_LAUNCH("scan_apply_kernel", launch_k(scan_apply_kernel, dim3(unsigned(chunks)), dim3(SCAN_T), 0, s, in, n_dev, mult, partial, out, total_dev));
  return ANQS_OK;
}

unsigned blocks_for(uint64_t n, int threads, uint64_t cap) {
  uint64_t b = (n + threads - 1) / threads;
  if (b > cap) b = cap;
  return unsigned(b ? b : 1);
}

}  // namespace

size_t sampler_workspace(const anqs_ham* H, uint64_t n_samples) {
  Arena A(nullptr, 0);
  Plan P;
  plan_ws(H, n_samples, A, P);
  return A.off;
}

int run_sampler(const anqs_model* M, const anqs_ham* H, uint64_t n_samples, uint64_t seed, uint64_t counter,
                const uint64_t* counter_dev, uint64_t* x_out, uint64_t* n_out, uint64_t* n_unique, void* ws,
                size_t ws_bytes, cudaStream_t s, int rank, int world, int split_level, bool binom) {
  Arena A(ws, ws_bytes);
  Plan P;
  plan_ws(H, n_samples, A, P);
  if (!A.fits()) return set_error(ANQS_ERR_CAPACITY, "sampler workspace needs %zu bytes", A.off);
  const int n = H->v.n;
  // Prefix-table mode (BF16 MLP, small sectors, multinomial splits on one
  // rank): the network's slot outputs of every physical prefix of every level
  // in one launch, then per level only the split; the frontier carries each
  // node's table row.  The draws and their order are those of the per-level
  // path, so the samples are the same bit for bit.
  const bool table = !binom && world == 1 && P.plog && M->d.kind == ANQS_MODEL_MLP &&
                     M->d.form == ANQS_FORM_BF16 && n_samples < (1ull << 31);
  // all levels in one cooperative launch when its CTAs can all be resident
  // (one CTA per SM at most, each CTA one window of draw blocks per round);
  // rows' thresholds, masks and children staged in shared memory when they fit
  LevelOffsets lvo{};
  int staged = 0, occ = 0, sms = 0;
  size_t dyn = 0;
  if (table) {
    for (int q = 0; q <= n; ++q) lvo.off[q] = H->pt_off[q];
    staged = H->pt_off[n] <= uint32_t(kStageRows) ? 1 : 0;
    dyn = PER_DYN + (staged ? STAGE_DYN : 0);
    ANQS_CUDA(cudaFuncSetAttribute(sample_levels_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(dyn)));
    ANQS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, sample_levels_kernel, SMALL_T, dyn));
    int dev = 0;
    ANQS_CUDA(cudaGetDevice(&dev));
    ANQS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  }
  const bool persistent = table && occ >= 1;
  if (!persistent) {
    ProfScope ps(PROF_SAMPLER, s);
    ANQS_CUDA_LAUNCH("sampler init_kernel", launch_k(init_kernel, dim3(1), dim3(1), 0, s, P.pre[0], P.cnt[0], P.n_front, n_samples, P.done, P.child, P.idx[0], reinterpret_cast<int*>(P.barrier)));
  }
  if (table) {
    // the persistent kernel needs only its grid barrier and the first
    // level's child counters cleared: the slot launch before it does that
    // instead of the initial kernel
    ZeroWords z{};
    if (persistent) {
      z.p[0] = reinterpret_cast<uint32_t*>(P.barrier);
      z.n[0] = kBarrierWords;
      z.p[1] = reinterpret_cast<uint32_t*>(P.child);
      z.n[1] = 8;  // child[0..3], uint64
    }
    ANQS_TRY(launch_mlp_tc_prefix_logits(M, H, P.plog, s, z));
    if (persistent) {
      uint64_t F = 1;
      for (int q = 0; q <= n; ++q) F = std::max(F, level_cap(H, n_samples, q));
      const unsigned grid = blocks_for(((n_samples + 3) / 4 + F + SMALL_T - 1) / SMALL_T, 1, uint64_t(sms));
      int* status = reinterpret_cast<int*>(static_cast<unsigned char*>(M->packed) + M->pack_off[n]);
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(grid);
      cfg.blockDim = dim3(SMALL_T);
      cfg.dynamicSmemBytes = dyn;
      cfg.stream = s;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeCooperative;
      attr[0].val.cooperative = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      ProfScope ps(PROF_SAMPLER, s);
      note_launch();
      ANQS_CUDA_LAUNCH("sampler sample_levels_kernel",
                       cudaLaunchKernelEx(&cfg, sample_levels_kernel, H->v, n, n_samples, seed, counter, counter_dev,
                                          static_cast<const float*>(P.plog), static_cast<const uint64_t*>(H->d_pt_x),
                                          static_cast<const int32_t*>(H->d_pt_child), lvo, staged, P.child, F * 4,
                                          P.barrier, x_out, n_out, n_unique, status, g_barrier_cfg));
      return ANQS_OK;
    }
  }
  bool prev_large = false;
  for (int p = 0; p < n; ++p) {
    const int cur = p & 1, nxt = cur ^ 1;
    const uint64_t Fp = level_cap(H, n_samples, p);
    uint64_t* nf = P.n_front + cur;
    if (world > 1 && p == split_level) {
      // shard: this rank continues from its share of the level-p frontier
      ProfScope ps(PROF_SAMPLER, s);
      ANQS_CUDA_LAUNCH("sampler shard_kernel",
                       launch_k(shard_kernel, dim3(1), dim3(SMALL_T), 0, s, P.pre[cur], P.cnt[cur], nf, rank, world));
    }
    if (!table) ANQS_TRY(logits_dispatch(M, H, p, P.pre[cur], nf, Fp, P.logits, s));
    ProfScope ps(PROF_SAMPLER, s);
    const bool last = (p == n - 1);
    if (binom) {
      ANQS_CUDA_LAUNCH("sampler binom_kernel", launch_k(binom_kernel, dim3(blocks_for(Fp, 128, 152 * 8)), dim3(128), 0, s, H->v, p, seed, counter, counter_dev, P.pre[cur], P.cnt[cur], nf, P.logits, P.child));
      ANQS_CUDA_LAUNCH("sampler flag_kernel", launch_k(flag_kernel, dim3(blocks_for(Fp * 4, 256, 152 * 8)), dim3(256), 0, s, P.child, nf, P.flags));
      uint64_t* nf_next = last ? n_unique : P.n_front + nxt;
      ANQS_TRY(scan(P.flags, nf, 4, Fp * 4, P.partial, P.pos, nf_next, s));
      ANQS_CUDA_LAUNCH("sampler scatter_kernel", launch_k(scatter_kernel, dim3(blocks_for(Fp * 4, 256, 152 * 8)), dim3(256), 0, s, p, P.pre[cur], P.child, nf, P.pos, last ? x_out : P.pre[nxt], last ? n_out : P.cnt[nxt]));
      continue;
    }
    const bool small = (Fp <= uint64_t(SMALL_F) && n_samples < (1ull << 31)) || table;
    if (small && prev_large) {
      // the multi-kernel path leaves its counters set; the small path expects them cleared
      ANQS_CUDA(cudaMemsetAsync(P.child, 0, Fp * 4 * sizeof(uint64_t), s));
    }
    prev_large = !small;
    if (small) {
      const uint64_t blocks = ((n_samples + 3) / 4 + Fp + SMALL_T - 1) / SMALL_T;
      ANQS_CUDA(cudaFuncSetAttribute(draw_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(SMALL_DYN)));
      ANQS_CUDA_LAUNCH("sampler draw_small_kernel", launch_k(draw_small_kernel, dim3(blocks_for(blocks, 1, 152)), dim3(SMALL_T), SMALL_DYN, s, H->v, p, seed, counter, counter_dev, P.pre[cur], P.cnt[cur], nf, table ? P.plog : P.logits, P.child, P.done, last ? x_out : P.pre[nxt], last ? n_out : P.cnt[nxt], last ? n_unique : P.n_front + nxt, table ? P.idx[cur] : nullptr, table && !last ? P.idx[nxt] : nullptr, H->d_pt_child, (table && p > 0) ? 0 : 1));
      continue;
    }
    ANQS_CUDA_LAUNCH("sampler prep_kernel", launch_k(prep_kernel, dim3(blocks_for(Fp, 256, 152 * 8)), dim3(256), 0, s, H->v, p, P.pre[cur], P.cnt[cur], nf, P.logits, P.thr, P.allowed, P.nblk, P.child));
    ANQS_TRY(scan(P.nblk, nf, 1, Fp, P.partial, P.nblk_scan, nullptr, s));
    const uint64_t max_draw_threads = (n_samples + 3) / 4 + Fp;
    ANQS_CUDA_LAUNCH("sampler draw_kernel", launch_k(draw_kernel, dim3(blocks_for(max_draw_threads, 256, 152 * 16)), dim3(256), 0, s, p, seed, counter, counter_dev, P.pre[cur], P.cnt[cur], nf, P.nblk_scan, P.thr, P.allowed, P.child, max_draw_threads));
    ANQS_CUDA_LAUNCH("sampler flag_kernel", launch_k(flag_kernel, dim3(blocks_for(Fp * 4, 256, 152 * 8)), dim3(256), 0, s, P.child, nf, P.flags));
    uint64_t* nf_next = last ? n_unique : P.n_front + nxt;
    ANQS_TRY(scan(P.flags, nf, 4, Fp * 4, P.partial, P.pos, nf_next, s));
    ANQS_CUDA_LAUNCH("sampler scatter_kernel", launch_k(scatter_kernel, dim3(blocks_for(Fp * 4, 256, 152 * 8)), dim3(256), 0, s, p, P.pre[cur], P.child, nf, P.pos, last ? x_out : P.pre[nxt], last ? n_out : P.cnt[nxt]));
  }
  if (world > 1 && split_level == n) {
    ProfScope ps(PROF_SAMPLER, s);
    ANQS_CUDA_LAUNCH("sampler shard_kernel",
                     launch_k(shard_kernel, dim3(1), dim3(SMALL_T), 0, s, x_out, n_out, n_unique, rank, world));
  }
  return ANQS_OK;
}

int logits_dispatch(const anqs_model* M, const anqs_ham* H, int p, const uint64_t* pre, const uint64_t* n_dev,
                    uint64_t max_rows, float* out8, cudaStream_t s) {
  switch (M->d.kind) {
    case ANQS_MODEL_MLP:
      if (M->d.form == ANQS_FORM_BF16)
        return launch_mlp_tc_slot_logits(M, H->v, p, pre, n_dev, max_rows, out8, s);
      return launch_mlp_fp32_slot_logits(M->mlp, p, pre, n_dev, max_rows, out8, s);
    case ANQS_MODEL_TF:
      if (M->d.form == ANQS_FORM_BF16) return launch_tf_tc_slot_logits(M, p, pre, n_dev, max_rows, out8, s);
      return launch_tf_fp32_slot_logits(M->tf, p, pre, n_dev, max_rows, out8, s);
    case ANQS_MODEL_TABLE:
      return launch_table_slot_logits(M, p, pre, n_dev, max_rows, out8, s);
    case ANQS_MODEL_NADE:
      return launch_nade_slot_logits(M->nade, H->v, p, pre, n_dev, max_rows, out8, s);
    default:
      return set_error(ANQS_ERR_UNSUPPORTED, "sampling for model kind %d not supported by this library", M->d.kind);
  }
}

void sampler_test_barrier(unsigned extra_arrivals, uint64_t limit_ns) {
  g_barrier_cfg.extra = extra_arrivals;
  g_barrier_cfg.limit_ns = limit_ns ? limit_ns : kBarrierNs;
}

}  // namespace anqs
