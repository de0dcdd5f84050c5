// 16-bit tensor-core form of the per-slot MLP ansatz (tcgen05 MMA, TMEM
// accumulators, bulk-copied weight images), with reuse of the parent
// determinant's slots for its connected determinants.
//
// Operands are fp16 (kind::f16, the rate of bf16): the weights are rounded to
// an 11-bit significand instead of 8, and so are the hidden activations (tanh
// values in [-1, 1], where fp16's narrower exponent range costs nothing).
// With bf16 operands the per-sample local-energy deviation reached 2e-2 Ha on
// the 7-orbital workload and the VMC gradient's relative L2 error 1.6e-3;
// fp16 operands make both about eight times smaller.
//
// A CTA of 128 threads owns a tile of 128 rows (one row per thread and per
// TMEM lane).  For each slot p the CTA bulk-copies slot p's packed weight
// image into shared memory, writes the one-hot input of v_<p as the A
// operand, and runs the layers as M=128 x N=W x K GEMMs on the tensor cores
// (fp16 operands, f32 accumulation in TMEM).  Epilogues read the
// accumulator from TMEM, add the bias and apply tanh in f32, and write the
// fp16 activations back as the next A operand; the last hidden layer feeds
// the head (8 outputs) as one more MMA with N = 16 and the head's weights as
// fp16 hi + lo parts, then the masked log-softmax (Appendix B.1 f3 with MU
// masking, Sec. III.C) in f32.
//
// Modes
//   PARENT  rows = unique samples x, all slots; writes log psi(x) and, per
//           (x, slot), the prefix sum of the slot terms and the masked
//           half-log-probabilities and phases of all 4 outcomes.
//   SUFFIX  rows = connected determinants x' (sorted by first differing slot
//           j); log psi(x') = parent prefix up to j + parent slot-j term of
//           v'_j + the network's slots p > j (Eq. anqs_def: slots <= j see
//           the same prefix as in x).  Weight-stationary: each CTA serves
//           one slot for the whole launch.
//   LOGPSI  rows = arbitrary determinants, all slots, log psi only.
//   LOGITS  rows = sampler frontier prefixes, one slot, the 8 raw outputs.
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "tc_ptx.cuh"

namespace anqs {

int logpsi_dispatch(const anqs_model* M, const anqs_ham* H, const uint64_t* x, uint64_t n_x, float* la, float* ph,
                    cudaStream_t s);

namespace {

constexpr int MT = 128;          // rows per tile = threads per CTA
constexpr int CACHE_F = 10;      // floats per (parent, slot) cache entry
constexpr uint64_t kWaitNs = 2000000000ull;  // bounded waits: 2 s
enum { MODE_PARENT = 0, MODE_SUFFIX = 1, MODE_LOGPSI = 2, MODE_LOGITS = 3 };
enum { ST_TIMEOUT = 1 };

// Layout of one slot's packed image (byte offsets from the image base).
struct SlotLayout {
  uint32_t k1;      // padded input width of layer 1 (multiple of 16, 0 for slot 0)
  uint32_t w1;      // layer-1 matrix [W][k1] fp16, canonical K-major
  uint32_t w1lo;    // its rounding residual W1 - fp16(W1), same layout, or 0 bytes when the split is
                    // off (the one-hot input is exact, so hi + lo makes layer 1 exact to about 2^-22 relative)
  uint32_t wk;      // hidden matrices [L-1][W][W] fp16, canonical, each W*W*2 bytes
  uint32_t bias;    // [L][W] f32
  uint32_t head;    // head [W][8] f32 (transposed: the 8 outputs of input k are adjacent)
  uint32_t hbias;   // [8] f32
  uint32_t head16;  // head as an MMA operand: [16][W] fp16 hi then [16][W] lo (rows 8..15 zero), canonical
  uint32_t bytes;   // total, multiple of 128
};

__host__ __device__ inline uint32_t round_up(uint32_t a, uint32_t b) { return (a + b - 1) / b * b; }

__host__ __device__ inline SlotLayout slot_layout(int p, int W, int L, int lo) {
  SlotLayout s;
  s.k1 = round_up(4u * p, 16u);
  s.w1 = 0;
  s.w1lo = round_up(s.w1 + uint32_t(W) * s.k1 * 2u, 128u);
  s.wk = round_up(s.w1lo + (lo ? uint32_t(W) * s.k1 * 2u : 0u), 128u);
  s.bias = round_up(s.wk + uint32_t(L - 1) * W * W * 2u, 128u);
  s.head = round_up(s.bias + uint32_t(L) * W * 4u, 128u);
  s.hbias = round_up(s.head + 8u * W * 4u, 128u);
  s.head16 = round_up(s.hbias + 8u * 4u, 128u);
  s.bytes = round_up(s.head16 + 2u * 16u * W * 2u, 128u);
  return s;
}

// The layer-1 split is on when the largest slot image with it still fits in
// shared memory next to the warpgroups' A tiles (n <= 11 at width 128).
constexpr int kNwg = 4;
__host__ __device__ inline int use_w1_split(int n, int W, int L) {
  const uint32_t kmax = uint32_t(W) > round_up(4u * (n - 1), 16u) ? uint32_t(W) : round_up(4u * (n - 1), 16u);
  const uint32_t img = round_up(slot_layout(n - 1, W, L, 1).bytes, 1024u);
  return img + uint32_t(kNwg) * 128u * kmax * 2u <= 227u * 1024u ? 1 : 0;
}

struct TcView {
  int n, W, L;
  int lo;                     // layer-1 hi/lo split on (use_w1_split)
  const unsigned char* img;   // packed images
  uint32_t img_off[ANQS_MAX_ORB + 1];
  uint32_t max_img;           // largest image (bytes)
  uint32_t kmax;              // widest A operand (columns)
  int nbuf;                   // weight-image buffers in shared memory (1 or 2)
  int* status;
};

// ---- packing: f32 parameters -> per-slot fp16/f32 images --------------------

// f32 -> fp16 bits, round to nearest, saturating at the largest finite value
__device__ __forceinline__ uint16_t f16_bits(float v) { return uint16_t(tc::pack_f16x2(v, 0.f) & 0xFFFFu); }
__device__ __forceinline__ float f16_value(uint16_t b) { return __half2float(__ushort_as_half(b)); }
__global__ void pack_kernel(MlpView m, TcView tv, unsigned char* img) {
  // no early trigger: a later kernel's prologue may read the packed images
  // before its own dependency wait, so the images are complete before any
  // dependent launch starts
  ANQS_PDL_WAIT();
  const int p = blockIdx.y;
  const int W = m.width, L = m.n_hidden;
  const SlotLayout S = slot_layout(p, W, L, tv.lo);
  unsigned char* base = img + tv.img_off[p];
  const float* W1 = m.params + m.slot_off[p];
  const float* b1 = W1 + size_t(W) * 4 * p;
  const float* Wk = b1 + W;
  const float* Wh = Wk + size_t(L - 1) * (size_t(W) * W + W);
  const float* bh = Wh + 8 * W;
  const uint32_t n1 = uint32_t(W) * S.k1;
  const uint32_t nk = uint32_t(L - 1) * W * W;
  const uint32_t total = n1 + nk + uint32_t(L) * W + 8u * W + 8u + 16u * W;
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    if (t < n1) {
      uint32_t r = t / S.k1, k = t % S.k1;
      float v = (k < 4u * p) ? W1[size_t(r) * 4 * p + k] : 0.f;
      const uint16_t hi = f16_bits(v);
      *reinterpret_cast<uint16_t*>(base + S.w1 + tc::canon_off(r, k, S.k1)) = hi;
      if (tv.lo)
        *reinterpret_cast<uint16_t*>(base + S.w1lo + tc::canon_off(r, k, S.k1)) = f16_bits(v - f16_value(hi));
    } else if (t < n1 + nk) {
      uint32_t u = t - n1, l = u / (W * W), e = u % (W * W), r = e / W, k = e % W;
      float v = Wk[size_t(l) * (size_t(W) * W + W) + size_t(r) * W + k];
      *reinterpret_cast<uint16_t*>(base + S.wk + l * W * W * 2u + tc::canon_off(r, k, W)) = f16_bits(v);
    } else if (t < n1 + nk + uint32_t(L) * W) {
      uint32_t u = t - n1 - nk, l = u / W, o = u % W;
      const float* bl = (l == 0) ? b1 : (Wk + size_t(l - 1) * (size_t(W) * W + W) + size_t(W) * W);
      reinterpret_cast<float*>(base + S.bias)[u] = bl[o];
    } else if (t < n1 + nk + uint32_t(L) * W + 8u * W) {
      uint32_t u = t - n1 - nk - uint32_t(L) * W, o = u / W, k = u % W;
      reinterpret_cast<float*>(base + S.head)[k * 8 + o] = Wh[o * W + k];
    } else if (t < n1 + nk + uint32_t(L) * W + 8u * W + 8u) {
      uint32_t u = t - n1 - nk - uint32_t(L) * W - 8u * W;
      reinterpret_cast<float*>(base + S.hbias)[u] = bh[u];
    } else {  // head as an MMA operand, hi and lo fp16 parts
      uint32_t u = t - n1 - nk - uint32_t(L) * W - 8u * W - 8u, o = u / W, k = u % W;
      const float v = o < 8 ? Wh[o * W + k] : 0.f;
      const uint16_t hi = f16_bits(v);
      *reinterpret_cast<uint16_t*>(base + S.head16 + tc::canon_off(o, k, W)) = hi;
      *reinterpret_cast<uint16_t*>(base + S.head16 + 16u * W * 2u + tc::canon_off(o, k, W)) = f16_bits(v - f16_value(hi));
    }
  }
}

// Bounded wait; on time-out waits once more (bounded) for the operation still
// in flight and reports failure.
__device__ __forceinline__ bool wait_bar(uint32_t bar, uint32_t phase) {
  if (tc::mbar_wait(bar, phase, kWaitNs)) return true;
  tc::mbar_wait(bar, phase, kWaitNs);
  return false;
}

struct TileArgs {
  const uint64_t* x;           // SLOTS: rows x[0..rows); SUFFIX: connected determinants
  Count rows;
  int p_lo, p_hi;              // SLOTS: slots [p_lo, p_hi)
  float* raw;                  // SLOTS output [row][p_hi - p_lo][8]
  int tpi;                     // SLOTS: 128-row tiles per work item (1..NWG; warpgroups >= tpi idle)
  int levels;                  // LEVELS: rows [lv_off[p], lv_off[p+1]) take slot p (p < levels), raw [row][8]
  uint32_t lv_off[ANQS_MAX_ORB + 1];
  ZeroWords zero;              // cleared by block 0 for the next kernel
};

constexpr int NWG = kNwg;     // warpgroups per CTA, one 128-row tile each in flight
constexpr int kMaxBatch = 32;  // problems of one persistent multi-problem launch
constexpr int NT = NWG * MT;

struct Ctx {
  const TcView* tv;
  unsigned char* s_a;        // this warpgroup's A tile
  uint32_t a_addr;
  uint32_t tmem;             // this warpgroup's two accumulators
  uint32_t lane_base;
  uint32_t bar_m;            // this warpgroup's MMA barrier
  int wg, t;
};

__device__ __forceinline__ void wg_sync(int wg) { asm volatile("bar.sync %0, 128;" ::"r"(1 + wg) : "memory"); }

// Warpgroup barrier that also ANDs a flag over the 128 threads, so that a
// bounded wait that gives up in some threads sends the whole warpgroup down
// the same path.
__device__ __forceinline__ bool wg_all(int wg, bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred q, s;\n\t"
      "setp.ne.u32 q, %1, 0;\n\t"
      "bar.red.and.pred s, %2, 128, q;\n\t"
      "selp.u32 %0, 1, 0, s;\n\t}\n"
      : "=r"(r)
      : "r"(uint32_t(v)), "r"(1 + wg)
      : "memory");
  return r != 0;
}

// All layers of slot p for the 128 rows of one tile (one warpgroup; row t =
// thread t).  Returns false if a wait timed out.
template <int W>
__device__ bool tile_slot(const Ctx& c, uint32_t& ph_m, int p, uint64_t x, const SlotLayout& S, uint32_t img_addr,
                          const unsigned char* img, float (&out)[8]) {
  constexpr uint32_t IDESC = tc::idesc_f16_f32(MT, W);
  const int L = c.tv->L;
  // layer-1 input: one-hot of v_<p (K = k1 columns)
  for (uint32_t k = 0; k < S.k1; k += 8) {
    uint32_t w4[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      uint32_t lo = 0, hi = 0;
      const uint32_t k0 = k + 2 * e, k1 = k0 + 1;
      if (k0 < 4u * p && ((x >> (2 * (k0 >> 2))) & 3ull) == (k0 & 3u)) lo = 0x3C00u;  // fp16 1.0
      if (k1 < 4u * p && ((x >> (2 * (k1 >> 2))) & 3ull) == (k1 & 3u)) hi = 0x3C00u;
      w4[e] = lo | (hi << 16);
    }
    *reinterpret_cast<uint4*>(c.s_a + tc::canon_off(c.t, k, S.k1)) = make_uint4(w4[0], w4[1], w4[2], w4[3]);
  }
  tc::fence_async_smem();
  tc::fence_before_sync();
  wg_sync(c.wg);
  const float* bias = reinterpret_cast<const float*>(img + S.bias);
  const float* hbias = reinterpret_cast<const float*>(img + S.hbias);
  bool ok = true;
  for (int layer = 0; layer < L; ++layer) {
    const uint32_t K = layer == 0 ? S.k1 : uint32_t(W);
    if (K > 0) {
      if (c.t == 0) {
        tc::fence_after_sync();
        const uint32_t b_addr = img_addr + (layer == 0 ? S.w1 : S.wk + uint32_t(layer - 1) * W * W * 2u);
#pragma unroll 1
        for (uint32_t ks = 0; ks < K / 16; ++ks)
          tc::mma_f16(c.tmem, tc::sdesc(c.a_addr + ks * 256u, 128u, K * 16u),
                      tc::sdesc(b_addr + ks * 256u, 128u, K * 16u), IDESC, ks > 0 ? 1u : 0u);
        if (layer == 0 && c.tv->lo) {  // + one-hot x (W1 - fp16(W1))
#pragma unroll 1
          for (uint32_t ks = 0; ks < K / 16; ++ks)
            tc::mma_f16(c.tmem, tc::sdesc(c.a_addr + ks * 256u, 128u, K * 16u),
                        tc::sdesc(img_addr + S.w1lo + ks * 256u, 128u, K * 16u), IDESC, 1u);
        }
        tc::mma_commit(c.bar_m);
      }
      ok = wg_all(c.wg, wait_bar(c.bar_m, ph_m));
      ph_m ^= 1;
      if (!ok) return false;
      tc::fence_after_sync();
    }
    const float* b = bias + layer * W;
#pragma unroll 1
    for (int c0 = 0; c0 < W; c0 += 32) {
      float v[32];
      if (K > 0) {
        tc::tmem_ld32(c.tmem + c.lane_base + uint32_t(c0), v);
      } else {
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = 0.f;
      }
#pragma unroll
      for (int i = 0; i < 32; i += 2) {
        const float2 bb = *reinterpret_cast<const float2*>(b + c0 + i);
        tc::add_f32x2(v[i], v[i + 1], bb.x, bb.y, v[i], v[i + 1]);
      }
      // the next GEMM's operand (after the last layer, the head's): f32 tanh,
      // rounded to fp16 (a half-precision tanh would add its own
      // approximation error to the rounding)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        uint32_t u[4];
#pragma unroll
        for (int e = 0; e < 4; ++e)
          u[e] = tc::pack_f16x2(tc::tanh_fast(v[8 * q + 2 * e]), tc::tanh_fast(v[8 * q + 2 * e + 1]));
        *reinterpret_cast<uint4*>(c.s_a + tc::canon_off(c.t, c0 + 8 * q, W)) = make_uint4(u[0], u[1], u[2], u[3]);
      }
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    wg_sync(c.wg);
  }
  // head: the 8 outputs as one MMA with N = 16 (weights as fp16 hi + lo parts,
  // rows 8..15 zero), into the accumulator's first columns (all of them were
  // read before the barrier above)
  if (c.t == 0) {
    tc::fence_after_sync();
    constexpr uint32_t IDESC_H = tc::idesc_f16_f32(MT, 16);
#pragma unroll 1
    for (uint32_t ks = 0; ks < uint32_t(W) / 16; ++ks)
      tc::mma_f16(c.tmem, tc::sdesc(c.a_addr + ks * 256u, 128u, W * 16u),
                  tc::sdesc(img_addr + S.head16 + ks * 256u, 128u, W * 16u), IDESC_H, ks > 0 ? 1u : 0u);
#pragma unroll 1
    for (uint32_t ks = 0; ks < uint32_t(W) / 16; ++ks)
      tc::mma_f16(c.tmem, tc::sdesc(c.a_addr + ks * 256u, 128u, W * 16u),
                  tc::sdesc(img_addr + S.head16 + 16u * W * 2u + ks * 256u, 128u, W * 16u), IDESC_H, 1u);
    tc::mma_commit(c.bar_m);
  }
  ok = wg_all(c.wg, wait_bar(c.bar_m, ph_m));
  ph_m ^= 1;
  if (!ok) return false;
  tc::fence_after_sync();
  float v8[8];
  tc::tmem_ld8(c.tmem + c.lane_base, v8);
#pragma unroll
  for (int o = 0; o < 8; ++o) out[o] = v8[o] + hbias[o];
  return true;
}

// Shared set-up of both kernels: barriers and TMEM (NWG*W columns: one
// accumulator per warpgroup).
template <int W>
__device__ __forceinline__ void setup(uint64_t* bars, uint32_t* s_tmem, int* s_abort) {
  if (threadIdx.x == 0) {
    for (int i = 0; i < 2 + NWG; ++i) tc::mbar_init(tc::smem_u32(&bars[i]), 1);
    tc::fence_mbar_init();
    *s_abort = 0;
  }
  if (threadIdx.x < 32) {
    tc::tmem_alloc(tc::smem_u32(s_tmem), NWG * W);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
}

template <int W>
__device__ __forceinline__ void teardown(const TcView& tv, uint32_t tmem, int abort) {
  if (abort && threadIdx.x == 0) atomicExch(tv.status, ST_TIMEOUT);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (threadIdx.x < 32) tc::tmem_dealloc(tmem, NWG * W);
}

__device__ __forceinline__ void load_slot(const TcView& tv, int p, uint32_t dst, uint32_t bar, int W, int L) {
  const SlotLayout S = slot_layout(p, W, L, tv.lo);
  tc::mbar_arrive_expect_tx(bar, S.bytes);
  tc::bulk_g2s(dst, tv.img + tv.img_off[p], S.bytes, bar);
}

// SLOTS: work item = (group of NWG 128-row tiles, slot p); writes the 8 raw
// outputs of slot p for every row.
template <int W>
__global__ void __launch_bounds__(NT, 1) mlp_tc_slots_kernel(TcView tv, TileArgs ta) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t bars[2 + NWG];  // 0,1: weights; 2..: MMA per warpgroup
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort;
  const int wg = threadIdx.x / MT, t = threadIdx.x % MT;
  setup<W>(bars, &s_tmem, &s_abort);
  const uint32_t img_stride = round_up(tv.max_img, 1024u);
  unsigned char* s_img = smem;
  Ctx c;
  c.tv = &tv;
  c.s_a = smem + img_stride * tv.nbuf + wg * (MT * tv.kmax * 2u);
  c.a_addr = tc::smem_u32(c.s_a);
  c.tmem = s_tmem + uint32_t(wg) * W;
  c.lane_base = uint32_t(t & ~31) << 16;
  c.bar_m = tc::smem_u32(&bars[2 + wg]);
  c.wg = wg;
  c.t = t;
  const uint32_t bar_w = tc::smem_u32(&bars[0]);
  uint32_t ph_w = 0, ph_m = 0;
  const int np = ta.p_hi - ta.p_lo;
  // A single-slot launch (one sampler level) fetches its weight image in the
  // prologue: the packed images were written before the previous kernel.
  int loaded = -1;     // slot whose image is in shared memory (or on its way)
  bool pending = false;
  if (np == 1 && !ta.levels) {
    if (threadIdx.x == 0) load_slot(tv, ta.p_lo, tc::smem_u32(s_img), bar_w, W, tv.L);
    loaded = ta.p_lo;
    pending = true;
  }
  ANQS_PDL_WAIT();
  ANQS_PDL_TRIGGER();
  if (blockIdx.x == 0)
    for (int r = 0; r < 2; ++r)
      for (int i = threadIdx.x; i < ta.zero.n[r]; i += NT) ta.zero.p[r][i] = 0u;
  const uint64_t n_rows = ta.rows.get();
  const int tpi = ta.tpi;
  const uint64_t n_groups = (n_rows + uint64_t(tpi) * MT - 1) / (uint64_t(tpi) * MT);
  const uint64_t n_items = n_groups * uint64_t(np);
  // LEVELS: items are (level p, group of its rows), levels in order
  uint64_t n_items_lv = 0;
  if (ta.levels)
    for (int q = 0; q < ta.levels; ++q)
      n_items_lv += (uint64_t(ta.lv_off[q + 1] - ta.lv_off[q]) + uint64_t(tpi) * MT - 1) / (uint64_t(tpi) * MT);
  for (uint64_t it = blockIdx.x; it < (ta.levels ? n_items_lv : n_items); it += gridDim.x) {
    int p = ta.p_lo + int(it / n_groups);
    uint64_t grp = it % n_groups, row_lo = 0, row_hi = n_rows;
    if (ta.levels) {
      uint64_t acc = 0;
      for (int q = 0; q < ta.levels; ++q) {
        const uint64_t g = (uint64_t(ta.lv_off[q + 1] - ta.lv_off[q]) + uint64_t(tpi) * MT - 1) / (uint64_t(tpi) * MT);
        if (it < acc + g) {
          p = q;
          grp = it - acc;
          row_lo = ta.lv_off[q];
          row_hi = ta.lv_off[q + 1];
          break;
        }
        acc += g;
      }
    }
    const SlotLayout S = slot_layout(p, W, tv.L, tv.lo);
    if (p != loaded) {
      // a copy still in flight into the buffer lands before the next one is issued
      if (pending) {
        if (!__syncthreads_and(wait_bar(bar_w, ph_w))) s_abort = 1;
        ph_w ^= 1;
        pending = false;
        if (s_abort) break;
      }
      if (threadIdx.x == 0) load_slot(tv, p, tc::smem_u32(s_img), bar_w, W, tv.L);
      loaded = p;
      pending = true;
    }
    const uint64_t r = row_lo + (grp * tpi + wg) * MT + t;
    const bool valid = wg < tpi && r < row_hi;
    const uint64_t x = valid ? ta.x[r] : 0ull;
    bool ok = true;
    if (pending) {
      ok = __syncthreads_and(wait_bar(bar_w, ph_w));
      ph_w ^= 1;
      pending = false;
    }
    float out[8];
    if (ok && wg < tpi && row_lo + (grp * tpi + wg) * MT < row_hi)
      ok = tile_slot<W>(c, ph_m, p, x, S, tc::smem_u32(s_img), s_img, out);
    if (!ok) s_abort = 1;
    if (ok && valid) {
      float4* dst = reinterpret_cast<float4*>(ta.raw + (ta.levels ? r : r * np + (p - ta.p_lo)) * 8);
      dst[0] = make_float4(out[0], out[1], out[2], out[3]);
      dst[1] = make_float4(out[4], out[5], out[6], out[7]);
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    if (s_abort) break;
  }
  if (pending && !__syncthreads_and(wait_bar(bar_w, ph_w))) s_abort = 1;  // prefetched image not used
  teardown<W>(tv, s_tmem, s_abort);
}

// One 128-row tile of the suffix work of slot p (one warpgroup): rows
// perm[tile*128 + t] of the connected determinants with first differing slot
// j < p (the first `rows` entries of the sorted order); writes each row's
// masked slot-p term T[row][p] = (log|psi_p(v_p)|, phase).  The caller loads
// the row index and its determinant (suffix_row), ahead of time where it can.
// The slot's mask is read before the MMAs start so that its latency overlaps
// them.  Returns false if a wait timed out.
struct SuffixRow {
  uint32_t row;
  uint64_t x;
};

// Loads of the sort's outputs go through L2: they are written by kernels that
// may have been launched just before this one.
__device__ __forceinline__ SuffixRow suffix_row(uint64_t tile, uint64_t rows, int t, const uint32_t* perm,
                                                const uint64_t* xp) {
  const uint64_t r = tile * MT + t;
  SuffixRow s{0u, 0ull};
  if (r < rows) {
    s.row = __ldcg(perm + r);
    s.x = __ldcg(reinterpret_cast<const unsigned long long*>(xp) + s.row);
  }
  return s;
}

template <int W>
__device__ __forceinline__ bool suffix_tile(const Ctx& c, uint32_t& ph_m, int p, int n, uint64_t tile, uint64_t rows,
                                            SuffixRow sr, const HamView& hv, const SlotLayout& Sl, uint32_t img_addr,
                                            const unsigned char* img, float2* T) {
  const bool valid = tile * MT + c.t < rows;
  const uint32_t row = sr.row;
  const uint64_t x = sr.x;
  unsigned pmk = 0, mk = 0;
  if (valid) {
    const uint64_t pm = (1ull << (2 * p)) - 1ull;
    const int a = __popcll(x & pm & 0x5555555555555555ull);
    const int bb = __popcll(x & pm & 0xAAAAAAAAAAAAAAAAull);
    pmk = slot_mask(hv, p, a, bb, x);
    mk = norm_mask(hv, p, pmk);
  }
  float out[8];
  const bool ok = tile_slot<W>(c, ph_m, p, x, Sl, img_addr, img, out);
  if (ok && valid) {
    float mx = -INFINITY;
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if ((mk >> u) & 1u) mx = fmaxf(mx, out[u]);
    float sum = 0.f;
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if ((mk >> u) & 1u) sum += __expf(out[u] - mx);
    const int v = int((x >> (2 * p)) & 3ull);
    const float ov = (v == 0) ? out[0] : (v == 1) ? out[1] : (v == 2) ? out[2] : out[3];
    const float pv = (v == 0) ? out[4] : (v == 1) ? out[5] : (v == 2) ? out[6] : out[7];
    const float lse = mx + __logf(sum);  // same expression order as finalize_kernel
    T[uint64_t(row) * n + p] = make_float2(((pmk >> v) & 1u) ? 0.5f * (ov - lse) : -INFINITY, pv);
  }
  return ok;
}

// SUFFIX (weight-stationary): the connected determinants sorted by first
// differing slot j make, for every slot p, the rows that need slot p (those
// with j < p) a prefix of the sorted order.  The grid is split among the
// slots in proportion to their tiles; a CTA loads its slot's weight image
// once and its warpgroups stream tiles of that slot independently (no
// CTA-wide barrier in the loop).  Each (row, slot) term goes to T[row][p];
// the local-energy kernel adds a row's terms to the parent's prefix.
template <int W>
__global__ void __launch_bounds__(NT, 1) mlp_tc_ws_kernel(TcView tv, HamView hv, const uint64_t* __restrict__ xp,
                                                         const uint32_t* __restrict__ perm,
                                                         const uint32_t* __restrict__ offsets,
                                                         float2* __restrict__ T) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t bars[2 + NWG];
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort;
  const int wg = threadIdx.x / MT, t = threadIdx.x % MT;
  const int n = tv.n;
  setup<W>(bars, &s_tmem, &s_abort);
  ANQS_PDL_WAIT();
  ANQS_PDL_TRIGGER();
  const uint32_t img_stride = round_up(tv.max_img, 1024u);
  Ctx c;
  c.tv = &tv;
  c.s_a = smem + img_stride + wg * (MT * tv.kmax * 2u);
  c.a_addr = tc::smem_u32(c.s_a);
  c.tmem = s_tmem + uint32_t(wg) * W;
  c.lane_base = uint32_t(t & ~31) << 16;
  c.bar_m = tc::smem_u32(&bars[2 + wg]);
  c.wg = wg;
  c.t = t;
  // partition of the grid among the slots (same result in every CTA); the
  // slots' tile counts go to shared memory once, not to every thread's stack
  __shared__ uint32_t tiles[ANQS_MAX_ORB];
  if (threadIdx.x < n) tiles[threadIdx.x] = uint32_t((uint64_t(offsets[threadIdx.x]) + MT - 1) / MT);
  __syncthreads();
  uint64_t total = 0;
  int S = 0;
  for (int p = 0; p < n; ++p) {
    total += tiles[p];
    S += tiles[p] ? 1 : 0;
  }
  int my_p = -1;
  uint64_t li = 0, gp = 0;
  if (total) {
    const uint64_t G = gridDim.x, spare = G > uint64_t(S) ? G - S : 0;
    uint64_t start = 0;
    for (int p = 0; p < n; ++p) {
      if (!tiles[p]) continue;
      const uint64_t g = 1 + spare * tiles[p] / total;
      if (blockIdx.x >= start && blockIdx.x < start + g) {
        my_p = p;
        li = blockIdx.x - start;
        gp = g;
      }
      start += g;
    }
  }
  if (my_p >= 0) {
    const int p = my_p;
    const SlotLayout Sl = slot_layout(p, W, tv.L, tv.lo);
    const uint32_t img_addr = tc::smem_u32(smem);
    if (threadIdx.x == 0) load_slot(tv, p, img_addr, tc::smem_u32(&bars[0]), W, tv.L);
    bool ok = __syncthreads_and(wait_bar(tc::smem_u32(&bars[0]), 0));
    const uint64_t rows = offsets[p];
    uint32_t ph_m = 0;
    // the next tile's rows are loaded while this tile runs
    uint64_t tile = li + gp * wg;
    SuffixRow nx = tile < tiles[p] ? suffix_row(tile, rows, t, perm, xp) : SuffixRow{0u, 0ull};
    for (; ok && tile < tiles[p]; tile += gp * NWG) {
      const SuffixRow cur = nx;
      if (tile + gp * NWG < tiles[p]) nx = suffix_row(tile + gp * NWG, rows, t, perm, xp);
      ok = suffix_tile<W>(c, ph_m, p, n, tile, rows, cur, hv, Sl, img_addr, smem, T);
    }
    if (!ok) s_abort = 1;
  }
  teardown<W>(tv, s_tmem, s_abort);
}

// ---- many problems in one persistent launch ---------------------------------
//
// The suffix work of up to kMaxBatch independent problems (each its own
// Hamiltonian, MLP and connected set, all of width W) in one launch of one
// CTA per SM.  A plan kernel turns the problems' sorted row counts into
// groups (problem b, slot p, tiles of slot p) in problem-major order; the
// tiles of all groups form one sequence.  Two schedules:
//   static   CTA i of G takes the contiguous tile range [i T / G, (i+1) T / G)
//            of the sequence: every CTA gets the same number of tiles, and it
//            synchronises and reloads the weight image only where its range
//            crosses into the next group;
//   dynamic  the groups are cut into work items of `chunk` tiles that CTAs
//            take from a global counter (the next item is fetched while the
//            current one runs); a CTA synchronises after every item and
//            reloads the image when the item's group differs.
// In both, the CTA's warpgroups share the tiles round-robin.  `chunk` and
// the schedule are what the batch autotuner chooses.  Every tile computes
// exactly what the single-problem launch computes for it, so the results are
// bit-identical.
struct MultiProblem {
  TcView tv;
  HamView hv;
  const uint64_t* xp;
  const uint32_t* perm;
  const uint32_t* offsets;
  float2* T;
};

struct MultiGroup {
  uint32_t bp;     // problem << 8 | slot
  uint32_t tiles;  // 128-row tiles of the slot
  uint32_t item0;  // first work item of the group (dynamic schedule)
  uint32_t tile0;  // first tile of the group in the sequence (static schedule)
};

struct MultiArgs {
  int n_prob, chunk, dynamic, pad;
  uint32_t max_img, kmax;
  MultiGroup* groups;  // [kMaxBatch * ANQS_MAX_ORB]
  uint32_t* ctl;       // [0] groups, [1] items, [2] next item (dynamic), [3] tiles
  MultiProblem prob[kMaxBatch];
};
static_assert(sizeof(MultiArgs) <= 32000, "kernel parameter block too large");

__global__ void multi_plan_kernel(const __grid_constant__ MultiArgs a) {
  ANQS_PDL_ENTRY();
  __shared__ uint32_t tiles[kMaxBatch][ANQS_MAX_ORB];
  for (int i = threadIdx.x; i < kMaxBatch * ANQS_MAX_ORB; i += blockDim.x) {
    const int b = i / ANQS_MAX_ORB, p = i % ANQS_MAX_ORB;
    uint32_t t = 0;
    if (b < a.n_prob && p < a.prob[b].tv.n) t = (__ldcg(a.prob[b].offsets + p) + MT - 1) / MT;
    tiles[b][p] = t;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t g = 0, items = 0, t0 = 0;
    for (int b = 0; b < a.n_prob; ++b)
      for (int p = 0; p < a.prob[b].tv.n; ++p)
        if (tiles[b][p]) {
          a.groups[g] = MultiGroup{uint32_t(b) << 8 | uint32_t(p), tiles[b][p], items, t0};
          items += (tiles[b][p] + uint32_t(a.chunk) - 1) / uint32_t(a.chunk);
          t0 += tiles[b][p];
          ++g;
        }
    a.ctl[0] = g;
    a.ctl[1] = items;
    a.ctl[2] = 0;
    a.ctl[3] = t0;
  }
}

// Last group g with key(g) <= v (keys ascending; group 0 has key 0), found by
// warp 0 and returned to every thread.  Contains a CTA barrier.
__device__ __forceinline__ uint32_t multi_find(const MultiGroup* groups, uint32_t n_groups, uint32_t v,
                                               bool by_tile, uint32_t* s_out) {
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    uint32_t best = 0;
    for (uint32_t g0 = 0; g0 < n_groups; g0 += 32) {
      const uint32_t g = g0 + lane;
      const bool le = g < n_groups && __ldcg(by_tile ? &groups[g].tile0 : &groups[g].item0) <= v;
      const unsigned m = __ballot_sync(0xffffffffu, le);
      if (m) best = g0 + 31 - __clz(m);
      if (m != 0xffffffffu) break;
    }
    if (lane == 0) *s_out = best;
  }
  __syncthreads();
  return *s_out;
}

template <int W>
__global__ void __launch_bounds__(NT, 1) mlp_tc_multi_kernel(const __grid_constant__ MultiArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t bars[2 + NWG];
  __shared__ uint32_t s_tmem, s_item[2], s_group;
  __shared__ int s_abort;
  const int wg = threadIdx.x / MT, t = threadIdx.x % MT;
  setup<W>(bars, &s_tmem, &s_abort);
  ANQS_PDL_WAIT();
  ANQS_PDL_TRIGGER();
  Ctx c;
  c.tv = &a.prob[0].tv;
  c.s_a = smem + round_up(a.max_img, 1024u) + wg * (MT * a.kmax * 2u);
  c.a_addr = tc::smem_u32(c.s_a);
  c.tmem = s_tmem + uint32_t(wg) * W;
  c.lane_base = uint32_t(t & ~31) << 16;
  c.bar_m = tc::smem_u32(&bars[2 + wg]);
  c.wg = wg;
  c.t = t;
  const uint32_t img_addr = tc::smem_u32(smem), bar_w = tc::smem_u32(&bars[0]);
  const uint32_t n_groups = __ldcg(a.ctl), n_items = __ldcg(a.ctl + 1), n_tiles = __ldcg(a.ctl + 3);
  uint32_t ph_w = 0, ph_m = 0, loaded = 0xffffffffu;
  // the tiles [t_lo, t_hi) of group g (positions within the group); false on a timed-out wait
  auto run = [&](uint32_t g, uint32_t t_lo, uint32_t t_hi) -> bool {
    const uint32_t bp = __ldcg(&a.groups[g].bp);
    const int b = int(bp >> 8), p = int(bp & 0xffu);
    const MultiProblem& P = a.prob[b];
    c.tv = &P.tv;
    const SlotLayout Sl = slot_layout(p, W, P.tv.L, P.tv.lo);
    if (bp != loaded) {  // every warpgroup is past its last read of the old image (barrier before)
      if (threadIdx.x == 0) load_slot(P.tv, p, img_addr, bar_w, W, P.tv.L);
      const bool ok = __syncthreads_and(wait_bar(bar_w, ph_w));
      ph_w ^= 1;
      loaded = bp;
      if (!ok) return false;
    }
    const uint64_t rows = __ldcg(P.offsets + p);
    bool ok = true;
    for (uint32_t tile = t_lo + wg; ok && tile < t_hi; tile += NWG)
      ok = suffix_tile<W>(c, ph_m, p, P.tv.n, tile, rows, suffix_row(tile, rows, c.t, P.perm, P.xp), P.hv, Sl, img_addr,
                          smem, P.T);
    tc::fence_async_smem();
    tc::fence_before_sync();
    return __syncthreads_and(ok);
  };
  if (!a.dynamic) {
    const uint32_t lo = uint32_t(uint64_t(n_tiles) * blockIdx.x / gridDim.x),
                   hi = uint32_t(uint64_t(n_tiles) * (blockIdx.x + 1) / gridDim.x);
    if (lo < hi) {
      for (uint32_t g = multi_find(a.groups, n_groups, lo, true, &s_group); g < n_groups; ++g) {
        const uint32_t g0 = __ldcg(&a.groups[g].tile0), gt = __ldcg(&a.groups[g].tiles);
        if (g0 >= hi) break;
        if (!run(g, (lo > g0 ? lo : g0) - g0, (hi < g0 + gt ? hi : g0 + gt) - g0)) {
          s_abort = 1;
          break;
        }
      }
    }
  } else {
    if (threadIdx.x == 0) s_item[0] = atomicAdd(a.ctl + 2, 1u);
    uint32_t g = 0, g_item0 = 1, g_item1 = 0;  // current group and its items [g_item0, g_item1)
    for (uint32_t k = 0;; ++k) {
      __syncthreads();
      const uint32_t item = s_item[k & 1];
      if (item >= n_items) break;
      if (threadIdx.x == 0) s_item[(k + 1) & 1] = atomicAdd(a.ctl + 2, 1u);  // read after the next barrier
      if (item < g_item0 || item >= g_item1) {
        g = multi_find(a.groups, n_groups, item, false, &s_group);
        g_item0 = __ldcg(&a.groups[g].item0);
        g_item1 = g_item0 + (__ldcg(&a.groups[g].tiles) + uint32_t(a.chunk) - 1) / uint32_t(a.chunk);
      }
      const uint32_t gt = __ldcg(&a.groups[g].tiles);
      const uint32_t t0 = (item - g_item0) * uint32_t(a.chunk), t1 = min(t0 + uint32_t(a.chunk), gt);
      if (!run(g, t0, t1)) {
        s_abort = 1;
        break;
      }
    }
  }
  if (s_abort && threadIdx.x < a.n_prob) atomicExch(a.prob[threadIdx.x].tv.status, ST_TIMEOUT);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (threadIdx.x < 32) tc::tmem_dealloc(s_tmem, NWG * W);
}

// ---- the adjoint (Eq. grad_def) on the tensor cores ------------------------
//
// One CTA of 128 threads per (128-row tile of the samples, slot p); thread t
// owns sample row t and TMEM lane t.  It recomputes slot p's forward pass in
// the 16-bit form (layer 1 from the hi part of W1), turns the cotangents of
// log|psi| and arg psi into the head's adjoint, and runs the backward pass:
//   data GEMMs    dh_{k-1} = dz_k W_k           (A: dz_k per row, B: W_k)
//   weight GEMMs  dW_k = dz_k^T h_{k-1}, dW_1 = dz_1^T u, dW_h = dout^T h_L
// The weight GEMMs reduce over the tile's rows, so their operands are the
// same per-row tiles read as MN-major matrices (K = rows), and the data GEMMs
// read the forward weight image as an MN-major B operand: no transposed copy
// of anything is made.  Operands are fp16; the cotangents of each tile are
// scaled by a power of two that puts their largest magnitude at 2^8 (the
// gradient is linear in them; the scale is divided out, exactly, when the
// tile's partial gradient is written).  Biases' gradients are the column sums
// of the dz tiles, one more small MMA per layer against the dout tile, whose
// column 8 holds ones.  Each tile writes its slot's block of a per-tile
// partial gradient; a reduction over the tiles follows.
__device__ __forceinline__ int popc_alpha_tc(uint64_t x, int p) {
  return __popcll(x & ((1ull << (2 * p)) - 1ull) & 0x5555555555555555ull);
}
__device__ __forceinline__ int popc_beta_tc(uint64_t x, int p) {
  return __popcll(x & ((1ull << (2 * p)) - 1ull) & 0xAAAAAAAAAAAAAAAAull);
}

// offsets of slot p's parameter blocks in the flat parameter vector
struct MlpPtrTc {
  uint64_t W1, b1, Wk, Wh, bh;
};
__device__ __forceinline__ MlpPtrTc slot_ptrs_tc(const MlpView& m, int p) {
  MlpPtrTc r;
  const uint64_t w = uint64_t(m.width);
  r.W1 = m.slot_off[p];
  r.b1 = r.W1 + w * 4u * uint64_t(p);
  r.Wk = r.b1 + w;
  r.Wh = r.Wk + uint64_t(m.n_hidden - 1) * (w * w + w);
  r.bh = r.Wh + 8u * w;
  return r;
}

struct GradArgs {
  TcView tv;
  MlpView m;
  HamView hv;
  const uint64_t* xs;
  Count n_x;
  CotSrc cot;
  float* part;  // [tiles][n_params]
  uint64_t n_params;
  uint32_t img_bytes, kmax1;  // image region (without W1's lo part), widest layer-1 input
};

// MN-major view of a tile stored per row in the canonical K-major layout with
// `cols` columns: the MMA's K runs over the rows (16 per step), M or N over
// the columns.
__device__ __forceinline__ uint64_t mn_desc(uint32_t base, uint32_t cols, uint32_t ks) {
  return tc::sdesc(base + ks * 2u * cols * 16u, cols * 16u, 128u);
}

__host__ __device__ constexpr uint32_t idesc_f16_mn(int M, int N, bool a_mn, bool b_mn) {
  return tc::idesc_f16_f32(M, N) | (a_mn ? (1u << 15) : 0u) | (b_mn ? (1u << 16) : 0u);
}

template <int W>
__global__ void __launch_bounds__(MT, 1) mlp_tc_grad_kernel(const __grid_constant__ GradArgs a) {
  static_assert(W == 128, "the weight GEMMs put the layer width on the MMA's M = 128");
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t bars[2];
  __shared__ uint32_t s_tmem;
  __shared__ float s_max[4], s_bh[4][8];
  __shared__ int s_abort;
  constexpr uint32_t TILE = MT * W * 2u;
  constexpr uint32_t C_ACC = 0, C_DW = W, C_DWH = 2 * W, C_DB = 2 * W + 16, C_DW1 = 2 * W + 32,
                     NCOL = W == 128 ? 512 : 256;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int p = blockIdx.y, L = a.m.n_hidden;
  const SlotLayout S = slot_layout(p, W, L, a.tv.lo);
  const uint32_t k1 = S.k1, lo_bytes = S.wk - S.w1lo;
  // shared memory: image (W1 hi | hidden | bias | f32 head) | H_1..H_{L-1} | P1 | P2 | U | dout (and ones)
  unsigned char* img = smem;
  const uint32_t o_wk = S.w1lo, o_bias = S.bias - lo_bytes, o_head = S.head - lo_bytes, o_hb = S.hbias - lo_bytes;
  unsigned char* Hb = smem + a.img_bytes;
  unsigned char* P1 = Hb + uint32_t(L - 1) * TILE;
  unsigned char* P2 = P1 + TILE;
  unsigned char* U = P2 + TILE;
  unsigned char* DO = U + MT * a.kmax1 * 2u;
  const uint32_t bar_w = tc::smem_u32(&bars[0]), bar_m = tc::smem_u32(&bars[1]);
  if (t == 0) {
    tc::mbar_init(bar_w, 1);
    tc::mbar_init(bar_m, 1);
    tc::fence_mbar_init();
    s_abort = 0;
    // the image, written by the packing kernel several launches back
    const unsigned char* src = a.tv.img + a.tv.img_off[p];
    tc::mbar_arrive_expect_tx(bar_w, S.w1lo + (S.head16 - S.wk));
    if (S.w1lo) tc::bulk_g2s(tc::smem_u32(img), src, S.w1lo, bar_w);
    tc::bulk_g2s(tc::smem_u32(img + o_wk), src + S.wk, S.head16 - S.wk, bar_w);
  }
  if (warp == 0) {
    tc::tmem_alloc(tc::smem_u32(&s_tmem), NCOL);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  ANQS_PDL_WAIT();
  ANQS_PDL_TRIGGER();
  const uint32_t tm = s_tmem, lb = uint32_t(t & ~31) << 16;
  const uint64_t n_x = a.n_x.get();
  const uint64_t row = uint64_t(blockIdx.x) * MT + t;
  const bool valid = row < n_x;
  const uint64_t x = valid ? a.xs[row] : 0ull;
  float cla = 0.f, cph = 0.f;
  if (valid) cot_of(a.cot, row, cla, cph);
  // scale of the tile's cotangents: a power of two, largest magnitude -> 2^8
  {
    float mx = fmaxf(fabsf(cla), fabsf(cph));
    for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) s_max[warp] = mx;
  }
  // one-hot input of v_<p (layer 1's A operand and dW_1's B operand)
  for (uint32_t k = 0; k < k1; k += 8) {
    uint32_t w4[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      uint32_t lo = 0, hi = 0;
      const uint32_t k0 = k + 2 * e, kk = k0 + 1;
      if (k0 < 4u * p && ((x >> (2 * (k0 >> 2))) & 3ull) == (k0 & 3u)) lo = 0x3C00u;
      if (kk < 4u * p && ((x >> (2 * (kk >> 2))) & 3ull) == (kk & 3u)) hi = 0x3C00u;
      w4[e] = lo | (hi << 16);
    }
    *reinterpret_cast<uint4*>(U + tc::canon_off(t, k, k1)) = make_uint4(w4[0], w4[1], w4[2], w4[3]);
  }
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  float mx = fmaxf(fmaxf(s_max[0], s_max[1]), fmaxf(s_max[2], s_max[3]));
  int e2 = 0;
  if (mx > 0.f) {
    frexpf(mx, &e2);  // mx in [2^(e2-1), 2^e2)
    e2 = 8 - e2;
  }
  const float sc = ldexpf(1.f, e2), inv_sc = ldexpf(1.f, -e2);
  bool ok = __syncthreads_and(wait_bar(bar_w, 0));
  uint32_t ph = 0;
  auto mma_wait = [&]() -> bool {
    const bool r = __syncthreads_and(wait_bar(bar_m, ph));
    ph ^= 1;
    tc::fence_after_sync();
    return r;
  };
  const float* bias = reinterpret_cast<const float*>(img + o_bias);
  const float4* head = reinterpret_cast<const float4*>(img + o_head);
  const float* hbias = reinterpret_cast<const float*>(img + o_hb);
  const uint32_t img_a = tc::smem_u32(img);
  // ---- forward: h_1 .. h_{L-1} to their tiles, z_L left in TMEM ----
  for (int layer = 0; ok && layer < L; ++layer) {
    const uint32_t K = layer == 0 ? k1 : uint32_t(W);
    if (K > 0) {
      if (t == 0) {
        tc::fence_after_sync();
        const uint32_t a_addr = layer == 0 ? tc::smem_u32(U) : tc::smem_u32(Hb + uint32_t(layer - 1) * TILE);
        const uint32_t b_addr = img_a + (layer == 0 ? 0u : o_wk + uint32_t(layer - 1) * W * W * 2u);
        for (uint32_t ks = 0; ks < K / 16; ++ks)
          tc::mma_f16(tm + C_ACC, tc::sdesc(a_addr + ks * 256u, 128u, K * 16u),
                      tc::sdesc(b_addr + ks * 256u, 128u, K * 16u), tc::idesc_f16_f32(MT, W), ks > 0 ? 1u : 0u);
        tc::mma_commit(bar_m);
      }
      ok = mma_wait();
    }
    if (!ok || layer == L - 1) break;
    unsigned char* dst = Hb + uint32_t(layer) * TILE;
    for (int c0 = 0; c0 < W; c0 += 32) {
      float v[32];
      if (K > 0) {
        tc::tmem_ld32(tm + lb + C_ACC + uint32_t(c0), v);
      } else {
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = 0.f;
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        uint32_t u4[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int i = 8 * q + 2 * e;
          u4[e] = tc::pack_f16x2(tc::tanh_fast(v[i] + bias[layer * W + c0 + i]),
                                 tc::tanh_fast(v[i + 1] + bias[layer * W + c0 + i + 1]));
        }
        *reinterpret_cast<uint4*>(dst + tc::canon_off(t, c0 + 8 * q, W)) = make_uint4(u4[0], u4[1], u4[2], u4[3]);
      }
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
  }
  const bool kL = (L == 1 ? k1 : uint32_t(W)) > 0;  // z_L is in TMEM (else it is zero)
  // ---- head (f32) and the adjoint of its 8 outputs ----
  float dout[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  if (ok) {
    float out[8];
#pragma unroll
    for (int o = 0; o < 8; ++o) out[o] = 0.f;
    for (int c0 = 0; c0 < W; c0 += 32) {
      float v[32];
      if (kL) {
        tc::tmem_ld32(tm + lb + C_ACC + uint32_t(c0), v);
      } else {
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = 0.f;
      }
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const float h = tc::tanh_fast(v[i] + bias[(L - 1) * W + c0 + i]);
        const float4 w0 = head[(c0 + i) * 2], w1 = head[(c0 + i) * 2 + 1];
        out[0] = fmaf(w0.x, h, out[0]);
        out[1] = fmaf(w0.y, h, out[1]);
        out[2] = fmaf(w0.z, h, out[2]);
        out[3] = fmaf(w0.w, h, out[3]);
        out[4] = fmaf(w1.x, h, out[4]);
        out[5] = fmaf(w1.y, h, out[5]);
        out[6] = fmaf(w1.z, h, out[6]);
        out[7] = fmaf(w1.w, h, out[7]);
      }
    }
#pragma unroll
    for (int o = 0; o < 8; ++o) out[o] += hbias[o];
    // d l_u = cot_la 1/2 (delta_uv - p~_u) over the allowed u; d phi_u = cot_ph delta_uv
    if (valid) {
      const unsigned pm = slot_mask(a.hv, p, popc_alpha_tc(x, p), popc_beta_tc(x, p), x), mk = norm_mask(a.hv, p, pm);
      const int v = int((x >> (2 * p)) & 3ull);
      if ((pm >> v) & 1u) {
        float m = -INFINITY;
        for (int u = 0; u < 4; ++u)
          if ((mk >> u) & 1u) m = fmaxf(m, out[u]);
        float ex[4], sum = 0.f;
        for (int u = 0; u < 4; ++u) {
          ex[u] = ((mk >> u) & 1u) ? __expf(out[u] - m) : 0.f;
          sum += ex[u];
        }
        const float c = 0.5f * cla * sc;
        for (int u = 0; u < 4; ++u) dout[u] = ((mk >> u) & 1u) ? c * ((u == v ? 1.f : 0.f) - ex[u] / sum) : 0.f;
        dout[4 + v] = cph * sc;
      }
    }
    // dout tile (fp16, 16 columns: dout, then a one in column 8): B operand of
    // dW_h and of the bias sums
    uint32_t d4[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) d4[e] = tc::pack_f16x2(dout[2 * e], dout[2 * e + 1]);
    *reinterpret_cast<uint4*>(DO + tc::canon_off(t, 0, 16)) = make_uint4(d4[0], d4[1], d4[2], d4[3]);
    *reinterpret_cast<uint4*>(DO + tc::canon_off(t, 8, 16)) = make_uint4(0x3C00u, 0u, 0u, 0u);
    // h_L (fp16) to P1, dz_L = (W_h^T dout) (1 - h_L^2) to P2
    for (int c0 = 0; c0 < W; c0 += 32) {
      float v[32];
      if (kL) {
        tc::tmem_ld32(tm + lb + C_ACC + uint32_t(c0), v);
      } else {
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = 0.f;
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        uint32_t hu[4], zu[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          float hh[2], zz[2];
#pragma unroll
          for (int j = 0; j < 2; ++j) {
            const int i = 8 * q + 2 * e + j, k = c0 + i;
            const float h = tc::tanh_fast(v[i] + bias[(L - 1) * W + k]);
            const float4 w0 = head[k * 2], w1 = head[k * 2 + 1];
            float dh = w0.x * dout[0];
            dh = fmaf(w0.y, dout[1], dh);
            dh = fmaf(w0.z, dout[2], dh);
            dh = fmaf(w0.w, dout[3], dh);
            dh = fmaf(w1.x, dout[4], dh);
            dh = fmaf(w1.y, dout[5], dh);
            dh = fmaf(w1.z, dout[6], dh);
            dh = fmaf(w1.w, dout[7], dh);
            hh[j] = h;
            zz[j] = dh * (1.f - h * h);
          }
          hu[e] = tc::pack_f16x2(hh[0], hh[1]);
          zu[e] = tc::pack_f16x2(zz[0], zz[1]);
        }
        *reinterpret_cast<uint4*>(P1 + tc::canon_off(t, c0 + 8 * q, W)) = make_uint4(hu[0], hu[1], hu[2], hu[3]);
        *reinterpret_cast<uint4*>(P2 + tc::canon_off(t, c0 + 8 * q, W)) = make_uint4(zu[0], zu[1], zu[2], zu[3]);
      }
    }
  }
  // d b_h: column sums of dout over the rows (f32, warp shuffles)
#pragma unroll
  for (int o = 0; o < 8; ++o) {
    float sum = dout[o];
    for (int d = 16; d; d >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, d);
    if (lane == 0) s_bh[warp][o] = sum;
  }
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  const MlpPtrTc P = slot_ptrs_tc(a.m, p);
  float* gbase = a.part + uint64_t(blockIdx.x) * a.n_params;
  if (t < 8) gbase[P.bh + t] = (s_bh[0][t] + s_bh[1][t] + s_bh[2][t] + s_bh[3][t]) * inv_sc;
  // ---- backward: step k = L .. 1; dz_k in Z, the next dz into the other buffer ----
  unsigned char* Z = P2;
  unsigned char* Zn = P1;
  for (int k = L; ok && k >= 1; --k) {
    const bool first = (k == L);
    // dW_k's B operand: h_{k-1} (U for k = 1); it has k1 columns at k = 1
    const uint32_t hprev = k == 1 ? tc::smem_u32(U) : tc::smem_u32(Hb + uint32_t(k - 2) * TILE);
    const uint32_t ncols = k == 1 ? k1 : uint32_t(W);
    if (t == 0) {
      tc::fence_after_sync();
      const uint32_t z = tc::smem_u32(Z);
      if (first)  // dW_h^T[k][o] = sum_r h_L[r][k] dout[r][o]
        for (uint32_t ks = 0; ks < MT / 16; ++ks)
          tc::mma_f16(tm + C_DWH, mn_desc(tc::smem_u32(P1), W, ks), mn_desc(tc::smem_u32(DO), 16, ks),
                      idesc_f16_mn(MT, 16, true, true), ks > 0 ? 1u : 0u);
      if (k >= 2)  // dh_{k-1} = dz_k W_k
        for (uint32_t ks = 0; ks < W / 16; ++ks)
          tc::mma_f16(tm + C_ACC, tc::sdesc(z + ks * 256u, 128u, W * 16u),
                      mn_desc(img_a + o_wk + uint32_t(k - 2) * W * W * 2u, W, ks),
                      idesc_f16_mn(MT, W, false, true), ks > 0 ? 1u : 0u);
      if (ncols > 0)  // dW_k = dz_k^T h_{k-1}
        for (uint32_t ks = 0; ks < MT / 16; ++ks)
          tc::mma_f16(tm + (k == 1 ? C_DW1 : C_DW), mn_desc(z, W, ks), mn_desc(hprev, ncols, ks),
                      idesc_f16_mn(MT, int(ncols), true, true), ks > 0 ? 1u : 0u);
      for (uint32_t ks = 0; ks < MT / 16; ++ks)  // db_k = dz_k^T 1 (column 8)
        tc::mma_f16(tm + C_DB, mn_desc(z, W, ks), mn_desc(tc::smem_u32(DO), 16, ks), idesc_f16_mn(MT, 16, true, true),
                    ks > 0 ? 1u : 0u);
      tc::mma_commit(bar_m);
    }
    ok = mma_wait();
    if (!ok) break;
    // dz_{k-1} = dh_{k-1} (1 - h_{k-1}^2), h_{k-1} from its tile
    if (k >= 2) {
      const unsigned char* hp = Hb + uint32_t(k - 2) * TILE;
      for (int c0 = 0; c0 < W; c0 += 32) {
        float v[32];
        tc::tmem_ld32(tm + lb + C_ACC + uint32_t(c0), v);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const uint4 h4 = *reinterpret_cast<const uint4*>(hp + tc::canon_off(t, c0 + 8 * q, W));
          const uint32_t hw[4] = {h4.x, h4.y, h4.z, h4.w};
          uint32_t zu[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const float2 h2 = __half22float2(*reinterpret_cast<const __half2*>(&hw[e]));
            zu[e] = tc::pack_f16x2(v[8 * q + 2 * e] * (1.f - h2.x * h2.x), v[8 * q + 2 * e + 1] * (1.f - h2.y * h2.y));
          }
          *reinterpret_cast<uint4*>(Zn + tc::canon_off(t, c0 + 8 * q, W)) = make_uint4(zu[0], zu[1], zu[2], zu[3]);
        }
      }
    }
    // dW_k (lane t = output unit t), unscaled, to the tile's partial gradient:
    // 32 columns at a time through shared memory (dz_k's tile, free now), so
    // that each warp store covers 32 consecutive columns of one row
    if (ncols > 0) {
      float* gw = gbase + (k == 1 ? P.W1 : P.Wk + uint64_t(k - 2) * (uint64_t(W) * W + W));
      const uint32_t ld = k == 1 ? 4u * p : uint32_t(W), nvalid = ld;
      float* stage = reinterpret_cast<float*>(Z);  // [128][33]
      for (uint32_t c0 = 0; c0 < ncols; c0 += 32) {
        float v[32];
        if (c0 + 32 <= ncols) {
          tc::tmem_ld32(tm + lb + (k == 1 ? C_DW1 : C_DW) + c0, v);
        } else {
          float v16[16];
          tc::tmem_ld16(tm + lb + (k == 1 ? C_DW1 : C_DW) + c0, v16);
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            v[i] = v16[i];
            v[16 + i] = 0.f;
          }
        }
#pragma unroll
        for (int i = 0; i < 32; ++i) stage[t * 33 + i] = v[i];
        __syncthreads();
        const uint32_t c = c0 + uint32_t(lane);
        if (c < nvalid)
          for (int r = warp; r < MT; r += 4) gw[uint64_t(r) * ld + c] = stage[r * 33 + lane] * inv_sc;
        __syncthreads();
      }
    }
    if (first) {  // dW_h[o][t]
      float v[8];
      tc::tmem_ld8(tm + lb + C_DWH, v);
#pragma unroll
      for (int o = 0; o < 8; ++o) gbase[P.Wh + uint64_t(o) * W + t] = v[o] * inv_sc;
    }
    {  // d b_k[t]
      float v[8];
      tc::tmem_ld8(tm + lb + C_DB + 8u, v);
      gbase[(k == 1 ? P.b1 : P.Wk + uint64_t(k - 2) * (uint64_t(W) * W + W) + uint64_t(W) * W) + t] = v[0] * inv_sc;
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    unsigned char* tmp = Z;
    Z = Zn;
    Zn = tmp;
  }
  if (!ok && t == 0) atomicExch(a.tv.status, ST_TIMEOUT);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tm, NCOL);
}

// One CTA of AT threads per parent x (grid-stride over the parents), its
// threads over the connected x': log psi(x') = parent prefix up to slot j +
// parent slot-j term of v'_j + the terms T[x'][p] of the slots p > j; then
// E_loc(x) = H_xx + sum H_xx' exp(log psi(x') - log psi(x)) with the ratio in
// float32 and the sum in FP64, reduced in a fixed order (deterministic).  The
// suffix terms come per (x', slot) (T[x'][p], MLP and NADE) or already summed
// per x' (T[x'], `tsum`: the transformer, whose suffix kernel holds a
// sequence's positions in one tile).  With so.counts set, the last CTA to
// finish also reduces the statistics of the sample set over every row.
constexpr int AT = 128;
__global__ void __launch_bounds__(AT) eloc_assemble_kernel(int n, uint32_t K, Count n_x_, const uint64_t* __restrict__ xp,
                                                           const uint8_t* __restrict__ js,
                                                           const float* __restrict__ cache,
                                                           const float2* __restrict__ T,
                                                           const double* __restrict__ hval,
                                                           const double* __restrict__ hdiag,
                                                           const float* __restrict__ la_x,
                                                           const float* __restrict__ ph_x, double* __restrict__ ere,
                                                           double* __restrict__ eim, int tsum, StatsOut so) {
  ANQS_PDL_ENTRY();
  __shared__ double red[2][AT / 32];
  __shared__ int s_last;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint64_t n_x = n_x_.get();
  for (uint64_t l = blockIdx.x; l < n_x; l += gridDim.x) {
    const float lx = la_x[l], px = ph_x[l];
    double re = 0.0, im = 0.0;
    for (uint32_t k = threadIdx.x; k < K; k += AT) {
      const uint64_t row = l * K + k;
      const int j = js[row];
      const uint64_t x = xp[row];
      const float* cc = cache + (l * n + j) * CACHE_F;
      const int vj = int((x >> (2 * j)) & 3ull);
      float la = cc[0] + cc[2 + vj], ph = cc[1] + cc[6 + vj];
      if (tsum) {
        if (j + 1 < n) {  // determinants with j = n - 1 have no suffix positions (and no T entry)
          const float2 tv = T[row];
          la += tv.x;
          ph += tv.y;
        }
      } else {
        // the terms of slots j+1 .. n-1, eight loads in flight at a time,
        // added in slot order (the padding adds zeros)
        for (int p0 = j + 1; p0 < n; p0 += 8) {
          float2 tv[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) tv[e] = p0 + e < n ? T[row * n + p0 + e] : make_float2(0.f, 0.f);
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            la += tv[e].x;
            ph += tv[e].y;
          }
        }
      }
      const double h = hval[row];
      const float r = expf(la - lx);
      float s, co;
      sincosf(ph - px, &s, &co);
      const double hr = h * double(r);
      re = fma(hr, double(co), re);
      im = fma(hr, double(s), im);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      re += __shfl_xor_sync(0xffffffffu, re, o);
      im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    if (lane == 0) {
      red[0][w] = re;
      red[1][w] = im;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double sr = 0.0, si = 0.0;
#pragma unroll
      for (int q = 0; q < AT / 32; ++q) {
        sr += red[0][q];
        si += red[1][q];
      }
      ere[l] = hdiag[l] + sr;
      eim[l] = si;
    }
    __syncthreads();
  }
  if (so.counts) {
    if (threadIdx.x == 0) {
      __threadfence();  // this CTA's rows (written by thread 0) before its ticket
      s_last = atomicAdd(so.ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (s_last) {
      __threadfence();
      cta_energy_stats<AT>(ere, eim, so.counts, n_x, so.stats);
    }
  }
}

// Per row: masked half-log-probabilities from the raw slot outputs, prefix
// sums and log psi (and the parent cache when requested).
__global__ void finalize_kernel(HamView hv, const uint64_t* __restrict__ xs, Count n_x_,
                                const float* __restrict__ raw, float* __restrict__ la_out, float* __restrict__ ph_out,
                                float* __restrict__ cache) {
  // one warp per row, lane p = slot p (n <= 32): the slots' loads go out
  // together; the prefix sums are passed from lane to lane in slot order, so
  // they are added in the same order as a running sum over the slots
  ANQS_PDL_ENTRY();
  const int n = hv.n, lane = threadIdx.x & 31;
  const uint64_t n_x = n_x_.get();
  const uint64_t w0 = (blockIdx.x * uint64_t(blockDim.x) + threadIdx.x) >> 5;
  const uint64_t nw = (uint64_t(gridDim.x) * blockDim.x) >> 5;
  for (uint64_t l = w0; l < n_x; l += nw) {
    const uint64_t x = xs[l];
    const int p = lane;
    float tla = 0.f, tph = 0.f;
    bool ok = true;
    if (p < n) {
      const float4* o4 = reinterpret_cast<const float4*>(raw + (l * n + p) * 8);
      const float4 q0 = o4[0], q1 = o4[1];
      const float o[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
      const uint64_t below = (1ull << (2 * p)) - 1ull;  // p < 32
      const int a = __popcll(x & below & 0x5555555555555555ull), b = __popcll(x & below & 0xAAAAAAAAAAAAAAAAull);
      const unsigned pmk = slot_mask(hv, p, a, b, x), mk = norm_mask(hv, p, pmk);
      float mx = -INFINITY;
      for (int u = 0; u < 4; ++u)
        if ((mk >> u) & 1u) mx = fmaxf(mx, o[u]);
      float s = 0.f;
      for (int u = 0; u < 4; ++u)
        if ((mk >> u) & 1u) s += __expf(o[u] - mx);
      const float lse = mx + __logf(s);
      if (cache) {
        float* cc = cache + (l * n + p) * CACHE_F;
        for (int u = 0; u < 4; ++u) {
          cc[2 + u] = ((pmk >> u) & 1u) ? 0.5f * (o[u] - lse) : -INFINITY;
          cc[6 + u] = o[4 + u];
        }
      }
      const int v = int((x >> (2 * p)) & 3ull);
      ok = (pmk >> v) & 1u;
      if (ok) tla = 0.5f * (o[v] - lse);
      tph = o[4 + v];
    }
    // a row is dead from its first unphysical slot on (from the start if it
    // has bits above its 2n qubits): its later slots add nothing to la
    const bool high = (n < 32) && ((x >> (2 * n)) != 0);
    const unsigned bad = __ballot_sync(0xffffffffu, !ok);
    const int first_bad = high ? 0 : bad ? __ffs(bad) - 1 : 32;
    if (p >= first_bad) tla = 0.f;
    float run_la = 0.f, run_ph = 0.f;  // sum over the slots before p
    for (int k = 1; k < n; ++k) {
      const float il = __shfl_sync(0xffffffffu, run_la + tla, k - 1);
      const float ip = __shfl_sync(0xffffffffu, run_ph + tph, k - 1);
      if (lane == k) {
        run_la = il;
        run_ph = ip;
      }
    }
    if (cache && p < n) {
      float* cc = cache + (l * n + p) * CACHE_F;
      cc[0] = run_la;
      cc[1] = run_ph;
    }
    const float tot_la = __shfl_sync(0xffffffffu, run_la + tla, n - 1);
    const float tot_ph = __shfl_sync(0xffffffffu, run_ph + tph, n - 1);
    if (lane == 0) {
      const bool dead = bad != 0 || high;
      la_out[l] = dead ? -INFINITY : tot_la;
      ph_out[l] = tot_ph;
    }
  }
}

// ---- sort of connected rows by first differing slot ---------------------------
// Histogram of the first slots into ctl[0, n) (zero on entry); the last CTA
// to finish then writes cursor[i] = offsets[i] = rows with first slot < i
// (exclusive prefix sums) and offsets[n] = rows.
__global__ void js_hist_kernel(const uint8_t* __restrict__ js, Count m_, int n, uint32_t* __restrict__ ctl,
                               uint32_t* __restrict__ cursor, uint32_t* __restrict__ offsets) {
  ANQS_PDL_ENTRY();
  __shared__ uint32_t h[ANQS_MAX_ORB];
  __shared__ int s_last;
  const uint64_t m = m_.get();
  for (int i = threadIdx.x; i < n; i += blockDim.x) h[i] = 0;
  __syncthreads();
  for (uint64_t t = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; t < m; t += uint64_t(gridDim.x) * blockDim.x)
    atomicAdd(&h[js[t]], 1u);
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    if (h[i]) atomicAdd(&ctl[i], h[i]);
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&ctl[TC_CTL_SORT_TICKET], 1u) == gridDim.x - 1;
  __syncthreads();
  if (s_last && threadIdx.x < 32) {  // one warp, lane i = slot i (n <= 32): an inclusive scan
    __threadfence();
    const int i = threadIdx.x;
    const uint32_t h_i = i < n ? __ldcg(ctl + i) : 0u;
    uint32_t inc = h_i;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t v = __shfl_up_sync(0xffffffffu, inc, o);
      if (i >= o) inc += v;
    }
    if (i < n) {
      cursor[i] = inc - h_i;
      offsets[i] = inc - h_i;
    }
    if (i == n - 1) offsets[n] = inc;
  }
}

__global__ void js_scatter_kernel(const uint8_t* __restrict__ js, Count m_, uint32_t* __restrict__ cursor,
                                  uint32_t* __restrict__ perm) {
  ANQS_PDL_ENTRY();
  const uint64_t m = m_.get();
  const int lane = threadIdx.x & 31;
  for (uint64_t t0 = blockIdx.x * uint64_t(blockDim.x); t0 < m; t0 += uint64_t(gridDim.x) * blockDim.x) {
    const uint64_t t = t0 + threadIdx.x;
    const int key = t < m ? int(js[t]) : -1;
    // lanes with the same key reserve their slots with one atomic
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    const int leader = __ffs(peers) - 1;
    const int rank = __popc(peers & ((1u << lane) - 1u));
    uint32_t base = 0;
    if (lane == leader && key >= 0) base = atomicAdd(&cursor[key], uint32_t(__popc(peers)));
    base = __shfl_sync(peers, base, leader);
    if (key >= 0) perm[base + rank] = uint32_t(t);
  }
}

// All three steps in one CTA for up to JS_SMALL rows: histogram in shared
// memory, offsets (offsets[n] = rows), scatter with warp-aggregated shared
// atomics.
constexpr uint64_t JS_SMALL = 8192;
__global__ void __launch_bounds__(1024) js_sort_small_kernel(const uint8_t* __restrict__ js, Count m_, int n,
                                                             uint32_t* __restrict__ offsets,
                                                             uint32_t* __restrict__ perm) {
  ANQS_PDL_ENTRY();
  __shared__ uint32_t h[ANQS_MAX_ORB], cur[ANQS_MAX_ORB];
  const uint64_t m = m_.get();
  const int lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < n; i += blockDim.x) h[i] = 0;
  __syncthreads();
  for (uint64_t t = threadIdx.x; t < m; t += blockDim.x) atomicAdd(&h[js[t]], 1u);
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t acc = 0;
    for (int i = 0; i < n; ++i) {
      cur[i] = acc;
      offsets[i] = acc;
      acc += h[i];
    }
    offsets[n] = acc;
  }
  __syncthreads();
  for (uint64_t t0 = 0; t0 < m; t0 += blockDim.x) {
    const uint64_t t = t0 + threadIdx.x;
    const int key = t < m ? int(js[t]) : -1;
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    const int leader = __ffs(peers) - 1;
    const int rank = __popc(peers & ((1u << lane) - 1u));
    uint32_t base = 0;
    if (lane == leader && key >= 0) base = atomicAdd(&cur[key], uint32_t(__popc(peers)));
    base = __shfl_sync(peers, base, leader);
    if (key >= 0) perm[base + rank] = uint32_t(t);
  }
}

int g_num_sms = 0;

int num_sms() {
  if (!g_num_sms) {
    int dev = 0;
    ANQS_CUDA(cudaGetDevice(&dev));
    ANQS_CUDA(cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev));
  }
  return g_num_sms;
}

constexpr size_t kSmemLimit = 227 * 1024;

size_t smem_bytes(const TcView& tv, int nbuf) {
  return size_t(round_up(tv.max_img, 1024u)) * nbuf + size_t(NWG) * MT * tv.kmax * 2u;
}

TcView make_view(const anqs_model* M) {
  TcView tv;
  tv.n = M->d.n_orb;
  tv.W = M->d.width;
  tv.L = M->d.n_hidden;
  tv.lo = use_w1_split(tv.n, tv.W, tv.L);
  tv.img = static_cast<const unsigned char*>(M->packed);
  tv.max_img = 0;
  for (int p = 0; p <= tv.n; ++p) tv.img_off[p] = uint32_t(M->pack_off[p]);
  for (int p = 0; p < tv.n; ++p) tv.max_img = std::max(tv.max_img, slot_layout(p, tv.W, tv.L, tv.lo).bytes);
  tv.kmax = std::max<uint32_t>(tv.W, round_up(4u * (tv.n - 1), 16u));
  tv.nbuf = smem_bytes(tv, 2) <= kSmemLimit ? 2 : 1;
  tv.status = reinterpret_cast<int*>(static_cast<unsigned char*>(M->packed) + M->pack_off[tv.n]);
  return tv;
}

template <int W>
int launch_slots_w(const TcView& tv, const TileArgs& ta, cudaStream_t s) {
  const uint64_t max_rows = ta.rows.n;
  const size_t sm = smem_bytes(tv, 1);
  // one 128-row tile per CTA (its warpgroup alone on the SM) while the
  // tiles of all slots fit in one wave, else NWG tiles per CTA
  const uint64_t np = uint64_t(ta.p_hi - ta.p_lo);
  uint64_t tiles = (max_rows + MT - 1) / MT * np;
  if (ta.levels) {
    tiles = 0;
    for (int q = 0; q < ta.levels; ++q) tiles += (uint64_t(ta.lv_off[q + 1] - ta.lv_off[q]) + MT - 1) / MT;
  }
  TileArgs a = ta;
  a.tpi = tiles <= uint64_t(num_sms()) ? 1 : NWG;
  uint64_t items = (max_rows + uint64_t(a.tpi) * MT - 1) / (uint64_t(a.tpi) * MT) * np;
  if (ta.levels) {
    items = 0;
    for (int q = 0; q < ta.levels; ++q)
      items += (uint64_t(ta.lv_off[q + 1] - ta.lv_off[q]) + uint64_t(a.tpi) * MT - 1) / (uint64_t(a.tpi) * MT);
  }
  const unsigned grid = unsigned(std::min<uint64_t>(items ? items : 1, uint64_t(num_sms())));
  TcView v1 = tv;
  v1.nbuf = 1;
  ANQS_CUDA(cudaFuncSetAttribute(mlp_tc_slots_kernel<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm)));
  ANQS_CUDA_LAUNCH("mlp_tc_slots_kernel", launch_k(mlp_tc_slots_kernel<W>, dim3(grid), dim3(NT), sm, s, v1, a));
  return ANQS_OK;
}

int launch_slots(const anqs_model* M, const TileArgs& ta, cudaStream_t s, int prof) {
  TcView tv = make_view(M);
  if (smem_bytes(tv, 1) > kSmemLimit) return set_error(ANQS_ERR_UNSUPPORTED, "BF16 MLP slot image too large");
  ProfScope ps(prof, s);
  return tv.W == 128 ? launch_slots_w<128>(tv, ta, s) : launch_slots_w<64>(tv, ta, s);
}

int launch_finalize(const HamView& hv, const uint64_t* x, Count n_x, const float* raw, float* la, float* ph,
                    float* cache, cudaStream_t s) {
  uint64_t blocks = (n_x.n + 3) / 4;  // four rows (warps) per CTA of 128 threads
  if (blocks > 152 * 16) blocks = 152 * 16;
  ANQS_CUDA_LAUNCH("finalize_kernel", launch_k(finalize_kernel, dim3(unsigned(blocks ? blocks : 1)), dim3(128), 0, s, hv, x, n_x, raw, la, ph, cache));
  return ANQS_OK;
}

struct ElocWs {
  uint64_t* xp;
  double* hv;
  uint8_t* js;
  double* hd;
  float *la_x, *ph_x, *raw, *cache;
  float2* T;
  uint32_t *perm, *hist, *cursor, *offsets, *ticket;
};

size_t plan_eloc(const anqs_ham* H, uint64_t n_x, Arena& A, ElocWs& w) {
  const uint64_t m = n_x * H->v.K;
  w.xp = A.take<uint64_t>(m);
  w.hv = A.take<double>(m);
  w.js = A.take<uint8_t>(m);
  w.hd = A.take<double>(n_x);
  w.la_x = A.take<float>(n_x);
  w.ph_x = A.take<float>(n_x);
  w.raw = A.take<float>(n_x * H->v.n * 8);
  w.cache = A.take<float>(n_x * H->v.n * CACHE_F);
  w.T = A.take<float2>(m * H->v.n);
  w.perm = A.take<uint32_t>(m);
  w.cursor = A.take<uint32_t>(ANQS_MAX_ORB);
  w.offsets = A.take<uint32_t>(ANQS_MAX_ORB + 1);
  w.hist = A.take<uint32_t>(TC_CTL_WORDS);
  w.ticket = w.hist + TC_CTL_STATS_TICKET;
  return A.off;
}

template <int W>
int launch_ws_w(const TcView& tv, const HamView& hv, const ElocWs& w, cudaStream_t s) {
  const size_t sm = smem_bytes(tv, 1);
  const unsigned grid = unsigned(std::max(num_sms(), tv.n));
  ANQS_CUDA(cudaFuncSetAttribute(mlp_tc_ws_kernel<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm)));
  ANQS_CUDA_LAUNCH("mlp_tc_ws_kernel", launch_k(mlp_tc_ws_kernel<W>, dim3(grid), dim3(NT), sm, s, tv, hv, w.xp, w.perm, w.offsets, w.T));
  return ANQS_OK;
}

}  // namespace

int mlp_tc_pack_alloc(anqs_model* M) {
  const int n = M->d.n_orb, W = M->d.width, L = M->d.n_hidden;
  if (W != 64 && W != 128) return set_error(ANQS_ERR_UNSUPPORTED, "BF16 MLP form supports width 64 or 128");
  const int lo = use_w1_split(n, W, L);
  M->pack_off.assign(n + 1, 0);
  uint64_t off = 0;
  for (int p = 0; p < n; ++p) {
    M->pack_off[p] = off;
    off += slot_layout(p, W, L, lo).bytes;
  }
  M->pack_off[n] = off;  // status word after the images
  M->packed_bytes = off + 256;
  TcView tv;
  tv.n = n;
  tv.W = W;
  tv.L = L;
  tv.lo = lo;
  tv.max_img = 0;
  for (int p = 0; p < n; ++p) tv.max_img = std::max(tv.max_img, slot_layout(p, W, L, lo).bytes);
  tv.kmax = std::max<uint32_t>(W, round_up(4u * (n - 1), 16u));
  if (smem_bytes(tv, 1) > kSmemLimit)
    return set_error(ANQS_ERR_UNSUPPORTED, "BF16 MLP slot image too large for shared memory (%zu bytes)",
                     smem_bytes(tv, 1));
  ANQS_CUDA(cudaMalloc(&M->packed, M->packed_bytes));
  ANQS_CUDA(cudaMemset(M->packed, 0, M->packed_bytes));
  M->tc_raw_rows = 32768;
  ANQS_CUDA(cudaMalloc(&M->tc_raw, M->tc_raw_rows * n * 8 * sizeof(float)));
  ANQS_CUDA(cudaStreamCreateWithFlags(&M->side, cudaStreamNonBlocking));
  ANQS_CUDA(cudaEventCreateWithFlags(&M->ev_fork, cudaEventDisableTiming));
  ANQS_CUDA(cudaEventCreateWithFlags(&M->ev_join, cudaEventDisableTiming));
  return ANQS_OK;
}

int mlp_tc_pack(anqs_model* M, cudaStream_t s) {
  TcView tv = make_view(M);
  dim3 grid(64, unsigned(M->d.n_orb));
  ANQS_CUDA_LAUNCH("pack_kernel", launch_k(pack_kernel, dim3(grid), dim3(256), 0, s, M->mlp, tv, static_cast<unsigned char*>(M->packed)));
  return ANQS_OK;
}

int mlp_tc_status(const anqs_model* M, int* status) {
  int v = 0;
  ANQS_CUDA(cudaMemcpy(&v, static_cast<const unsigned char*>(M->packed) + M->pack_off[M->d.n_orb], sizeof(int),
                       cudaMemcpyDeviceToHost));
  *status = v;
  return ANQS_OK;
}

// anqs_logpsi in the BF16 form: chunks of the model's scratch rows.
int launch_mlp_tc_logpsi(const anqs_model* M, const HamView& hv, const uint64_t* x, uint64_t n_x, float* la,
                         float* ph, cudaStream_t s) {
  for (uint64_t off = 0; off < n_x; off += M->tc_raw_rows) {
    const uint64_t k = std::min<uint64_t>(M->tc_raw_rows, n_x - off);
    TileArgs ta{};
    ta.x = x + off;
    ta.rows = host_count(k);
    ta.p_lo = 0;
    ta.p_hi = M->d.n_orb;
    ta.raw = M->tc_raw;
    ANQS_TRY(launch_slots(M, ta, s, PROF_TC_PARENT));
    ProfScope ps(PROF_TC_FINALIZE, s);
    ANQS_TRY(launch_finalize(hv, x + off, host_count(k), M->tc_raw, la + off, ph + off, nullptr, s));
  }
  return ANQS_OK;
}

int launch_mlp_tc_prefix_logits(const anqs_model* M, const anqs_ham* H, float* out8, cudaStream_t s,
                                ZeroWords zero) {
  const int n = H->v.n;
  TileArgs ta{};
  ta.zero = zero;
  ta.x = H->d_pt_x;
  ta.rows = host_count(H->pt_x.size());
  ta.p_lo = 0;
  ta.p_hi = 1;
  ta.raw = out8;
  ta.levels = n;
  for (int q = 0; q <= n; ++q) ta.lv_off[q] = H->pt_off[q];
  return launch_slots(M, ta, s, PROF_TC_SLOT);
}

int launch_mlp_tc_slot_logits(const anqs_model* M, const HamView& hv, int p, const uint64_t* pre,
                              const uint64_t* n_dev, uint64_t max_rows, float* out8, cudaStream_t s) {
  (void)hv;
  TileArgs ta{};
  ta.x = pre;
  ta.rows = Count{max_rows, n_dev, 1};
  ta.p_lo = p;
  ta.p_hi = p + 1;
  ta.raw = out8;
  return launch_slots(M, ta, s, PROF_TC_SLOT);
}

int launch_tc_finalize(const HamView& hv, const uint64_t* x, Count n_x, const float* raw, float* la, float* ph,
                       float* cache, cudaStream_t s) {
  return launch_finalize(hv, x, n_x, raw, la, ph, cache, s);
}

int launch_js_sort(const uint8_t* js, Count mc, int n, uint32_t* ctl, uint32_t* cursor, uint32_t* offsets,
                   uint32_t* perm, cudaStream_t s) {
  if (mc.n <= JS_SMALL) {
    ANQS_CUDA_LAUNCH("js_sort_small_kernel", launch_k(js_sort_small_kernel, dim3(1), dim3(1024), 0, s, js, mc, n, offsets, perm));
    return ANQS_OK;
  }
  const unsigned g = unsigned(std::min<uint64_t>((mc.n + 255) / 256, 152 * 4));
  ANQS_CUDA_LAUNCH("js_hist_kernel", launch_k(js_hist_kernel, dim3(g ? g : 1), dim3(256), 0, s, js, mc, n, ctl, cursor, offsets));
  ANQS_CUDA_LAUNCH("js_scatter_kernel", launch_k(js_scatter_kernel, dim3(g ? g : 1), dim3(256), 0, s, js, mc, cursor, perm));
  return ANQS_OK;
}

int launch_eloc_assemble(int n, uint32_t K, Count n_x, const uint64_t* xp, const uint8_t* js, const float* cache,
                         const float2* T, const double* hval, const double* hdiag, const float* la_x,
                         const float* ph_x, double* ere, double* eim, const StatsOut& so, cudaStream_t s,
                         bool tsum) {
  uint64_t blocks = n_x.n;
  if (blocks > 152 * 16) blocks = 152 * 16;
  ANQS_CUDA_LAUNCH("eloc_assemble_kernel", launch_k(eloc_assemble_kernel, dim3(unsigned(blocks ? blocks : 1)), dim3(AT), 0, s, n, K, n_x, xp, js, cache, T, hval, hdiag, la_x, ph_x, ere, eim, tsum ? 1 : 0, so));
  return ANQS_OK;
}

size_t eloc_tc_workspace(const anqs_model* M, const anqs_ham* H, uint64_t n_x) {
  (void)M;
  Arena A(nullptr, 0);
  ElocWs w;
  return plan_eloc(H, n_x, A, w);
}

// The local energy of one problem in three stages, so that a batch can run
// the middle one for many problems in one launch.
//   pre:    connected set, parents' slots and caches, sort by first slot
//   suffix: the connected determinants' slots p > j (mlp_tc_ws_kernel)
//   post:   E_loc assembly
static int plan_ws(const anqs_ham* H, Count n_x, void* ws, size_t ws_bytes, ElocWs& w) {
  Arena A(ws, ws_bytes);
  plan_eloc(H, n_x.n, A, w);
  if (!A.fits()) return set_error(ANQS_ERR_CAPACITY, "workspace needs %zu bytes", A.off);
  if (n_x.n * H->v.K > 0xffffffffull)
    return set_error(ANQS_ERR_UNSUPPORTED, "more than 2^32 connected determinants per call");
  return ANQS_OK;
}

// Two independent chains: the connected set and its sort by first slot (on
// s), the parents' slot outputs and finalize (on sp: the model's second
// stream when forking).  The control words are zeroed by the connected-set
// kernel, on the stream of the histogram and the assembly that use them.
int eloc_tc_pre(const anqs_model* M, const anqs_ham* H, const uint64_t* x, Count n_x, void* ws, size_t ws_bytes,
                cudaStream_t s, bool fork) {
  ElocWs w;
  ANQS_TRY(plan_ws(H, n_x, ws, ws_bytes, w));
  const Count mc = scaled(n_x, H->v.K);
  cudaStream_t sp = s;
  if (fork && M->side) {
    ANQS_CUDA(cudaEventRecord(M->ev_fork, s));
    ANQS_CUDA(cudaStreamWaitEvent(M->side, M->ev_fork, 0));
    sp = M->side;
  }
  int r = launch_connected(H->v, x, n_x, w.xp, w.hv, w.js, w.hd, s, w.hist);
  if (r == ANQS_OK) {
    TileArgs ta{};
    ta.x = x;
    ta.rows = n_x;
    ta.p_lo = 0;
    ta.p_hi = H->v.n;
    ta.raw = w.raw;
    r = launch_slots(M, ta, sp, PROF_TC_PARENT);
    if (r == ANQS_OK) {
      ProfScope ps(PROF_TC_FINALIZE, sp);
      r = launch_finalize(H->v, x, n_x, w.raw, w.la_x, w.ph_x, w.cache, sp);
    }
  }
  if (r == ANQS_OK) {
    ProfScope ps(PROF_TC_SORT, s);
    r = launch_js_sort(w.js, mc, H->v.n, w.hist, w.cursor, w.offsets, w.perm, s);
  }
  if (sp != s) {  // join, also after an error, so that no work of the call is left outside s
    if (cudaEventRecord(M->ev_join, sp) != cudaSuccess || cudaStreamWaitEvent(s, M->ev_join, 0) != cudaSuccess) {
      cudaGetLastError();
      if (r == ANQS_OK) r = set_error(ANQS_ERR_CUDA, "stream join");
    }
  }
  return r;
}

int eloc_tc_post(const anqs_ham* H, Count n_x, double* ere, double* eim, const uint64_t* counts, double* stats,
                 void* ws, size_t ws_bytes, cudaStream_t s) {
  ElocWs w;
  ANQS_TRY(plan_ws(H, n_x, ws, ws_bytes, w));
  ProfScope ps(PROF_TC_ELOC, s);
  return launch_eloc_assemble(H->v.n, uint32_t(H->v.K), n_x, w.xp, w.js, w.cache, w.T, w.hv, w.hd, w.la_x, w.ph_x,
                              ere, eim, StatsOut{counts, stats, w.ticket}, s);
}

int run_eloc_tc(const anqs_model* M, const anqs_ham* H, const uint64_t* x, Count n_x, double* ere, double* eim,
                const uint64_t* counts, double* stats, void* ws, size_t ws_bytes, cudaStream_t s) {
  ElocWs w;
  ANQS_TRY(plan_ws(H, n_x, ws, ws_bytes, w));
  ANQS_TRY(eloc_tc_pre(M, H, x, n_x, ws, ws_bytes, s, true));
  {
    TcView tv = make_view(M);
    ProfScope ps(PROF_TC_SUFFIX, s);
    ANQS_TRY(tv.W == 128 ? launch_ws_w<128>(tv, H->v, w, s) : launch_ws_w<64>(tv, H->v, w, s));
  }
  return eloc_tc_post(H, n_x, ere, eim, counts, stats, ws, ws_bytes, s);
}

// Shared memory of the tensor-core adjoint of model M (0 when it does not
// apply: width other than 128, more than 3 hidden layers, or too large).
static size_t tc_grad_smem(const anqs_model* M, uint32_t* img_bytes, uint32_t* kmax1) {
  const int n = M->d.n_orb, W = M->d.width, L = M->d.n_hidden;
  if (W != 128 || L < 1 || L > 3) return 0;
  const int lo = use_w1_split(n, W, L);
  uint32_t img = 0, k1 = 0;
  for (int p = 0; p < n; ++p) {
    const SlotLayout S = slot_layout(p, W, L, lo);
    img = std::max(img, S.w1lo + (S.head16 - S.wk));
    k1 = std::max(k1, S.k1);
  }
  img = round_up(img, 1024u);
  if (img_bytes) *img_bytes = img;
  if (kmax1) *kmax1 = k1;
  const size_t tile = size_t(MT) * W * 2;
  const size_t sm = size_t(img) + size_t(L - 1) * tile + 2 * tile + size_t(MT) * k1 * 2 + size_t(MT) * 16 * 2;
  return sm <= kSmemLimit ? sm : 0;
}

bool mlp_tc_grad_supported(const anqs_model* M) { return tc_grad_smem(M, nullptr, nullptr) > 0; }

// The VMC gradient of a 16-bit MLP on the tensor cores: per-tile partial
// gradients in `part` ([tiles][n_params], tiles of 128 rows), then their sum.
int launch_mlp_tc_grad(const anqs_model* M, const HamView& hv, const uint64_t* x, Count n_x, const CotSrc& cot,
                       float* grad, float* part, cudaStream_t s) {
  GradArgs a{};
  const size_t sm = tc_grad_smem(M, &a.img_bytes, &a.kmax1);
  if (!sm) return set_error(ANQS_ERR_UNSUPPORTED, "tensor-core adjoint does not apply to this model");
  if (!part) return set_error(ANQS_ERR_ARG, "tensor-core adjoint needs the partial-gradient workspace");
  a.tv = make_view(M);
  a.m = M->mlp;
  a.hv = hv;
  a.xs = x;
  a.n_x = n_x;
  a.cot = cot;
  a.part = part;
  a.n_params = M->mlp.slot_off[M->mlp.n];
  const uint64_t tiles = std::max<uint64_t>((n_x.n + MT - 1) / MT, 1);
  if (tiles > 0x7fffffffull) return set_error(ANQS_ERR_UNSUPPORTED, "too many rows");
  ANQS_CUDA(cudaFuncSetAttribute(mlp_tc_grad_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm)));
  {
    ProfScope ps(PROF_MLP_TC_GRAD, s);
    ANQS_CUDA_LAUNCH("mlp_tc_grad_kernel", launch_k(mlp_tc_grad_kernel<128>, dim3(unsigned(tiles), unsigned(M->d.n_orb)),
                                                    dim3(MT), sm, s, a));
  }
  return launch_grad_partial_sum(part, n_x, a.n_params, MT, grad, s);
}

int mlp_tc_multi_max() { return kMaxBatch; }

size_t mlp_tc_multi_groups_bytes() { return size_t(kMaxBatch) * ANQS_MAX_ORB * sizeof(MultiGroup); }

// The suffix stage of n problems (16-bit MLPs of one width, each after its
// pre stage) in one plan launch and one persistent launch on s.
int launch_mlp_tc_multi(const MultiEloc* q, int n, int chunk, int dynamic, void* groups, uint32_t* ctl,
                        cudaStream_t s) {
  if (n < 1 || n > kMaxBatch) return set_error(ANQS_ERR_ARG, "%d problems for one multi-problem launch", n);
  if (chunk < 1) return set_error(ANQS_ERR_ARG, "chunk must be >= 1");
  MultiArgs a{};
  a.n_prob = n;
  a.chunk = chunk;
  a.dynamic = dynamic ? 1 : 0;
  a.groups = static_cast<MultiGroup*>(groups);
  a.ctl = ctl;
  int W = 0;
  for (int k = 0; k < n; ++k) {
    const TcView tv = make_view(q[k].model);
    if (k == 0) W = tv.W;
    if (tv.W != W) return set_error(ANQS_ERR_ARG, "multi-problem launch needs one network width");
    ElocWs w;
    ANQS_TRY(plan_ws(q[k].ham, host_count(q[k].n_x), q[k].ws, q[k].ws_bytes, w));
    a.prob[k].tv = tv;
    a.prob[k].hv = q[k].ham->v;
    a.prob[k].xp = w.xp;
    a.prob[k].perm = w.perm;
    a.prob[k].offsets = w.offsets;
    a.prob[k].T = w.T;
    a.max_img = std::max(a.max_img, tv.max_img);
    a.kmax = std::max(a.kmax, tv.kmax);
  }
  const size_t sm = size_t(round_up(a.max_img, 1024u)) + size_t(NWG) * MT * a.kmax * 2u;
  if (sm > kSmemLimit) return set_error(ANQS_ERR_UNSUPPORTED, "multi-problem launch needs %zu bytes of shared memory", sm);
  ProfScope ps(PROF_TC_SUFFIX, s);
  ANQS_CUDA_LAUNCH("multi_plan_kernel", launch_k(multi_plan_kernel, dim3(1), dim3(256), 0, s, a));
  if (W == 128) {
    ANQS_CUDA(cudaFuncSetAttribute(mlp_tc_multi_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm)));
    ANQS_CUDA_LAUNCH("mlp_tc_multi_kernel", launch_k(mlp_tc_multi_kernel<128>, dim3(num_sms()), dim3(NT), sm, s, a));
  } else {
    ANQS_CUDA(cudaFuncSetAttribute(mlp_tc_multi_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm)));
    ANQS_CUDA_LAUNCH("mlp_tc_multi_kernel", launch_k(mlp_tc_multi_kernel<64>, dim3(num_sms()), dim3(NT), sm, s, a));
  }
  return ANQS_OK;
}

}  // namespace anqs
