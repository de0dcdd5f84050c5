// 16-bit tensor-core form of the causal-transformer ansatz (d = 64): tcgen05
// MMAs with TMEM accumulators for every projection, with reuse of the parent
// determinant's keys and values for its connected determinants.
//
// The GEMM operands (weights, LayerNorm outputs, attention outputs, FFN
// hidden units) and the stored keys and values are fp16, not bf16: the same
// MMA instruction at the same rate, but an 11-bit significand, which cuts the
// activation rounding error of the log-amplitudes eightfold.  The activations
// of this network are O(1) to O(10), far inside fp16's range; conversions
// saturate at +-65504 rather than overflow.  Weights that are bf16 values are
// fp16 values too (down to 2^-17 in magnitude).
//
// A CTA runs two warpgroups; each owns a tile of 128 rows (one row = one
// (sequence, position) pair = one thread = one TMEM lane).  The residual
// stream of a row stays in the registers of its thread.  Per block:
//   LN1 -> A (fp16, canonical K-major)      MMA  qkv = A Wqkv^T   (N = 192)
//   k, v (+bias) -> shared memory (fp16)     causal attention per row on the
//   CUDA cores (online softmax over the keys 0..t) -> A
//   MMA  o = A Wo^T (N = 64)                 h += o + bo;  LN2 -> A
//   FFN in 4 chunks of 64 hidden units: MMA f1_c = A W1_c^T, ReLU -> H_c
//   (fp16), MMA acc2 += H_c W2_c^T; f1_{c+1} runs while chunk c's epilogue
//   does, H alternates between two buffers.   h += acc2 + b2
// then LNf and the f32 head (8 outputs).  Weights of a block sit in two
// bulk-copied halves (q|k|v|o: 32 KB, FFN: 64 KB); each half of the next
// block (or of the next tile's first block) is fetched as soon as the MMAs
// that read the current one are done.
//
// Modes
//   FULL    sequences x[s] (determinants or sampler prefixes), positions
//           0..P-1: the 8 raw outputs of every position (or of the last one
//           only), optionally the keys and values of every position and block
//           (the parent cache).
//   SUFFIX  connected determinants x', grouped by first differing slot j:
//           positions t = j+1..n-1 only (positions <= j see the same tokens as
//           in the parent x, Eq. anqs_def); keys and values of positions <= j
//           come from the parent cache; writes the sum over those positions of
//           the masked slot terms, one (log|psi|, phase) pair T[x'] per
//           connected determinant (a sequence's positions are rows of one tile).
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "tc_ptx.cuh"

namespace anqs {

// d_model 128 (tf_tc128.cu)
bool tf128_supported(const anqs_model* M);
size_t tf128_packed_bytes(const anqs_model* M);
int tf128_pack(anqs_model* M, cudaStream_t s);
int tf128_status_offset(const anqs_model* M);
int launch_tf128_full(const anqs_model* M, const HamView& hv, const uint64_t* x, Count n_seq, int P, int last_only,
                      float* raw, __half* kv_out, int prof, cudaStream_t s);
int launch_tf128_suffix(const anqs_model* M, const HamView& hv, const uint64_t* xp, const uint32_t* perm,
                        const uint32_t* offsets, uint32_t K, const __half* kv_in, float2* T, uint64_t m_max,
                        int prof, cudaStream_t s);

namespace {

constexpr int D = 64;
constexpr int MT = 128;
constexpr int NWG = 2;
constexpr int NT = NWG * MT;
constexpr uint32_t WQKV_BYTES = 3 * D * D * 2;             // [3D][D]
constexpr uint32_t WA_BYTES = 4 * D * D * 2;               // q|k|v rows then Wo [D][D]
constexpr uint32_t WF_BYTES = 8 * D * D * 2;               // W1 chunks [4][D][D], W2 chunks [4][D][D]
constexpr uint32_t LAYER_BYTES = WA_BYTES + WF_BYTES;
constexpr uint32_t A_BYTES = MT * D * 2;                    // one A operand tile (K = 64)
constexpr uint32_t KV_STRIDE = 2 * D * 2 + 16;              // bytes per row of k|v (padded)
constexpr uint32_t KV_BYTES = MT * KV_STRIDE;               // also holds the two FFN hidden chunks
constexpr uint32_t TP_FLOATS = (5 + ANQS_MAX_ORB) * D;     // tok, pos
constexpr uint32_t OFF_WA = 0, OFF_WF = WA_BYTES, OFF_WG = WA_BYTES + WF_BYTES;
constexpr uint32_t WG_BYTES = A_BYTES + KV_BYTES;
constexpr uint32_t OFF_TP = OFF_WG + NWG * WG_BYTES;
constexpr uint32_t OFF_HEAD = OFF_TP + TP_FLOATS * 4;
constexpr int kMaxL = 4;                                   // blocks of the 16-bit d-64 form
constexpr uint32_t LP_FLOATS = 13 * D;                     // per block: ln1 g,b | bq bk bv bo | ln2 g,b | b1 (4D) | b2
constexpr uint32_t OFF_LP = OFF_HEAD + (8 * D + 8) * 4;    // every block's, then the final LayerNorm's g, b
constexpr uint32_t SMEM_BYTES = OFF_LP + (kMaxL * LP_FLOATS + 2 * D) * 4;
constexpr uint32_t TMEM_WG = 256;  // columns per warpgroup: [0,192) qkv / o / f1 buffers, [192,256) acc2
constexpr uint64_t kWaitNs = 2000000000ull;
constexpr int MODE_FULL = 0, MODE_SUFFIX = 1;
static_assert(2 * A_BYTES <= KV_BYTES, "hidden chunks live in the k|v region");
static_assert(SMEM_BYTES <= 227 * 1024, "shared memory");

struct Args {
  const unsigned char* img;  // packed fp16 blocks
  const float* params;       // f32 parameters (tok, pos, LayerNorms, biases, head)
  int n, L;
  HamView hv;
  int mode;
  // FULL
  const uint64_t* x;
  Count n_seq;
  int P, last_only;
  float* raw;
  __half* kv_out;
  // SUFFIX
  const uint64_t* xp;
  const uint32_t* perm;
  const uint32_t* offsets;
  uint32_t K;
  const __half* kv_in;
  float2* T;
  int* status;
};

struct LayerP {
  const float *ln1_g, *ln1_b, *bq, *bk, *bv, *bo, *ln2_g, *ln2_b, *b1, *b2;
};

__device__ __forceinline__ LayerP layer_p(const float* params, int n, int l) {
  const size_t per = 12 * size_t(D) * D + 13 * D;
  const float* b = params + 5 * D + size_t(n) * D + size_t(l) * per;
  LayerP P;
  P.ln1_g = b;
  P.ln1_b = b + D;
  P.bq = b + 2 * D + D * D;
  P.bk = P.bq + D + D * D;
  P.bv = P.bk + D + D * D;
  P.bo = P.bv + D + D * D;
  P.ln2_g = P.bo + D;
  P.ln2_b = P.ln2_g + D;
  P.b1 = P.ln2_b + D + 4 * D * D;
  P.b2 = P.b1 + 4 * D + 4 * D * D;
  return P;
}

// ---- packing: f32 parameters -> per-block fp16 canonical images ---------------
__global__ void tf_pack_kernel(const float* __restrict__ params, int n, int L, unsigned char* __restrict__ img) {
  // no early trigger: a later kernel's prologue may read the packed images
  // before its own dependency wait, so the images are complete before any
  // dependent launch starts
  ANQS_PDL_WAIT();
  const size_t per = 12 * size_t(D) * D + 13 * D;
  const uint32_t per_layer = LAYER_BYTES / 2;  // elements
  for (uint64_t e = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; e < uint64_t(L) * per_layer;
       e += uint64_t(gridDim.x) * blockDim.x) {
    const int l = int(e / per_layer);
    uint32_t u = uint32_t(e % per_layer);
    const float* b = params + 5 * D + size_t(n) * D + size_t(l) * per;
    const float *wq = b + 2 * D, *wk = wq + D * D + D, *wv = wk + D * D + D, *wo = wv + D * D + D;
    const float* w1 = wo + D * D + D + 2 * D;
    const float* w2 = w1 + 4 * D * D + 4 * D;
    float v;
    uint32_t off;
    if (u < 3 * D * D) {  // q|k|v rows
      const uint32_t r = u / D, k = u % D;
      v = (r < D ? wq : r < 2 * D ? wk : wv)[(r % D) * D + k];
      off = tc::canon_off(r, k, D);
    } else if (u < 4 * D * D) {
      u -= 3 * D * D;
      const uint32_t r = u / D, k = u % D;
      v = wo[r * D + k];
      off = WQKV_BYTES + tc::canon_off(r, k, D);
    } else if (u < 8 * D * D) {  // W1 chunk c: rows 64c..64c+63 of W1 [4D][D]
      u -= 4 * D * D;
      const uint32_t c = u / (D * D), r = (u / D) % D, k = u % D;
      v = w1[(c * D + r) * D + k];
      off = WA_BYTES + c * D * D * 2 + tc::canon_off(r, k, D);
    } else {  // W2 chunk c: columns 64c..64c+63 of W2 [D][4D]
      u -= 8 * D * D;
      const uint32_t c = u / (D * D), r = (u / D) % D, k = u % D;
      v = w2[r * 4 * D + c * D + k];
      off = WA_BYTES + 4 * D * D * 2 + c * D * D * 2 + tc::canon_off(r, k, D);
    }
    *reinterpret_cast<uint16_t*>(img + size_t(l) * LAYER_BYTES + off) = __half_as_ushort(__float2half_rn(v));
  }
}

__device__ __forceinline__ bool wait_bar(uint32_t bar, uint32_t phase) {
  if (tc::mbar_wait(bar, phase, kWaitNs)) return true;
  tc::mbar_wait(bar, phase, kWaitNs);
  return false;
}

__device__ __forceinline__ void load_half(const Args& a, int layer, bool ffn, uint32_t dst, uint32_t bar) {
  const uint32_t bytes = ffn ? WF_BYTES : WA_BYTES;
  tc::mbar_arrive_expect_tx(bar, bytes);
  tc::bulk_g2s(dst, a.img + size_t(layer) * LAYER_BYTES + (ffn ? WA_BYTES : 0u), bytes, bar);
}

// LayerNorm of the thread's row (eps 1e-5, biased variance) -> fp16 row t of
// a canonical K-major [128][64] operand
__device__ __forceinline__ void ln_store(const float (&h)[D], const float* g, const float* b, unsigned char* sA,
                                         int t) {
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < D; ++c) s += h[c];
  const float mean = s * (1.0f / D);
  float q = 0.f;
#pragma unroll
  for (int c = 0; c < D; ++c) q = fmaf(h[c] - mean, h[c] - mean, q);
  const float rs = 1.0f / sqrtf(q * (1.0f / D) + 1e-5f);
#pragma unroll
  for (int c0 = 0; c0 < D; c0 += 8) {
    const float4 g0 = *reinterpret_cast<const float4*>(g + c0), g1 = *reinterpret_cast<const float4*>(g + c0 + 4);
    const float4 b0 = *reinterpret_cast<const float4*>(b + c0), b1 = *reinterpret_cast<const float4*>(b + c0 + 4);
    const float gg[8] = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w};
    const float bb[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
    uint32_t w[4];
#pragma unroll
    for (int e = 0; e < 4; ++e)
      w[e] = tc::pack_f16x2(fmaf((h[c0 + 2 * e] - mean) * rs, gg[2 * e], bb[2 * e]),
                             fmaf((h[c0 + 2 * e + 1] - mean) * rs, gg[2 * e + 1], bb[2 * e + 1]));
    *reinterpret_cast<uint4*>(sA + tc::canon_off(t, c0, D)) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

__device__ __forceinline__ void issue_gemm(uint32_t d_tmem, uint32_t a_addr, uint32_t b_addr, uint32_t idesc,
                                           uint32_t accumulate) {
#pragma unroll
  for (uint32_t ks = 0; ks < D / 16; ++ks)
    tc::mma_f16(d_tmem, tc::sdesc(a_addr + ks * 256u, 128u, D * 16u), tc::sdesc(b_addr + ks * 256u, 128u, D * 16u),
                 idesc, (accumulate || ks > 0) ? 1u : 0u);
}

__device__ __forceinline__ void f16x8_to_f32(const uint4 u, float (&f)[8]) {
  const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const float2 v = __half22float2(*reinterpret_cast<const __half2*>(&w[e]));
    f[2 * e] = v.x;
    f[2 * e + 1] = v.y;
  }
}

// Row geometry of one tile
struct Tile {
  bool live;   // the tile has rows
  int P, t0, S;
  uint64_t first;  // FULL: first sequence; SUFFIX: first index into perm
  uint64_t count;  // sequences available from `first`
};

template <int DH>
__global__ void __launch_bounds__(NT, 1) tf_tc_kernel(Args a) {
  constexpr int H = D / DH;
  constexpr uint32_t IDESC_QKV = tc::idesc_f16_f32(MT, 3 * D);
  constexpr uint32_t IDESC_64 = tc::idesc_f16_f32(MT, D);
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t bars[4];  // 0: q|k|v|o weights, 1: FFN weights, 2: MMA chain, 3: FFN2 chain
  __shared__ uint32_t s_tmem;
  __shared__ uint64_t s_tiles[ANQS_MAX_ORB + 1];
  const int wg = threadIdx.x / MT, t = threadIdx.x % MT;
  const int n = a.n, L = a.L;
  if (threadIdx.x == 0) {
    for (int i = 0; i < 4; ++i) tc::mbar_init(tc::smem_u32(&bars[i]), 1);
    tc::fence_mbar_init();
  }
  if (threadIdx.x < 32) {
    tc::tmem_alloc(tc::smem_u32(&s_tmem), NWG * TMEM_WG);
    tc::tmem_relinquish();
  }
  ANQS_PDL_WAIT();
  ANQS_PDL_TRIGGER();
  float* s_tp = reinterpret_cast<float*>(smem + OFF_TP);
  float* s_head = reinterpret_cast<float*>(smem + OFF_HEAD);
  float* s_lp = reinterpret_cast<float*>(smem + OFF_LP);
  {
    const size_t tail = 5 * size_t(D) + size_t(n) * D + size_t(L) * (12 * size_t(D) * D + 13 * D);
    for (int i = threadIdx.x; i < (5 + n) * D; i += NT) s_tp[i] = a.params[i];
    for (int i = threadIdx.x; i < 8 * D + 8; i += NT) s_head[i] = a.params[tail + 2 * D + i];
    // every block's LayerNorm parameters and biases, and the final LayerNorm's
    for (int l = 0; l < L; ++l) {
      const LayerP g = layer_p(a.params, n, l);
      float* d = s_lp + l * LP_FLOATS;
      for (int i = threadIdx.x; i < D; i += NT) {
        d[i] = g.ln1_g[i];
        d[D + i] = g.ln1_b[i];
        d[2 * D + i] = g.bq[i];
        d[3 * D + i] = g.bk[i];
        d[4 * D + i] = g.bv[i];
        d[5 * D + i] = g.bo[i];
        d[6 * D + i] = g.ln2_g[i];
        d[7 * D + i] = g.ln2_b[i];
        d[12 * D + i] = g.b2[i];
      }
      for (int i = threadIdx.x; i < 4 * D; i += NT) d[8 * D + i] = g.b1[i];
    }
    for (int i = threadIdx.x; i < 2 * D; i += NT) s_lp[kMaxL * LP_FLOATS + i] = a.params[tail + i];
  }
  // work: FULL one group; SUFFIX the groups j = 0..n-2 (P = n-1-j positions)
  uint64_t total = 0;
  if (threadIdx.x == 0) {
    if (a.mode == MODE_FULL) {
      const uint64_t S = MT / a.P, ns = a.n_seq.get();
      total = (ns + S - 1) / S;
      s_tiles[0] = 0;
      s_tiles[1] = total;
    } else {
      s_tiles[0] = 0;
      for (int j = 0; j < n - 1; ++j) {
        const uint64_t cnt = a.offsets[j + 1] - a.offsets[j], S = MT / (n - 1 - j);
        total += (cnt + S - 1) / S;
        s_tiles[j + 1] = total;
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const int n_groups = a.mode == MODE_FULL ? 1 : n - 1;
  total = s_tiles[n_groups];
  const uint32_t tmem = s_tmem + uint32_t(wg) * TMEM_WG;
  const uint32_t lane_base = uint32_t((t & ~31)) << 16;
  unsigned char* sA = smem + OFF_WG + wg * WG_BYTES;
  unsigned char* sKV = sA + A_BYTES;
  const uint32_t a_addr = tc::smem_u32(sA), kv_addr = tc::smem_u32(sKV);
  const uint32_t wa_addr = tc::smem_u32(smem + OFF_WA), wf_addr = tc::smem_u32(smem + OFF_WF);
  const uint32_t bar_wa = tc::smem_u32(&bars[0]), bar_wf = tc::smem_u32(&bars[1]);
  const uint32_t bar_m = tc::smem_u32(&bars[2]), bar_2 = tc::smem_u32(&bars[3]);
  uint32_t ph_wa = 0, ph_wf = 0, ph_m = 0, ph_2 = 0;
  bool pend_a = false, pend_f = false, ok = true;
  const uint64_t n_pairs = (total + 1) / 2;
  if (threadIdx.x == 0 && uint64_t(blockIdx.x) < n_pairs) {
    load_half(a, 0, false, wa_addr, bar_wa);
    load_half(a, 0, true, wf_addr, bar_wf);
  }
  pend_a = pend_f = uint64_t(blockIdx.x) < n_pairs;
  const float scale = 1.0f / sqrtf(float(DH));
  for (uint64_t pair = blockIdx.x; ok && pair < n_pairs; pair += gridDim.x) {
    const bool more = pair + gridDim.x < n_pairs;
    // ---- this warpgroup's tile and this thread's row ----
    const uint64_t tile = 2 * pair + wg;
    Tile tl{};
    if (tile < total) {
      int g = 0;
      while (s_tiles[g + 1] <= tile) ++g;
      const uint64_t k = tile - s_tiles[g];
      tl.live = true;
      if (a.mode == MODE_FULL) {
        tl.P = a.P;
        tl.t0 = 0;
        tl.S = MT / tl.P;
        tl.first = k * tl.S;
        tl.count = a.n_seq.get() - tl.first;
      } else {
        tl.P = n - 1 - g;
        tl.t0 = g + 1;
        tl.S = MT / tl.P;
        tl.first = a.offsets[g] + k * tl.S;
        tl.count = a.offsets[g + 1] - tl.first;
      }
    }
    const int s_loc = tl.live ? t / tl.P : 0;
    const bool valid = tl.live && s_loc < tl.S && uint64_t(s_loc) < tl.count;
    const int pos = valid ? tl.t0 + t % tl.P : 0;
    uint64_t x = 0, seq = 0, parent = 0;
    if (valid) {
      if (a.mode == MODE_FULL) {
        seq = tl.first + s_loc;
        x = a.x[seq];
      } else {
        seq = a.perm[tl.first + s_loc];  // row of the connected list
        x = a.xp[seq];
        parent = seq / a.K;
      }
    }
    const int row0 = s_loc * (valid ? tl.P : 0);  // tile row of this sequence's first computed position
    float h[D];
    {
      const int token = pos == 0 ? 4 : int((x >> (2 * (pos - 1))) & 3ull);
#pragma unroll
      for (int c = 0; c < D; ++c) h[c] = s_tp[token * D + c] + s_tp[(5 + pos) * D + c];
    }
    for (int l = 0; ok && l < L; ++l) {
      LayerP lp;  // this block's small parameters, staged in shared memory
      {
        const float* d = s_lp + l * LP_FLOATS;
        lp.ln1_g = d;
        lp.ln1_b = d + D;
        lp.bq = d + 2 * D;
        lp.bk = d + 3 * D;
        lp.bv = d + 4 * D;
        lp.bo = d + 5 * D;
        lp.ln2_g = d + 6 * D;
        lp.ln2_b = d + 7 * D;
        lp.b1 = d + 8 * D;
        lp.b2 = d + 12 * D;
      }
      ln_store(h, lp.ln1_g, lp.ln1_b, sA, t);
      tc::fence_async_smem();
      tc::fence_before_sync();
      if (pend_a) {
        ok = __syncthreads_and(wait_bar(bar_wa, ph_wa));
        ph_wa ^= 1;
        pend_a = false;
      } else {
        __syncthreads();
      }
      if (!ok) break;
      // q|k|v
      if (threadIdx.x == 0) {
        tc::fence_after_sync();
        for (int w = 0; w < NWG; ++w)
          issue_gemm(s_tmem + uint32_t(w) * TMEM_WG, tc::smem_u32(smem + OFF_WG + w * WG_BYTES), wa_addr, IDESC_QKV, 0);
        tc::mma_commit(bar_m);
      }
      ok = __syncthreads_and(wait_bar(bar_m, ph_m));
      ph_m ^= 1;
      if (!ok) break;
      tc::fence_after_sync();
      // k, v of this row (+ bias) -> shared memory (and the parent cache)
#pragma unroll 1
      for (int c0 = D; c0 < 3 * D; c0 += 32) {
        float v[32];
        tc::tmem_ld32(tmem + lane_base + uint32_t(c0), v);
        const float* bias = c0 < 2 * D ? lp.bk + (c0 - D) : lp.bv + (c0 - 2 * D);
        uint32_t w[16];
#pragma unroll
        for (int i = 0; i < 32; i += 2) w[i / 2] = tc::pack_f16x2(v[i] + bias[i], v[i + 1] + bias[i + 1]);
        uint4* dst = reinterpret_cast<uint4*>(sKV + t * KV_STRIDE + (c0 - D) * 2);
#pragma unroll
        for (int q = 0; q < 4; ++q) dst[q] = make_uint4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
        if (valid && a.kv_out) {
          uint4* g = reinterpret_cast<uint4*>(a.kv_out + ((seq * L + l) * n + pos) * (2 * D) + (c0 - D));
#pragma unroll
          for (int q = 0; q < 4; ++q) g[q] = make_uint4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
        }
      }
      __syncthreads();
      // causal attention of this row over the keys 0..pos
      const __half* pkv = a.kv_in ? a.kv_in + (parent * L + l) * size_t(n) * (2 * D) : nullptr;
#pragma unroll 1
      for (int hd = 0; hd < H; ++hd) {
        float q[DH];
        if constexpr (DH == 16) {
          tc::tmem_ld16(tmem + lane_base + uint32_t(hd * DH), q);
        } else {
          tc::tmem_ld32(tmem + lane_base + uint32_t(hd * DH), q);
        }
#pragma unroll
        for (int e = 0; e < DH; ++e) q[e] = (q[e] + lp.bq[hd * DH + e]) * scale;
        float m = -INFINITY, lsum = 0.f, acc[DH];
#pragma unroll
        for (int e = 0; e < DH; ++e) acc[e] = 0.f;
        const int upto = valid ? pos : -1;
        // one key: score, online-softmax update of (m, lsum, acc)
        auto step = [&](const uint4 (&kw)[DH / 8], const uint4 (&vw)[DH / 8]) {
          float s0 = 0.f, s1 = 0.f;
#pragma unroll
          for (int e8 = 0; e8 < DH; e8 += 8) {
            float kf[8];
            f16x8_to_f32(kw[e8 / 8], kf);
#pragma unroll
            for (int e = 0; e < 8; e += 2) tc::fma_f32x2(q[e8 + e], q[e8 + e + 1], kf[e], kf[e + 1], s0, s1, s0, s1);
          }
          const float sc = s0 + s1;
          const float mn = fmaxf(m, sc);
          const float corr = __expf(m - mn), p = __expf(sc - mn);
          lsum = fmaf(lsum, corr, p);
#pragma unroll
          for (int e8 = 0; e8 < DH; e8 += 8) {
            float vf[8];
            f16x8_to_f32(vw[e8 / 8], vf);
#pragma unroll
            for (int e = 0; e < 8; e += 2) {
              float p0, p1;
              tc::fma_f32x2(p, p, vf[e], vf[e + 1], 0.f, 0.f, p0, p1);
              tc::fma_f32x2(acc[e8 + e], acc[e8 + e + 1], corr, corr, p0, p1, acc[e8 + e], acc[e8 + e + 1]);
            }
          }
          m = mn;
        };
        // keys of positions < t0 from the parent cache (global memory; the
        // next key's words are loaded before this key's arithmetic), then
        // the tile's own keys from shared memory
        const int n_par = min(upto + 1, tl.t0);
        if (n_par > 0) {
          const uint4* gp = reinterpret_cast<const uint4*>(pkv);
          uint4 kw[DH / 8], vw[DH / 8];
#pragma unroll
          for (int e = 0; e < DH / 8; ++e) {
            kw[e] = __ldg(gp + (hd * DH) / 8 + e);
            vw[e] = __ldg(gp + (D + hd * DH) / 8 + e);
          }
#pragma unroll 1
          for (int u = 0; u < n_par; ++u) {
            uint4 kn[DH / 8], vn[DH / 8];
            const uint4* np = gp + size_t(u + 1 < n_par ? u + 1 : u) * (2 * D / 8);
#pragma unroll
            for (int e = 0; e < DH / 8; ++e) {
              kn[e] = __ldg(np + (hd * DH) / 8 + e);
              vn[e] = __ldg(np + (D + hd * DH) / 8 + e);
            }
            step(kw, vw);
#pragma unroll
            for (int e = 0; e < DH / 8; ++e) kw[e] = kn[e], vw[e] = vn[e];
          }
        }
#pragma unroll 1
        for (int u = tl.t0; u <= upto; ++u) {
          const uint4* sp = reinterpret_cast<const uint4*>(sKV + (row0 + u - tl.t0) * KV_STRIDE);
          uint4 kw[DH / 8], vw[DH / 8];
#pragma unroll
          for (int e = 0; e < DH / 8; ++e) {
            kw[e] = sp[(hd * DH) / 8 + e];
            vw[e] = sp[(D + hd * DH) / 8 + e];
          }
          step(kw, vw);
        }
        const float inv = valid ? 1.0f / lsum : 0.f;
#pragma unroll
        for (int e8 = 0; e8 < DH; e8 += 8) {
          uint32_t w[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) w[e] = tc::pack_f16x2(acc[e8 + 2 * e] * inv, acc[e8 + 2 * e + 1] * inv);
          *reinterpret_cast<uint4*>(sA + tc::canon_off(t, hd * DH + e8, D)) = make_uint4(w[0], w[1], w[2], w[3]);
        }
      }
      tc::fence_async_smem();
      tc::fence_before_sync();
      __syncthreads();
      // output projection
      if (threadIdx.x == 0) {
        tc::fence_after_sync();
        for (int w = 0; w < NWG; ++w)
          issue_gemm(s_tmem + uint32_t(w) * TMEM_WG, tc::smem_u32(smem + OFF_WG + w * WG_BYTES), wa_addr + WQKV_BYTES,
                     IDESC_64, 0);
        tc::mma_commit(bar_m);
      }
      ok = __syncthreads_and(wait_bar(bar_m, ph_m));
      ph_m ^= 1;
      if (!ok) break;
      tc::fence_after_sync();
      const bool next_exists = (l + 1 < L) || more;
      if (threadIdx.x == 0 && next_exists) load_half(a, (l + 1) % L, false, wa_addr, bar_wa);
      pend_a = next_exists;
#pragma unroll
      for (int c0 = 0; c0 < D; c0 += 32) {
        float v[32];
        tc::tmem_ld32(tmem + lane_base + uint32_t(c0), v);
#pragma unroll
        for (int i = 0; i < 32; ++i) h[c0 + i] += v[i] + lp.bo[c0 + i];
      }
      ln_store(h, lp.ln2_g, lp.ln2_b, sA, t);
      tc::fence_async_smem();
      tc::fence_before_sync();
      if (pend_f) {
        ok = __syncthreads_and(wait_bar(bar_wf, ph_wf));
        ph_wf ^= 1;
        pend_f = false;
      } else {
        __syncthreads();
      }
      if (!ok) break;
      // FFN in 4 chunks
      if (threadIdx.x == 0) {
        tc::fence_after_sync();
        for (int w = 0; w < NWG; ++w)
          issue_gemm(s_tmem + uint32_t(w) * TMEM_WG, tc::smem_u32(smem + OFF_WG + w * WG_BYTES), wf_addr, IDESC_64, 0);
        tc::mma_commit(bar_m);
      }
      ok = __syncthreads_and(wait_bar(bar_m, ph_m));
      ph_m ^= 1;
      if (!ok) break;
      tc::fence_after_sync();
#pragma unroll 1
      for (int c = 0; c < 4; ++c) {
        if (threadIdx.x == 0 && c + 1 < 4) {
          for (int w = 0; w < NWG; ++w)
            issue_gemm(s_tmem + uint32_t(w) * TMEM_WG + uint32_t(((c + 1) & 1) * D),
                       tc::smem_u32(smem + OFF_WG + w * WG_BYTES), wf_addr + uint32_t(c + 1) * D * D * 2, IDESC_64, 0);
          tc::mma_commit(bar_m);
        }
        if (c >= 1) {
          ok = __syncthreads_and(wait_bar(bar_2, ph_2));
          ph_2 ^= 1;
          if (!ok) break;
        }
        unsigned char* sH = sKV + (c & 1) * A_BYTES;
#pragma unroll
        for (int c0 = 0; c0 < D; c0 += 32) {
          float v[32];
          tc::tmem_ld32(tmem + lane_base + uint32_t((c & 1) * D + c0), v);
#pragma unroll
          for (int q8 = 0; q8 < 32; q8 += 8) {
            uint32_t w[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const int i = q8 + 2 * e;
              w[e] = tc::pack_f16x2(fmaxf(v[i] + lp.b1[c * D + c0 + i], 0.f),
                                     fmaxf(v[i + 1] + lp.b1[c * D + c0 + i + 1], 0.f));
            }
            *reinterpret_cast<uint4*>(sH + tc::canon_off(t, c0 + q8, D)) = make_uint4(w[0], w[1], w[2], w[3]);
          }
        }
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        if (threadIdx.x == 0) {
          tc::fence_after_sync();
          for (int w = 0; w < NWG; ++w)
            issue_gemm(s_tmem + uint32_t(w) * TMEM_WG + 3 * D,
                       tc::smem_u32(smem + OFF_WG + w * WG_BYTES + A_BYTES + (c & 1) * A_BYTES),
                       wf_addr + 4 * D * D * 2 + uint32_t(c) * D * D * 2, IDESC_64, c > 0 ? 1u : 0u);
          tc::mma_commit(bar_2);
        }
        if (c + 1 < 4) {
          ok = __syncthreads_and(wait_bar(bar_m, ph_m));
          ph_m ^= 1;
          if (!ok) break;
          tc::fence_after_sync();
        }
      }
      if (!ok) break;
      ok = __syncthreads_and(wait_bar(bar_2, ph_2));
      ph_2 ^= 1;
      if (!ok) break;
      tc::fence_after_sync();
      if (threadIdx.x == 0 && next_exists) load_half(a, (l + 1) % L, true, wf_addr, bar_wf);
      pend_f = next_exists;
#pragma unroll
      for (int c0 = 0; c0 < D; c0 += 32) {
        float v[32];
        tc::tmem_ld32(tmem + lane_base + uint32_t(3 * D + c0), v);
#pragma unroll
        for (int i = 0; i < 32; ++i) h[c0 + i] += v[i] + lp.b2[c0 + i];
      }
    }
    if (!ok) break;
    // final LayerNorm and head
    {
      const float* g = s_lp + kMaxL * LP_FLOATS;
      const float* b = g + D;
      float s = 0.f;
#pragma unroll
      for (int c = 0; c < D; ++c) s += h[c];
      const float mean = s * (1.0f / D);
      float q = 0.f;
#pragma unroll
      for (int c = 0; c < D; ++c) q = fmaf(h[c] - mean, h[c] - mean, q);
      const float rs = 1.0f / sqrtf(q * (1.0f / D) + 1e-5f);
      float out[8];
#pragma unroll
      for (int o = 0; o < 8; ++o) out[o] = s_head[8 * D + o];
#pragma unroll
      for (int c = 0; c < D; ++c) {
        const float y = fmaf((h[c] - mean) * rs, g[c], b[c]);
#pragma unroll
        for (int o = 0; o < 8; ++o) out[o] = fmaf(y, s_head[o * D + c], out[o]);
      }
      if (valid) {
        if (a.mode == MODE_FULL) {
          if (!a.last_only || pos == a.P - 1) {
            float4* dst = reinterpret_cast<float4*>(a.raw + (a.last_only ? seq : seq * a.P + pos) * 8);
            dst[0] = make_float4(out[0], out[1], out[2], out[3]);
            dst[1] = make_float4(out[4], out[5], out[6], out[7]);
          }
        } else {
          const uint64_t pm = (1ull << (2 * pos)) - 1ull;
          const unsigned pmk = slot_mask(a.hv, pos, __popcll(x & pm & 0x5555555555555555ull),
                                         __popcll(x & pm & 0xAAAAAAAAAAAAAAAAull), x);
          const unsigned mk = norm_mask(a.hv, pos, pmk);
          float mx = -INFINITY;
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if ((mk >> u) & 1u) mx = fmaxf(mx, out[u]);
          float sum = 0.f;
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if ((mk >> u) & 1u) sum += __expf(out[u] - mx);
          const int v = int((x >> (2 * pos)) & 3ull);
          const float ov = (v == 0) ? out[0] : (v == 1) ? out[1] : (v == 2) ? out[2] : out[3];
          const float pv = (v == 0) ? out[4] : (v == 1) ? out[5] : (v == 2) ? out[6] : out[7];
          const float lse = mx + __logf(sum);
          // the row's term to shared memory (the k|v region is free now); the
          // sequence's first row adds its positions' terms below
          reinterpret_cast<float2*>(sKV)[t] = make_float2(((pmk >> v) & 1u) ? 0.5f * (ov - lse) : -INFINITY, pv);
        }
      }
    }
    if (a.mode == MODE_SUFFIX) {
      // one sum per connected determinant, over its positions in order: T[x']
      __syncthreads();
      if (valid && pos == tl.t0) {
        const float2* tr = reinterpret_cast<const float2*>(sKV) + t;
        float sl = 0.f, sp = 0.f;
        for (int i = 0; i < tl.P; ++i) {
          sl += tr[i].x;
          sp += tr[i].y;
        }
        a.T[seq] = make_float2(sl, sp);
      }
    }
    __syncthreads();  // shared k|v and hidden buffers are rewritten by the next tile
  }
  // weights fetched for a tile that never came (or abandoned after a time-out)
  if (pend_a && !__syncthreads_and(wait_bar(bar_wa, ph_wa))) ok = false;
  if (pend_f && !__syncthreads_and(wait_bar(bar_wf, ph_wf))) ok = false;
  if (!ok && threadIdx.x == 0) atomicExch(a.status, 1);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (threadIdx.x < 32) tc::tmem_dealloc(s_tmem, NWG * TMEM_WG);
}

int g_sms = 0;

int sms() {
  if (!g_sms) {
    int dev = 0;
    ANQS_CUDA(cudaGetDevice(&dev));
    ANQS_CUDA(cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev));
  }
  return g_sms;
}

int launch(const anqs_model* M, Args a, uint64_t max_tiles, int prof, cudaStream_t s) {
  a.img = static_cast<const unsigned char*>(M->packed);
  a.params = M->params;
  a.n = M->d.n_orb;
  a.L = M->d.n_layers;
  a.status = reinterpret_cast<int*>(static_cast<unsigned char*>(M->packed) + size_t(a.L) * LAYER_BYTES);
  const uint64_t pairs = (max_tiles + 1) / 2;
  const unsigned grid = unsigned(std::max<uint64_t>(1, std::min<uint64_t>(pairs, uint64_t(sms()))));
  const int dh = D / M->d.n_heads;
  ProfScope ps(prof, s);
  if (dh == 16) {
    ANQS_CUDA(cudaFuncSetAttribute(tf_tc_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(SMEM_BYTES)));
    ANQS_CUDA_LAUNCH("tf_tc_kernel", launch_k(tf_tc_kernel<16>, dim3(grid), dim3(NT), SMEM_BYTES, s, a));
  } else {
    ANQS_CUDA(cudaFuncSetAttribute(tf_tc_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(SMEM_BYTES)));
    ANQS_CUDA_LAUNCH("tf_tc_kernel", launch_k(tf_tc_kernel<32>, dim3(grid), dim3(NT), SMEM_BYTES, s, a));
  }
  return ANQS_OK;
}

Args full_args(const uint64_t* x, Count n_seq, int P, int last_only, float* raw, __half* kv_out,
               const HamView& hv) {
  Args a{};
  a.mode = MODE_FULL;
  a.x = x;
  a.n_seq = n_seq;
  a.P = P;
  a.last_only = last_only;
  a.raw = raw;
  a.kv_out = kv_out;
  a.hv = hv;
  return a;
}

struct TfElocWs {
  uint64_t* xp;
  double* hv;
  uint8_t* js;
  double* hd;
  float *la_x, *ph_x, *raw, *cache;
  float2* T;
  uint32_t *perm, *hist, *cursor, *offsets, *ticket;
  __half* kv;
};

size_t plan(const anqs_model* M, const anqs_ham* H, uint64_t n_x, Arena& A, TfElocWs& w) {
  const uint64_t n = H->v.n, m = n_x * H->v.K;
  w.xp = A.take<uint64_t>(m);
  w.hv = A.take<double>(m);
  w.js = A.take<uint8_t>(m);
  w.hd = A.take<double>(n_x);
  w.la_x = A.take<float>(n_x);
  w.ph_x = A.take<float>(n_x);
  w.raw = A.take<float>(n_x * n * 8);
  w.cache = A.take<float>(n_x * n * TC_CACHE_F);
  w.T = A.take<float2>(m);  // one sum of the suffix positions' terms per connected determinant
  w.perm = A.take<uint32_t>(m);
  w.cursor = A.take<uint32_t>(ANQS_MAX_ORB);
  w.offsets = A.take<uint32_t>(ANQS_MAX_ORB + 1);
  w.hist = A.take<uint32_t>(TC_CTL_WORDS);
  w.ticket = w.hist + TC_CTL_STATS_TICKET;
  w.kv = A.take<__half>(n_x * uint64_t(M->d.n_layers) * n * 2 * uint64_t(M->d.d_model));
  return A.off;
}

}  // namespace

int tf_tc_pack_alloc(anqs_model* M) {
  if (M->d.d_model != D && M->d.d_model != 128)
    return set_error(ANQS_ERR_UNSUPPORTED, "BF16 transformer form supports d_model 64 or 128");
  if (M->d.d_model / M->d.n_heads != 16 && M->d.d_model / M->d.n_heads != 32)
    return set_error(ANQS_ERR_UNSUPPORTED, "BF16 transformer form supports head width 16 or 32");
  if (M->d.d_model == D && M->d.n_layers > kMaxL)
    return set_error(ANQS_ERR_UNSUPPORTED, "BF16 transformer form at d_model 64 supports up to %d blocks", kMaxL);
  M->packed_bytes = M->d.d_model == 128 ? tf128_packed_bytes(M) : size_t(M->d.n_layers) * LAYER_BYTES + 256;
  ANQS_CUDA(cudaMalloc(&M->packed, M->packed_bytes));
  ANQS_CUDA(cudaMemset(M->packed, 0, M->packed_bytes));
  M->tc_raw_rows = 32768;
  ANQS_CUDA(cudaMalloc(&M->tc_raw, M->tc_raw_rows * M->d.n_orb * 8 * sizeof(float)));
  return ANQS_OK;
}

int tf_tc_pack(anqs_model* M, cudaStream_t s) {
  if (M->d.d_model == 128) return tf128_pack(M, s);
  ANQS_CUDA_LAUNCH("tf_pack_kernel", launch_k(tf_pack_kernel, dim3(152), dim3(256), 0, s, M->params, M->d.n_orb,
                                              M->d.n_layers, static_cast<unsigned char*>(M->packed)));
  return ANQS_OK;
}

int tf_tc_status(const anqs_model* M, int* status) {
  int v = 0;
  const size_t off = M->d.d_model == 128 ? size_t(tf128_status_offset(M)) : size_t(M->d.n_layers) * LAYER_BYTES;
  ANQS_CUDA(cudaMemcpy(&v, static_cast<const unsigned char*>(M->packed) + off, sizeof(int), cudaMemcpyDeviceToHost));
  *status = v;
  return ANQS_OK;
}

int launch_tf_tc_logpsi(const anqs_model* M, const HamView& hv, const uint64_t* x, uint64_t n_x, float* la,
                        float* ph, cudaStream_t s) {
  const int n = M->d.n_orb;
  for (uint64_t off = 0; off < n_x; off += M->tc_raw_rows) {
    const uint64_t k = std::min<uint64_t>(M->tc_raw_rows, n_x - off);
    if (M->d.d_model == 128) {
      ANQS_TRY(launch_tf128_full(M, hv, x + off, host_count(k), n, 0, M->tc_raw, nullptr, PROF_TF_TC_PARENT, s));
    } else {
      Args a = full_args(x + off, host_count(k), n, 0, M->tc_raw, nullptr, hv);
      ANQS_TRY(launch(M, a, (k + MT / n - 1) / (MT / n), PROF_TF_TC_PARENT, s));
    }
    ProfScope ps(PROF_TC_FINALIZE, s);
    ANQS_TRY(launch_tc_finalize(hv, x + off, host_count(k), M->tc_raw, la + off, ph + off, nullptr, s));
  }
  return ANQS_OK;
}

int launch_tf_tc_slot_logits(const anqs_model* M, int p, const uint64_t* pre, const uint64_t* n_dev,
                             uint64_t max_rows, float* out8, cudaStream_t s) {
  HamView hv{};
  if (M->d.d_model == 128)
    return launch_tf128_full(M, hv, pre, Count{max_rows, n_dev, 1}, p + 1, 1, out8, nullptr, PROF_TF_TC_SLOT, s);
  Args a = full_args(pre, Count{max_rows, n_dev, 1}, p + 1, 1, out8, nullptr, hv);
  const uint64_t S = MT / (p + 1);
  return launch(M, a, (max_rows + S - 1) / S, PROF_TF_TC_SLOT, s);
}

size_t tf_tc_eloc_workspace(const anqs_model* M, const anqs_ham* H, uint64_t n_x) {
  Arena A(nullptr, 0);
  TfElocWs w;
  return plan(M, H, n_x, A, w);
}

int run_eloc_tf_tc(const anqs_model* M, const anqs_ham* H, const uint64_t* x, Count n_x, double* ere, double* eim,
                   const uint64_t* counts, double* stats, void* ws, size_t ws_bytes, cudaStream_t s) {
  Arena A(ws, ws_bytes);
  TfElocWs w;
  plan(M, H, n_x.n, A, w);
  if (!A.fits()) return set_error(ANQS_ERR_CAPACITY, "workspace needs %zu bytes", A.off);
  const int n = H->v.n;
  const uint64_t K = H->v.K;
  const Count mc = scaled(n_x, K);
  if (mc.n > 0xffffffffull) return set_error(ANQS_ERR_UNSUPPORTED, "more than 2^32 connected determinants per call");
  ANQS_TRY(launch_connected(H->v, x, n_x, w.xp, w.hv, w.js, w.hd, s, w.hist));
  {
    if (M->d.d_model == 128) {
      ANQS_TRY(launch_tf128_full(M, H->v, x, n_x, n, 0, w.raw, w.kv, PROF_TF_TC_PARENT, s));
    } else {
      Args a = full_args(x, n_x, n, 0, w.raw, w.kv, H->v);
      ANQS_TRY(launch(M, a, (n_x.n + MT / n - 1) / (MT / n), PROF_TF_TC_PARENT, s));
    }
    ProfScope ps(PROF_TC_FINALIZE, s);
    ANQS_TRY(launch_tc_finalize(H->v, x, n_x, w.raw, w.la_x, w.ph_x, w.cache, s));
  }
  {
    ProfScope ps(PROF_TC_SORT, s);
    ANQS_TRY(launch_js_sort(w.js, mc, n, w.hist, w.cursor, w.offsets, w.perm, s));
  }
  if (M->d.d_model == 128) {
    ANQS_TRY(launch_tf128_suffix(M, H->v, w.xp, w.perm, w.offsets, uint32_t(K), w.kv, w.T, mc.n, PROF_TF_TC_SUFFIX,
                                 s));
  } else {
    Args a{};
    a.mode = MODE_SUFFIX;
    a.hv = H->v;
    a.xp = w.xp;
    a.perm = w.perm;
    a.offsets = w.offsets;
    a.K = uint32_t(K);
    a.kv_in = w.kv;
    a.T = w.T;
    uint64_t tiles = 0;  // upper bound over the groups
    for (int j = 0; j + 1 < n; ++j) tiles += mc.n / uint64_t(MT / (n - 1 - j)) + 1;
    ANQS_TRY(launch(M, a, tiles, PROF_TF_TC_SUFFIX, s));
  }
  {
    ProfScope ps(PROF_TC_ELOC, s);
    ANQS_TRY(launch_eloc_assemble(n, uint32_t(K), n_x, w.xp, w.js, w.cache, w.T, w.hv, w.hd, w.la_x, w.ph_x, ere,
                                  eim, StatsOut{counts, stats, w.ticket}, s, true));
  }
  return ANQS_OK;
}

}  // namespace anqs
