// 16-bit tensor-core form of the causal-transformer ansatz at d_model = 128
// (tcgen05 MMAs with TMEM accumulators), with reuse of the parent
// determinant's keys and values for its connected determinants.  GEMM
// operands and stored keys and values are fp16 (see tf_tc.cu for why).
//
// The network is the one of the FP32 form (decoder-only, pre-LayerNorm, eps
// 1e-5, causal multi-head attention, ReLU FFN of width 4d, head d -> 8 whose
// outputs enter the masked slot conditional of Appendix B.1 f3 with MU
// masking, Sec. III.C); Eq. anqs_def makes log psi the sum of the slot terms.
//
// A CTA owns one tile of 128 rows (one row = one (sequence, position) pair =
// one TMEM lane) and runs two compute warpgroups, each holding half of the
// model dimensions of every row: its 64 residual-stream values in
// registers, its 64 columns of every epilogue, its half of the attention
// heads.  LayerNorm statistics and the head's partial sums cross between the
// halves through shared memory.  A layer's weights (384 KB in fp16) do not
// fit in shared memory: they are cut into twelve [128 out][128 in] chunks
// (q, k, v, o, the four W1 row blocks and the four W2 column blocks, stored
// in the order the MMAs consume them) that stream through a ring of three
// 32 KB stages with bulk copies, one mbarrier pair per stage (full: bytes
// arrived; empty: the MMAs reading it are done).  The thread that issues the
// MMAs also requests the chunks: whenever a stage is free it requests the
// next chunk without waiting, and it blocks only when the chunk its next
// GEMM needs has not been requested yet.
//
// Tensor memory (512 columns): q | k | v accumulators at 0 | 128 | 256 (the
// output projection reuses q's columns), the two FFN hidden-chunk
// accumulators at 128 and 256 (after k and v are consumed), the FFN output
// accumulator at 384.  Per block:
//   LN1 -> A (fp16)        MMA q, k, v = A W^T
//   k, v (+ bias) -> shared memory and the parent cache; causal attention of
//   each row over keys 0..t on the CUDA cores (online softmax, f32) -> A
//   MMA o = A Wo^T         h += o + bo;  LN2 -> A
//   FFN chunk c: MMA f1_c = A W1_c^T (issued one chunk ahead), ReLU -> H_c
//   (fp16, two buffers in the key/value region), MMA acc2 += H_c W2_c^T
//   h += acc2 + b2
// then LNf and the f32 head.
//
// Modes (as for d_model 64)
//   FULL    sequences x[s], positions 0..P-1: the 8 raw outputs of every
//           position (or of the last one), optionally keys and values of
//           every position and block (the parent cache).
//   SUFFIX  connected determinants x' grouped by first differing slot j:
//           positions j+1..n-1 only, keys and values of positions <= j from
//           the parent cache; writes the masked slot terms T[x'][t].
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "tc_ptx.cuh"

namespace anqs {


namespace {

constexpr int D = 128;
constexpr int MT = 128;
constexpr int HD = D / 2;                       // model dimensions per warpgroup
constexpr int NT = 256;                         // two warpgroups
constexpr uint32_t CHUNK = D * D * 2;           // one weight chunk, [128][128] fp16 canonical K-major
constexpr int NCH = 12;                         // chunks per layer, in consumption order
constexpr uint32_t LAYER_BYTES = NCH * CHUNK;
constexpr int NS = 3;                           // ring stages
constexpr uint32_t A_BYTES = MT * D * 2;        // one A operand tile (K = 128)
constexpr uint32_t KV_STRIDE = 2 * D * 2 + 16;  // bytes per row of k|v (padded)
constexpr uint32_t KV_BYTES = MT * KV_STRIDE;   // also holds the two FFN hidden chunks
constexpr uint32_t OFF_W = 0;
constexpr uint32_t OFF_A = NS * CHUNK;
constexpr uint32_t OFF_KV = OFF_A + A_BYTES;
constexpr uint32_t OFF_HEAD = OFF_KV + KV_BYTES;              // head [8][D] f32 + bias [8]
constexpr uint32_t OFF_RED = OFF_HEAD + (8 * D + 8) * 4;      // exchange [2 slots][2 halves][128] f32
constexpr uint32_t OFF_HX = OFF_RED + 2 * 2 * MT * 4;         // head partials of half 1 [128][8] f32
constexpr uint32_t OFF_LP = OFF_HX + MT * 8 * 4;              // the layer's LayerNorm parameters and biases
constexpr uint32_t LP_FLOATS = 14 * D;                         // ln1 g,b | bq bk bv bo | ln2 g,b | b1 (4D) | b2
constexpr uint32_t SMEM_BYTES = OFF_LP + LP_FLOATS * 4;
constexpr uint64_t kWaitNs = 2000000000ull;
constexpr int MODE_FULL = 0, MODE_SUFFIX = 1;
// chunk indices within a layer
enum { C_Q = 0, C_K, C_V, C_O, C_W1_0, C_W1_1, C_W2_0, C_W1_2, C_W2_1, C_W1_3, C_W2_2, C_W2_3 };
static_assert(2 * A_BYTES <= KV_BYTES, "hidden chunks live in the k|v region");
static_assert(SMEM_BYTES <= 227 * 1024, "shared memory");

struct Args {
  const unsigned char* img;  // packed fp16 chunks, LAYER_BYTES per layer
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

__host__ __device__ inline size_t layer_floats() { return 12 * size_t(D) * D + 13 * D; }

// The small parameters of block l (LayerNorms and biases, 14 D floats) are
// copied to shared memory at the start of the block; lp points there.
__device__ __forceinline__ const float* layer_small(const float* params, int n, int l, int part) {
  // part: 0 ln1 g, 1 ln1 b, 2 bq, 3 bk, 4 bv, 5 bo, 6 ln2 g, 7 ln2 b, 8 b1 (4 D), 9 b2
  const float* b = params + 5 * D + size_t(n) * D + size_t(l) * layer_floats();
  switch (part) {
    case 0: return b;
    case 1: return b + D;
    case 2: return b + 2 * D + D * D;
    case 3: return b + 2 * D + 2 * D * D + D;
    case 4: return b + 2 * D + 3 * D * D + 2 * D;
    case 5: return b + 2 * D + 4 * D * D + 3 * D;
    case 6: return b + 2 * D + 4 * D * D + 4 * D;
    case 7: return b + 2 * D + 4 * D * D + 5 * D;
    case 8: return b + 2 * D + 4 * D * D + 6 * D + 4 * D * D;
    default: return b + 2 * D + 4 * D * D + 6 * D + 4 * D * D + 4 * D + 4 * D * D;
  }
}

__device__ __forceinline__ void stage_layer(const float* params, int n, int l, float* s_lp) {
  for (int i = threadIdx.x; i < int(LP_FLOATS); i += blockDim.x) {
    const int r = i / D;
    const int part = r < 8 ? r : (r < 12 ? 8 : 9);
    const int off = r < 8 ? i % D : (r < 12 ? i - 8 * D : i - 12 * D);
    s_lp[i] = layer_small(params, n, l, part)[off];
  }
}

__device__ __forceinline__ LayerP staged_p(const float* s_lp) {
  LayerP P;
  P.ln1_g = s_lp;
  P.ln1_b = s_lp + D;
  P.bq = s_lp + 2 * D;
  P.bk = s_lp + 3 * D;
  P.bv = s_lp + 4 * D;
  P.bo = s_lp + 5 * D;
  P.ln2_g = s_lp + 6 * D;
  P.ln2_b = s_lp + 7 * D;
  P.b1 = s_lp + 8 * D;
  P.b2 = s_lp + 12 * D;
  return P;
}

// ---- packing: f32 parameters -> per-layer fp16 chunks --------------------------
__global__ void tf128_pack_kernel(const float* __restrict__ params, int n, int L, unsigned char* __restrict__ img) {
  // no early trigger: a later kernel's prologue may read the packed images
  // before its own dependency wait, so the images are complete before any
  // dependent launch starts
  ANQS_PDL_WAIT();
  const uint32_t per_layer = LAYER_BYTES / 2;  // elements
  for (uint64_t e = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; e < uint64_t(L) * per_layer;
       e += uint64_t(gridDim.x) * blockDim.x) {
    const int l = int(e / per_layer);
    const uint32_t u = uint32_t(e % per_layer);
    const int ch = int(u / (D * D));
    const uint32_t r = (u / D) % D, k = u % D;
    const float* b = params + 5 * D + size_t(n) * D + size_t(l) * layer_floats();
    const float *wq = b + 2 * D, *wk = wq + D * D + D, *wv = wk + D * D + D, *wo = wv + D * D + D;
    const float* w1 = wo + D * D + D + 2 * D;  // [4D][D]
    const float* w2 = w1 + 4 * D * D + 4 * D;  // [D][4D]
    float v;
    switch (ch) {
      case C_Q: v = wq[r * D + k]; break;
      case C_K: v = wk[r * D + k]; break;
      case C_V: v = wv[r * D + k]; break;
      case C_O: v = wo[r * D + k]; break;
      case C_W1_0: case C_W1_1: case C_W1_2: case C_W1_3: {
        const int c = ch == C_W1_0 ? 0 : ch == C_W1_1 ? 1 : ch == C_W1_2 ? 2 : 3;
        v = w1[(size_t(c) * D + r) * D + k];  // rows 128c..128c+127 of W1
        break;
      }
      default: {
        const int c = ch == C_W2_0 ? 0 : ch == C_W2_1 ? 1 : ch == C_W2_2 ? 2 : 3;
        v = w2[size_t(r) * 4 * D + size_t(c) * D + k];  // columns 128c..128c+127 of W2
        break;
      }
    }
    *reinterpret_cast<uint16_t*>(img + size_t(l) * LAYER_BYTES + size_t(ch) * CHUNK + tc::canon_off(r, k, D)) =
        __half_as_ushort(__float2half_rn(v));
  }
}

__device__ __forceinline__ bool wait_bar(uint32_t bar, uint32_t phase) {
  if (tc::mbar_wait(bar, phase, kWaitNs)) return true;
  tc::mbar_wait(bar, phase, kWaitNs);
  return false;
}

// barrier over the CTA's 256 threads (named barrier 1), and the same with an
// AND of a flag over the threads
__device__ __forceinline__ void csync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }
__device__ __forceinline__ bool call(bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred q, p;\n\t"
      "setp.ne.u32 q, %1, 0;\n\t"
      "bar.red.and.pred p, 1, 256, q;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(r)
      : "r"(uint32_t(v))
      : "memory");
  return r != 0;
}

// Sum of a per-row value over the two halves (shared-memory exchange in one
// of two alternating slots, so a slot is rewritten only after a later
// barrier).
struct Xch {
  float* red;  // [2][2][MT]
  int slot;
  __device__ __forceinline__ float sum(float v, int h, int t) {
    float* r = red + slot * 2 * MT;
    r[h * MT + t] = v;
    csync();
    const float o = r[(1 - h) * MT + t];
    slot ^= 1;
    return v + o;
  }
};

// LayerNorm (eps 1e-5, biased variance) of the row whose half-h dimensions
// this thread holds -> fp16 into its 64 columns of the canonical K-major
// [128][128] operand
__device__ __forceinline__ void ln_store(const float (&hh)[HD], const float* __restrict__ g,
                                         const float* __restrict__ b, unsigned char* sA, int h, int t, Xch& xc) {
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < HD; ++c) s += hh[c];
  const float mean = xc.sum(s, h, t) * (1.0f / D);
  float q = 0.f;
#pragma unroll
  for (int c = 0; c < HD; ++c) q = fmaf(hh[c] - mean, hh[c] - mean, q);
  const float rs = 1.0f / sqrtf(xc.sum(q, h, t) * (1.0f / D) + 1e-5f);
  const int cb = h * HD;
#pragma unroll
  for (int c0 = 0; c0 < HD; c0 += 8) {
    const float4 g0 = *reinterpret_cast<const float4*>(g + cb + c0);
    const float4 g1 = *reinterpret_cast<const float4*>(g + cb + c0 + 4);
    const float4 b0 = *reinterpret_cast<const float4*>(b + cb + c0);
    const float4 b1 = *reinterpret_cast<const float4*>(b + cb + c0 + 4);
    const float gg[8] = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w};
    const float bb[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
    uint32_t w[4];
#pragma unroll
    for (int e = 0; e < 4; ++e)
      w[e] = tc::pack_f16x2(fmaf((hh[c0 + 2 * e] - mean) * rs, gg[2 * e], bb[2 * e]),
                             fmaf((hh[c0 + 2 * e + 1] - mean) * rs, gg[2 * e + 1], bb[2 * e + 1]));
    *reinterpret_cast<uint4*>(sA + tc::canon_off(t, cb + c0, D)) = make_uint4(w[0], w[1], w[2], w[3]);
  }
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
  bool live;
  int P, t0, S;
  uint64_t first;  // FULL: first sequence; SUFFIX: first index into perm
  uint64_t count;  // sequences available from `first`
};

__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(bar), "r"(phase)
      : "memory");
  return ok != 0;
}

// The weight ring as seen by the one thread that issues the MMAs and
// requests the chunks.  Chunk g of this CTA's stream (its tiles x L layers x
// NCH chunks, in consumption order) sits in stage g % NS; the k-th use of a
// stage is phase k of its barriers.
struct Ring {
  uint32_t w_addr, full, empty;
  const unsigned char* img;
  int L;
  uint64_t g;     // next chunk to consume
  uint64_t gl;    // next chunk to request
  uint64_t gmax;  // chunks in the stream
  // Request chunks while their stages are free (the MMAs of the chunk NS
  // earlier are done); with `need`, wait (bounded) until chunk g is requested.
  __device__ __forceinline__ bool pump(bool need) {
    while (gl < gmax && gl < g + NS) {
      const uint32_t st = uint32_t(gl % NS), ph = uint32_t((gl / NS) & 1) ^ 1u;
      if (!mbar_test(empty + 8u * st, ph)) {
        if (!(need && gl == g)) break;
        if (!wait_bar(empty + 8u * st, ph)) return false;
      }
      const int l = int((gl / NCH) % uint64_t(L)), ci = int(gl % NCH);
      tc::mbar_arrive_expect_tx(full + 8u * st, CHUNK);
      tc::bulk_g2s(w_addr + st * CHUNK, img + size_t(l) * LAYER_BYTES + size_t(ci) * CHUNK, CHUNK, full + 8u * st);
      ++gl;
    }
    return true;
  }
  // D (+)= A W_chunk^T over K = 128 for the next chunk of the stream; its
  // stage is released (empty) when these MMAs complete.  False on time-out.
  __device__ __forceinline__ bool gemm(uint32_t d_tmem, uint32_t a_addr, uint32_t accumulate) {
    constexpr uint32_t IDESC = tc::idesc_f16_f32(MT, D);
    if (!pump(true)) return false;
    const uint32_t st = uint32_t(g % NS), ph = uint32_t((g / NS) & 1);
    if (!wait_bar(full + 8u * st, ph)) return false;
    ++g;
    tc::fence_after_sync();
    const uint32_t b_addr = w_addr + st * CHUNK;
#pragma unroll
    for (uint32_t ks = 0; ks < D / 16; ++ks)
      tc::mma_f16(d_tmem, tc::sdesc(a_addr + ks * 256u, 128u, D * 16u), tc::sdesc(b_addr + ks * 256u, 128u, D * 16u),
                   IDESC, (accumulate || ks > 0) ? 1u : 0u);
    tc::mma_commit(empty + 8u * st);
    return pump(false);
  }
  // copies requested and never consumed (a stream left early) land before
  // the CTA leaves
  __device__ __forceinline__ bool drain() {
    bool ok = true;
    for (uint64_t k = g; k < gl; ++k)
      ok = wait_bar(full + 8u * uint32_t(k % NS), uint32_t((k / NS) & 1)) && ok;
    return ok;
  }
};

template <int DH>
__global__ void __launch_bounds__(NT, 1) tf128_kernel(Args a) {
  constexpr int H = D / DH;        // heads
  constexpr int HPH = H / 2;       // heads per half
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t bars[2 * NS + 2];  // full[NS], empty[NS], MMA chain, FFN-output chain
  __shared__ uint32_t s_tmem;
  __shared__ uint64_t s_tiles[ANQS_MAX_ORB + 1];
  __shared__ int s_abort;
  const int warp = threadIdx.x / 32;
  const int n = a.n, L = a.L;
  if (threadIdx.x == 0) {
    for (int i = 0; i < 2 * NS + 2; ++i) tc::mbar_init(tc::smem_u32(&bars[i]), 1);
    tc::fence_mbar_init();
    s_abort = 0;
  }
  if (warp == 0) {
    tc::tmem_alloc(tc::smem_u32(&s_tmem), 512);
    tc::tmem_relinquish();
  }
  ANQS_PDL_WAIT();
  ANQS_PDL_TRIGGER();
  float* s_head = reinterpret_cast<float*>(smem + OFF_HEAD);
  {
    const size_t tail = 5 * size_t(D) + size_t(n) * D + size_t(L) * layer_floats();
    for (int i = threadIdx.x; i < 8 * D + 8; i += NT) s_head[i] = a.params[tail + 2 * D + i];
  }
  // work: FULL one group; SUFFIX the groups j = 0..n-2 (P = n-1-j positions)
  if (threadIdx.x == 0) {
    uint64_t total = 0;
    s_tiles[0] = 0;
    if (a.mode == MODE_FULL) {
      const uint64_t S = MT / a.P, ns = a.n_seq.get();
      s_tiles[1] = (ns + S - 1) / S;
    } else {
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
  const uint64_t total = s_tiles[n_groups];
  const uint32_t w_addr = tc::smem_u32(smem + OFF_W);
  const uint32_t bar_full = tc::smem_u32(&bars[0]), bar_empty = tc::smem_u32(&bars[NS]);
  const uint32_t bar_m = tc::smem_u32(&bars[2 * NS]), bar_2 = tc::smem_u32(&bars[2 * NS + 1]);

  {
    // ---- compute warpgroups
    const int h = threadIdx.x / MT, t = threadIdx.x % MT;
    const uint32_t tmem = s_tmem;
    const uint32_t lane_base = uint32_t(t & ~31) << 16;
    unsigned char* sA = smem + OFF_A;
    unsigned char* sKV = smem + OFF_KV;
    const uint32_t a_addr = tc::smem_u32(sA);
    Xch xc{reinterpret_cast<float*>(smem + OFF_RED), 0};
    float* s_hx = reinterpret_cast<float*>(smem + OFF_HX);
    float* s_lp = reinterpret_cast<float*>(smem + OFF_LP);
    const bool issuer = threadIdx.x == 0;
    const uint64_t my_tiles = total > blockIdx.x ? (total - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    Ring ring{w_addr, bar_full, bar_empty, a.img, L, 0, 0, my_tiles * uint64_t(L) * NCH};
    if (issuer && !ring.pump(false)) atomicExch(&s_abort, 1);
    uint32_t ph_m = 0, ph_2 = 0;
    bool ok = true;
    const float scale = 1.0f / sqrtf(float(DH));
    const int cb = h * HD;  // this half's first model dimension
    for (uint64_t tile = blockIdx.x; ok && tile < total; tile += gridDim.x) {
      // ---- this thread's row
      Tile tl{};
      {
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
      const int s_loc = t / tl.P;
      const bool valid = s_loc < tl.S && uint64_t(s_loc) < tl.count;
      const int pos = valid ? tl.t0 + t % tl.P : 0;
      uint64_t x = 0, seq = 0, parent = 0;
      if (valid) {
        if (a.mode == MODE_FULL) {
          seq = tl.first + s_loc;
          x = a.x[seq];
        } else {
          seq = a.perm[tl.first + s_loc];
          x = a.xp[seq];
          parent = seq / a.K;
        }
      }
      const int row0 = s_loc * (valid ? tl.P : 0);
      float hh[HD];
      {
        const int token = pos == 0 ? 4 : int((x >> (2 * (pos - 1))) & 3ull);
        const float* tk = a.params + token * D + cb;
        const float* ps = a.params + (5 + pos) * D + cb;
#pragma unroll
        for (int c = 0; c < HD; c += 4) {
          const float4 u = __ldg(reinterpret_cast<const float4*>(tk + c));
          const float4 w = __ldg(reinterpret_cast<const float4*>(ps + c));
          hh[c] = u.x + w.x, hh[c + 1] = u.y + w.y, hh[c + 2] = u.z + w.z, hh[c + 3] = u.w + w.w;
        }
      }
      for (int l = 0; ok && l < L; ++l) {
        csync();  // the previous block's readers of the staged parameters are done
        stage_layer(a.params, n, l, s_lp);
        csync();
        const LayerP lp = staged_p(s_lp);
        ln_store(hh, lp.ln1_g, lp.ln1_b, sA, h, t, xc);
        tc::fence_async_smem();
        tc::fence_before_sync();
        csync();
        // q | k | v
        if (issuer) {
          bool r = ring.gemm(tmem, a_addr, 0);
          r = r && ring.gemm(tmem + 128u, a_addr, 0);
          r = r && ring.gemm(tmem + 256u, a_addr, 0);
          if (r) tc::mma_commit(bar_m);
          else atomicExch(&s_abort, 1);
        }
        ok = call(wait_bar(bar_m, ph_m));
        ph_m ^= 1;
        if (!ok) break;
        tc::fence_after_sync();
        // k, v of this row and half (+ bias) -> shared memory (and the parent cache)
#pragma unroll 1
        for (int kv = 0; kv < 2; ++kv) {
#pragma unroll 1
          for (int c0 = 0; c0 < HD; c0 += 32) {
            float v[32];
            tc::tmem_ld32(tmem + lane_base + uint32_t(128 * (kv + 1) + cb + c0), v);
            const float* bias = (kv == 0 ? lp.bk : lp.bv) + cb + c0;
            uint32_t w[16];
#pragma unroll
            for (int i = 0; i < 32; i += 2) w[i / 2] = tc::pack_f16x2(v[i] + bias[i], v[i + 1] + bias[i + 1]);
            const int off = kv * D + cb + c0;  // element offset within the k|v row
            uint4* dst = reinterpret_cast<uint4*>(sKV + t * KV_STRIDE + off * 2);
#pragma unroll
            for (int q = 0; q < 4; ++q) dst[q] = make_uint4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
            if (valid && a.kv_out) {
              uint4* gd = reinterpret_cast<uint4*>(a.kv_out + ((seq * L + l) * n + pos) * (2 * D) + off);
#pragma unroll
              for (int q = 0; q < 4; ++q) gd[q] = make_uint4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
            }
          }
        }
        csync();
        // causal attention of this row over the keys 0..pos, this half's heads
        const __half* pkv = a.kv_in ? a.kv_in + (parent * L + l) * size_t(n) * (2 * D) : nullptr;
#pragma unroll 1
        for (int hq = 0; hq < HPH; ++hq) {
          const int hd = h * HPH + hq;
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
        csync();
        // output projection (into q's columns)
        if (issuer) {
          if (ring.gemm(tmem, a_addr, 0)) tc::mma_commit(bar_m);
          else atomicExch(&s_abort, 1);
        }
        ok = call(wait_bar(bar_m, ph_m));
        ph_m ^= 1;
        if (!ok) break;
        tc::fence_after_sync();
#pragma unroll
        for (int c0 = 0; c0 < HD; c0 += 32) {
          float v[32];
          tc::tmem_ld32(tmem + lane_base + uint32_t(cb + c0), v);
#pragma unroll
          for (int i = 0; i < 32; ++i) hh[c0 + i] += v[i] + lp.bo[cb + c0 + i];
        }
        ln_store(hh, lp.ln2_g, lp.ln2_b, sA, h, t, xc);
        tc::fence_async_smem();
        tc::fence_before_sync();
        csync();
        // FFN in 4 chunks of 128 hidden units; f1_c in columns 128 + 128 (c & 1)
        if (issuer) {
          if (ring.gemm(tmem + 128u, a_addr, 0)) tc::mma_commit(bar_m);
          else atomicExch(&s_abort, 1);
        }
        ok = call(wait_bar(bar_m, ph_m));
        ph_m ^= 1;
        if (!ok) break;
        tc::fence_after_sync();
#pragma unroll 1
        for (int c = 0; c < 4; ++c) {
          if (issuer && c + 1 < 4) {
            if (ring.gemm(tmem + 128u + uint32_t(((c + 1) & 1) * 128), a_addr, 0)) tc::mma_commit(bar_m);
            else atomicExch(&s_abort, 1);
          }
          if (c >= 1) {  // the FFN-output MMA of chunk c-1 (and all before it) done: H buffer c & 1 is free
            ok = call(wait_bar(bar_2, ph_2));
            ph_2 ^= 1;
            if (!ok) break;
          }
          unsigned char* sH = sKV + (c & 1) * A_BYTES;
#pragma unroll
          for (int c0 = 0; c0 < HD; c0 += 32) {
            float v[32];
            tc::tmem_ld32(tmem + lane_base + uint32_t(128 + (c & 1) * 128 + cb + c0), v);
            const float* b1 = lp.b1 + c * D + cb + c0;
#pragma unroll
            for (int q8 = 0; q8 < 32; q8 += 8) {
              uint32_t w[4];
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                const int i = q8 + 2 * e;
                w[e] = tc::pack_f16x2(fmaxf(v[i] + b1[i], 0.f), fmaxf(v[i + 1] + b1[i + 1], 0.f));
              }
              *reinterpret_cast<uint4*>(sH + tc::canon_off(t, cb + c0 + q8, D)) = make_uint4(w[0], w[1], w[2], w[3]);
            }
          }
          tc::fence_async_smem();
          tc::fence_before_sync();
          csync();
          if (issuer) {
            if (ring.gemm(tmem + 384u, tc::smem_u32(sH), c > 0 ? 1u : 0u)) tc::mma_commit(bar_2);
            else atomicExch(&s_abort, 1);
          }
          if (c + 1 < 4) {
            ok = call(wait_bar(bar_m, ph_m));
            ph_m ^= 1;
            if (!ok) break;
            tc::fence_after_sync();
          }
        }
        if (!ok) break;
        ok = call(wait_bar(bar_2, ph_2));
        ph_2 ^= 1;
        if (!ok) break;
        tc::fence_after_sync();
#pragma unroll
        for (int c0 = 0; c0 < HD; c0 += 32) {
          float v[32];
          tc::tmem_ld32(tmem + lane_base + uint32_t(384 + cb + c0), v);
#pragma unroll
          for (int i = 0; i < 32; ++i) hh[c0 + i] += v[i] + lp.b2[cb + c0 + i];
        }
      }
      if (!ok) break;
      // final LayerNorm and head (partial sums over this half's dimensions)
      {
        const size_t tail = 5 * size_t(D) + size_t(n) * D + size_t(L) * layer_floats();
        const float* g = a.params + tail;
        const float* b = g + D;
        float s = 0.f;
#pragma unroll
        for (int c = 0; c < HD; ++c) s += hh[c];
        const float mean = xc.sum(s, h, t) * (1.0f / D);
        float q = 0.f;
#pragma unroll
        for (int c = 0; c < HD; ++c) q = fmaf(hh[c] - mean, hh[c] - mean, q);
        const float rs = 1.0f / sqrtf(xc.sum(q, h, t) * (1.0f / D) + 1e-5f);
        float out[8];
#pragma unroll
        for (int o = 0; o < 8; ++o) out[o] = 0.f;
#pragma unroll
        for (int c = 0; c < HD; ++c) {
          const float y = fmaf((hh[c] - mean) * rs, __ldg(g + cb + c), __ldg(b + cb + c));
#pragma unroll
          for (int o = 0; o < 8; ++o) out[o] = fmaf(y, s_head[o * D + cb + c], out[o]);
        }
        if (h == 1) {
#pragma unroll
          for (int o = 0; o < 8; ++o) s_hx[t * 8 + o] = out[o];
        }
        csync();
        if (h == 0 && valid) {
#pragma unroll
          for (int o = 0; o < 8; ++o) out[o] += s_hx[t * 8 + o] + s_head[8 * D + o];
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
            // the row's term to its own exchange slot (read above); the
            // sequence's first row adds its positions' terms below
            reinterpret_cast<float2*>(s_hx + t * 8)[0] =
                make_float2(((pmk >> v) & 1u) ? 0.5f * (ov - lse) : -INFINITY, pv);
          }
        }
      }
      if (a.mode == MODE_SUFFIX) {
        // one sum per connected determinant, over its positions in order: T[x']
        csync();
        if (h == 0 && valid && pos == tl.t0) {
          float sl = 0.f, sp = 0.f;
          for (int i = 0; i < tl.P; ++i) {
            const float2 tv = reinterpret_cast<const float2*>(s_hx + (t + i) * 8)[0];
            sl += tv.x;
            sp += tv.y;
          }
          a.T[seq] = make_float2(sl, sp);
        }
      }
      csync();  // shared k|v, hidden buffers and exchange slots are rewritten by the next tile
    }
    if (!ok) atomicExch(&s_abort, 1);
    if (issuer && !ring.drain()) atomicExch(&s_abort, 1);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (threadIdx.x == 0 && s_abort) atomicExch(a.status, 1);
  if (warp == 0) tc::tmem_dealloc(s_tmem, 512);
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
  const unsigned grid = unsigned(std::max<uint64_t>(1, std::min<uint64_t>(max_tiles, uint64_t(sms()))));
  const int dh = D / M->d.n_heads;
  ProfScope ps(prof, s);
  if (dh == 16) {
    ANQS_CUDA(cudaFuncSetAttribute(tf128_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(SMEM_BYTES)));
    ANQS_CUDA_LAUNCH("tf128_kernel", launch_k(tf128_kernel<16>, dim3(grid), dim3(NT), SMEM_BYTES, s, a));
  } else {
    ANQS_CUDA(cudaFuncSetAttribute(tf128_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(SMEM_BYTES)));
    ANQS_CUDA_LAUNCH("tf128_kernel", launch_k(tf128_kernel<32>, dim3(grid), dim3(NT), SMEM_BYTES, s, a));
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

}  // namespace

// Entry points used by the d_model dispatch of the BF16 transformer form.
bool tf128_supported(const anqs_model* M) {
  return M->d.d_model == D && (D / M->d.n_heads == 16 || D / M->d.n_heads == 32);
}

size_t tf128_packed_bytes(const anqs_model* M) { return size_t(M->d.n_layers) * LAYER_BYTES + 256; }

int tf128_pack(anqs_model* M, cudaStream_t s) {
  ANQS_CUDA_LAUNCH("tf128_pack_kernel", launch_k(tf128_pack_kernel, dim3(304), dim3(256), 0, s, M->params,
                                                 M->d.n_orb, M->d.n_layers, static_cast<unsigned char*>(M->packed)));
  return ANQS_OK;
}

int tf128_status_offset(const anqs_model* M) { return int(size_t(M->d.n_layers) * LAYER_BYTES); }

int launch_tf128_full(const anqs_model* M, const HamView& hv, const uint64_t* x, Count n_seq, int P, int last_only,
                      float* raw, __half* kv_out, int prof, cudaStream_t s) {
  Args a = full_args(x, n_seq, P, last_only, raw, kv_out, hv);
  const uint64_t S = MT / P;
  return launch(M, a, (n_seq.n + S - 1) / S, prof, s);
}

int launch_tf128_suffix(const anqs_model* M, const HamView& hv, const uint64_t* xp, const uint32_t* perm,
                        const uint32_t* offsets, uint32_t K, const __half* kv_in, float2* T, uint64_t m_max,
                        int prof, cudaStream_t s) {
  Args a{};
  a.mode = MODE_SUFFIX;
  a.hv = hv;
  a.xp = xp;
  a.perm = perm;
  a.offsets = offsets;
  a.K = K;
  a.kv_in = kv_in;
  a.T = T;
  const int n = hv.n;
  uint64_t tiles = 0;  // upper bound over the groups
  for (int j = 0; j + 1 < n; ++j) tiles += m_max / uint64_t(MT / (n - 1 - j)) + 1;
  return launch(M, a, tiles, prof, s);
}

}  // namespace anqs
