// BF16 tensor-core form of the per-slot MLP ansatz (tcgen05 MMA, TMEM
// accumulators, bulk-copied weight images), with reuse of the parent
// determinant's slots for its connected determinants.
//
// A CTA of 128 threads owns a tile of 128 rows (one row per thread and per
// TMEM lane).  For each slot p the CTA bulk-copies slot p's packed weight
// image into shared memory, writes the one-hot input of v_<p as the A
// operand, and runs the layers as M=128 x N=W x K GEMMs on the tensor cores
// (bf16 operands, f32 accumulation in TMEM).  Epilogues read the
// accumulator from TMEM, add the bias and apply tanh in f32, and write the
// bf16 activations back as the next A operand; the last hidden layer feeds
// the f32 head (8 outputs) on the CUDA cores, then the masked log-softmax
// (Appendix B.1 f3 with MU masking, Sec. III.C) in f32.
//
// Modes
//   PARENT  rows = unique samples x, all slots; writes log psi(x) and, per
//           (x, slot), the prefix sum of the slot terms and the masked
//           half-log-probabilities and phases of all 4 outcomes.
//   SUFFIX  rows = connected determinants x' (sorted by first differing slot
//           j); log psi(x') = parent prefix up to j + parent slot-j term of
//           v'_j + the network's slots p > j (Eq. anqs_def: slots <= j see
//           the same prefix as in x).
//   LOGPSI  rows = arbitrary determinants, all slots, log psi only.
//   LOGITS  rows = sampler frontier prefixes, one slot, the 8 raw outputs.
#include <cuda_bf16.h>

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
  uint32_t w1;      // layer-1 matrix [W][k1] bf16, canonical K-major
  uint32_t wk;      // hidden matrices [L-1][W][W] bf16, canonical, each W*W*2 bytes
  uint32_t bias;    // [L][W] f32
  uint32_t head;    // [8][W] f32
  uint32_t hbias;   // [8] f32
  uint32_t bytes;   // total, multiple of 128
};

__host__ __device__ inline uint32_t round_up(uint32_t a, uint32_t b) { return (a + b - 1) / b * b; }

__host__ __device__ inline SlotLayout slot_layout(int p, int W, int L) {
  SlotLayout s;
  s.k1 = round_up(4u * p, 16u);
  s.w1 = 0;
  s.wk = round_up(s.w1 + uint32_t(W) * s.k1 * 2u, 128u);
  s.bias = round_up(s.wk + uint32_t(L - 1) * W * W * 2u, 128u);
  s.head = round_up(s.bias + uint32_t(L) * W * 4u, 128u);
  s.hbias = round_up(s.head + 8u * W * 4u, 128u);
  s.bytes = round_up(s.hbias + 8u * 4u, 128u);
  return s;
}

struct TcView {
  int n, W, L;
  const unsigned char* img;   // packed images
  uint32_t img_off[ANQS_MAX_ORB + 1];
  uint32_t max_img;           // largest image (bytes)
  int* status;
};

// ---- packing: f32 parameters -> per-slot bf16/f32 images --------------------
__global__ void pack_kernel(MlpView m, TcView tv, unsigned char* img) {
  const int p = blockIdx.y;
  const int W = m.width, L = m.n_hidden;
  const SlotLayout S = slot_layout(p, W, L);
  unsigned char* base = img + tv.img_off[p];
  const float* W1 = m.params + m.slot_off[p];
  const float* b1 = W1 + size_t(W) * 4 * p;
  const float* Wk = b1 + W;
  const float* Wh = Wk + size_t(L - 1) * (size_t(W) * W + W);
  const float* bh = Wh + 8 * W;
  const uint32_t n1 = uint32_t(W) * S.k1;
  const uint32_t nk = uint32_t(L - 1) * W * W;
  const uint32_t total = n1 + nk + uint32_t(L) * W + 8u * W + 8u;
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    if (t < n1) {
      uint32_t r = t / S.k1, k = t % S.k1;
      float v = (k < 4u * p) ? W1[size_t(r) * 4 * p + k] : 0.f;
      *reinterpret_cast<uint16_t*>(base + S.w1 + tc::canon_off(r, k, S.k1)) =
          __bfloat16_as_ushort(__float2bfloat16_rn(v));
    } else if (t < n1 + nk) {
      uint32_t u = t - n1, l = u / (W * W), e = u % (W * W), r = e / W, k = e % W;
      float v = Wk[size_t(l) * (size_t(W) * W + W) + size_t(r) * W + k];
      *reinterpret_cast<uint16_t*>(base + S.wk + l * W * W * 2u + tc::canon_off(r, k, W)) =
          __bfloat16_as_ushort(__float2bfloat16_rn(v));
    } else if (t < n1 + nk + uint32_t(L) * W) {
      uint32_t u = t - n1 - nk, l = u / W, o = u % W;
      const float* bl = (l == 0) ? b1 : (Wk + size_t(l - 1) * (size_t(W) * W + W) + size_t(W) * W);
      reinterpret_cast<float*>(base + S.bias)[u] = bl[o];
    } else if (t < n1 + nk + uint32_t(L) * W + 8u * W) {
      uint32_t u = t - n1 - nk - uint32_t(L) * W;
      reinterpret_cast<float*>(base + S.head)[u] = Wh[u];
    } else {
      uint32_t u = t - n1 - nk - uint32_t(L) * W - 8u * W;
      reinterpret_cast<float*>(base + S.hbias)[u] = bh[u];
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
  // PARENT / LOGPSI / LOGITS: rows are x[0..n_rows); SUFFIX: rows perm[0..n_rows)
  const uint64_t* x;
  const uint64_t* n_rows_dev;  // LOGITS: device-side row count
  uint64_t n_rows;
  int p_single;                // LOGITS: the slot
  // SUFFIX
  const uint32_t* perm;
  const uint8_t* js;
  const float* cache;          // [n_parents][n][CACHE_F]
  uint32_t K;
  // outputs
  float* la;
  float* ph;
  float* cache_out;            // PARENT
  float* logits_out;           // LOGITS [n_rows][8]
};

template <int W, int MODE>
__global__ void __launch_bounds__(MT, 1) mlp_tc_kernel(TcView tv, HamView hv, TileArgs ta) {
  extern __shared__ __align__(1024) unsigned char smem[];
  // [0, max_img): slot image; then the A tile (128 rows x max(W, k1) bf16)
  unsigned char* s_img = smem;
  unsigned char* s_a = smem + round_up(tv.max_img, 1024u);
  __shared__ __align__(8) uint64_t s_bar[2];  // 0: weights, 1: mma
  __shared__ uint32_t s_tmem;
  __shared__ int s_jmin, s_abort;

  const int tid = threadIdx.x;
  const int n = tv.n, L = tv.L;
  const uint32_t bar_w = tc::smem_u32(&s_bar[0]), bar_m = tc::smem_u32(&s_bar[1]);
  const uint32_t a_addr = tc::smem_u32(s_a), img_addr = tc::smem_u32(s_img);
  constexpr uint32_t kCols = 2 * W;  // two accumulators
  constexpr uint32_t IDESC = tc::idesc_bf16_f32(MT, W);

  if (tid == 0) {
    tc::mbar_init(bar_w, 1);
    tc::mbar_init(bar_m, 1);
    tc::fence_mbar_init();
    s_abort = 0;
  }
  if (tid < 32) {
    tc::tmem_alloc(tc::smem_u32(&s_tmem), kCols);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = s_tmem;
  const uint32_t lane_base = uint32_t(tid & ~31) << 16;  // warp w reads TMEM lanes 32w..32w+31
  uint32_t ph_w = 0, ph_m = 0;

  const uint64_t n_rows = (MODE == MODE_LOGITS) ? *ta.n_rows_dev : ta.n_rows;
  const uint64_t n_tiles = (n_rows + MT - 1) / MT;
  for (uint64_t tile = blockIdx.x; tile < n_tiles && !s_abort; tile += gridDim.x) {
    const uint64_t r = tile * MT + tid;
    const bool valid = r < n_rows;
    uint64_t x = 0;
    int j = -1;
    float la = 0.f, phs = 0.f;
    uint64_t out_idx = r;
    if (MODE == MODE_SUFFIX) {
      if (valid) {
        const uint32_t row = ta.perm[r];
        out_idx = row;
        x = ta.x[row];
        j = ta.js[row];
        const uint64_t parent = row / ta.K;
        const float* c = ta.cache + (parent * n + j) * CACHE_F;
        const int vj = int((x >> (2 * j)) & 3ull);
        la = c[0] + c[2 + vj];
        phs = c[1] + c[6 + vj];
      } else {
        j = n;  // no slots
      }
    } else if (valid) {
      x = ta.x[r];
    }
    if (MODE == MODE_LOGITS) j = ta.p_single - 1;
    if (tid == 0) s_jmin = n;
    __syncthreads();
    if (valid || MODE != MODE_SUFFIX) atomicMin(&s_jmin, j);
    __syncthreads();
    const int p0 = (MODE == MODE_LOGITS) ? ta.p_single : s_jmin + 1;
    const int p1 = (MODE == MODE_LOGITS) ? ta.p_single + 1 : n;
    bool dead = false;

    for (int p = p0; p < p1; ++p) {
      const SlotLayout S = slot_layout(p, W, L);
      // weights of slot p (the previous slot's readers are done: barrier at loop end)
      if (tid == 0) {
        tc::mbar_arrive_expect_tx(bar_w, S.bytes);
        tc::bulk_g2s(img_addr, tv.img + tv.img_off[p], S.bytes, bar_w);
      }
      // layer-1 input: one-hot of v_<p, K = k1 columns
      for (uint32_t c = 0; c < S.k1; c += 8) {
        uint32_t w4[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          uint32_t lo = 0, hi = 0;
          const uint32_t k0 = c + 2 * e, k1 = k0 + 1;
          if (k0 < 4u * p && ((x >> (2 * (k0 >> 2))) & 3ull) == (k0 & 3u)) lo = 0x3F80u;
          if (k1 < 4u * p && ((x >> (2 * (k1 >> 2))) & 3ull) == (k1 & 3u)) hi = 0x3F80u;
          w4[e] = lo | (hi << 16);
        }
        *reinterpret_cast<uint4*>(s_a + tc::canon_off(tid, c, S.k1)) = make_uint4(w4[0], w4[1], w4[2], w4[3]);
      }
      tc::fence_async_smem();
      tc::fence_before_sync();
      __syncthreads();
      if (!wait_bar(bar_w, ph_w)) s_abort = 1;
      ph_w ^= 1;
      __syncthreads();
      if (s_abort) break;
      const float* bias = reinterpret_cast<const float*>(s_img + S.bias);
      const float* head = reinterpret_cast<const float*>(s_img + S.head);
      const float* hbias = reinterpret_cast<const float*>(s_img + S.hbias);
      float out[8];
#pragma unroll
      for (int o = 0; o < 8; ++o) out[o] = 0.f;

      bool aborted = false;
      for (int layer = 0; layer < L; ++layer) {
        const uint32_t K = layer == 0 ? S.k1 : uint32_t(W);
        const uint32_t d_tmem = tmem + uint32_t(layer & 1) * W;
        if (K > 0) {
          if (tid == 0) {
            tc::fence_after_sync();
            const uint32_t b_addr = img_addr + (layer == 0 ? S.w1 : S.wk + uint32_t(layer - 1) * W * W * 2u);
#pragma unroll 1
            for (uint32_t ks = 0; ks < K / 16; ++ks) {
              const uint64_t ad = tc::sdesc(a_addr + ks * 256u, 128u, K * 16u);
              const uint64_t bd = tc::sdesc(b_addr + ks * 256u, 128u, K * 16u);
              tc::mma_bf16(d_tmem, ad, bd, IDESC, ks > 0 ? 1u : 0u);
            }
            tc::mma_commit(bar_m);
          }
          if (!wait_bar(bar_m, ph_m)) s_abort = 1;
          ph_m ^= 1;
          __syncthreads();
          if (s_abort) {
            aborted = true;
            break;
          }
          tc::fence_after_sync();
        }
        const bool last = (layer == L - 1);
        const float* b = bias + layer * W;
#pragma unroll 1
        for (int c0 = 0; c0 < W; c0 += 32) {
          float v[32];
          if (K > 0) {
            tc::tmem_ld32(d_tmem + lane_base + uint32_t(c0), v);
          } else {
#pragma unroll
            for (int i = 0; i < 32; ++i) v[i] = 0.f;
          }
#pragma unroll
          for (int i = 0; i < 32; ++i) v[i] = tc::tanh_fast(v[i] + b[c0 + i]);
          if (!last) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              uint4 u;
              u.x = tc::pack_bf16x2(v[8 * q + 0], v[8 * q + 1]);
              u.y = tc::pack_bf16x2(v[8 * q + 2], v[8 * q + 3]);
              u.z = tc::pack_bf16x2(v[8 * q + 4], v[8 * q + 5]);
              u.w = tc::pack_bf16x2(v[8 * q + 6], v[8 * q + 7]);
              *reinterpret_cast<uint4*>(s_a + tc::canon_off(tid, c0 + 8 * q, W)) = u;
            }
          } else {
#pragma unroll
            for (int o = 0; o < 8; ++o) {
              const float* hw = head + o * W + c0;
              float acc = out[o];
#pragma unroll
              for (int i = 0; i < 32; ++i) acc = fmaf(hw[i], v[i], acc);
              out[o] = acc;
            }
          }
        }
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
      }
      if (aborted) break;
#pragma unroll
      for (int o = 0; o < 8; ++o) out[o] += hbias[o];

      if (MODE == MODE_LOGITS) {
        if (valid)
#pragma unroll
          for (int o = 0; o < 8; ++o) ta.logits_out[r * 8 + o] = out[o];
      } else if (valid && j < p) {
        // masked log-softmax of slot p for this row's prefix (f32)
        const uint64_t pm = (p == 0) ? 0ull : ((1ull << (2 * p)) - 1ull);
        const int a = __popcll(x & pm & 0x5555555555555555ull), bb = __popcll(x & pm & 0xAAAAAAAAAAAAAAAAull);
        const unsigned mk = slot_mask(hv, p, a, bb);
        float mx = -INFINITY;
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if ((mk >> u) & 1u) mx = fmaxf(mx, out[u]);
        float s = 0.f;
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if ((mk >> u) & 1u) s += __expf(out[u] - mx);
        const float lse = mx + __logf(s);
        const int v = int((x >> (2 * p)) & 3ull);
        if (MODE == MODE_PARENT) {
          float* c = ta.cache_out + (r * n + p) * CACHE_F;
          c[0] = la;
          c[1] = phs;
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            c[2 + u] = ((mk >> u) & 1u) ? 0.5f * (out[u] - lse) : -INFINITY;
            c[6 + u] = out[4 + u];
          }
        }
        if (!((mk >> v) & 1u)) dead = true;
        la += 0.5f * (out[v] - lse);
        phs += out[4 + v];
      }
    }
    if (MODE != MODE_LOGITS && valid) {
      bool outside = dead || (n < 32 && (x >> (2 * n)) != 0);
      ta.la[out_idx] = outside ? -INFINITY : la;
      ta.ph[out_idx] = phs;
    }
    __syncthreads();
  }
  if (s_abort && tid == 0) atomicExch(tv.status, ST_TIMEOUT);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (tid < 32) tc::tmem_dealloc(tmem, kCols);
}

// ---- sort of connected rows by first differing slot ---------------------------
__global__ void js_hist_kernel(const uint8_t* __restrict__ js, uint64_t m, int n, uint32_t* __restrict__ hist) {
  __shared__ uint32_t h[ANQS_MAX_ORB];
  for (int i = threadIdx.x; i < n; i += blockDim.x) h[i] = 0;
  __syncthreads();
  for (uint64_t t = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; t < m; t += uint64_t(gridDim.x) * blockDim.x)
    atomicAdd(&h[js[t]], 1u);
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    if (h[i]) atomicAdd(&hist[i], h[i]);
}

__global__ void js_offsets_kernel(const uint32_t* __restrict__ hist, int n, uint32_t* __restrict__ cursor) {
  if (threadIdx.x == 0) {
    uint32_t acc = 0;
    for (int i = 0; i < n; ++i) {
      cursor[i] = acc;
      acc += hist[i];
    }
  }
}

__global__ void js_scatter_kernel(const uint8_t* __restrict__ js, uint64_t m, uint32_t* __restrict__ cursor,
                                  uint32_t* __restrict__ perm) {
  for (uint64_t t = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; t < m; t += uint64_t(gridDim.x) * blockDim.x)
    perm[atomicAdd(&cursor[js[t]], 1u)] = uint32_t(t);
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

TcView make_view(const anqs_model* M) {
  TcView tv;
  tv.n = M->d.n_orb;
  tv.W = M->d.width;
  tv.L = M->d.n_hidden;
  tv.img = static_cast<const unsigned char*>(M->packed);
  tv.max_img = 0;
  for (int p = 0; p <= tv.n; ++p) tv.img_off[p] = uint32_t(M->pack_off[p]);
  for (int p = 0; p < tv.n; ++p) tv.max_img = std::max(tv.max_img, slot_layout(p, tv.W, tv.L).bytes);
  tv.status = reinterpret_cast<int*>(static_cast<unsigned char*>(M->packed) + M->pack_off[tv.n]);
  return tv;
}

size_t smem_bytes(const TcView& tv) {
  uint32_t kmax = std::max<uint32_t>(tv.W, round_up(4u * (tv.n - 1), 16u));
  return round_up(tv.max_img, 1024u) + size_t(MT) * kmax * 2u;
}

template <int MODE>
int launch_mode(const anqs_model* M, const HamView& hv, const TileArgs& ta, uint64_t max_rows, cudaStream_t s,
                int prof) {
  TcView tv = make_view(M);
  size_t sm = smem_bytes(tv);
  if (sm > 227 * 1024) return set_error(ANQS_ERR_UNSUPPORTED, "BF16 MLP slot image needs %zu bytes of shared memory", sm);
  uint64_t tiles = (max_rows + MT - 1) / MT;
  unsigned grid = unsigned(std::min<uint64_t>(tiles ? tiles : 1, uint64_t(num_sms())));
  ProfScope ps(prof, s);
  if (tv.W == 128) {
    ANQS_CUDA(cudaFuncSetAttribute(mlp_tc_kernel<128, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm)));
    mlp_tc_kernel<128, MODE><<<grid, MT, sm, s>>>(tv, hv, ta);
  } else {
    ANQS_CUDA(cudaFuncSetAttribute(mlp_tc_kernel<64, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm)));
    mlp_tc_kernel<64, MODE><<<grid, MT, sm, s>>>(tv, hv, ta);
  }
  ANQS_LAUNCHED("mlp_tc_kernel");
  return ANQS_OK;
}

struct ElocWs {
  uint64_t* xp;
  double* hv;
  uint8_t* js;
  double* hd;
  float *la_x, *ph_x, *cache, *la_p, *ph_p;
  uint32_t *perm, *hist, *cursor;
};

size_t plan_eloc(const anqs_ham* H, uint64_t n_x, Arena& A, ElocWs& w) {
  const uint64_t m = n_x * H->v.K;
  w.xp = A.take<uint64_t>(m);
  w.hv = A.take<double>(m);
  w.js = A.take<uint8_t>(m);
  w.hd = A.take<double>(n_x);
  w.la_x = A.take<float>(n_x);
  w.ph_x = A.take<float>(n_x);
  w.cache = A.take<float>(n_x * H->v.n * CACHE_F);
  w.la_p = A.take<float>(m);
  w.ph_p = A.take<float>(m);
  w.perm = A.take<uint32_t>(m);
  w.hist = A.take<uint32_t>(ANQS_MAX_ORB);
  w.cursor = A.take<uint32_t>(ANQS_MAX_ORB);
  return A.off;
}

}  // namespace

int mlp_tc_pack_alloc(anqs_model* M) {
  const int n = M->d.n_orb, W = M->d.width, L = M->d.n_hidden;
  if (W != 64 && W != 128) return set_error(ANQS_ERR_UNSUPPORTED, "BF16 MLP form supports width 64 or 128");
  M->pack_off.assign(n + 1, 0);
  uint64_t off = 0;
  for (int p = 0; p < n; ++p) {
    M->pack_off[p] = off;
    off += slot_layout(p, W, L).bytes;
  }
  M->pack_off[n] = off;  // status word after the images
  M->packed_bytes = off + 256;
  TcView tv;
  tv.n = n;
  tv.W = W;
  tv.L = L;
  tv.max_img = 0;
  for (int p = 0; p < n; ++p) tv.max_img = std::max(tv.max_img, slot_layout(p, W, L).bytes);
  if (smem_bytes(tv) > 227 * 1024)
    return set_error(ANQS_ERR_UNSUPPORTED, "BF16 MLP slot image too large for shared memory (%zu bytes)", smem_bytes(tv));
  ANQS_CUDA(cudaMalloc(&M->packed, M->packed_bytes));
  ANQS_CUDA(cudaMemset(M->packed, 0, M->packed_bytes));
  return ANQS_OK;
}

int mlp_tc_pack(anqs_model* M, cudaStream_t s) {
  TcView tv = make_view(M);
  dim3 grid(64, unsigned(M->d.n_orb));
  pack_kernel<<<grid, 256, 0, s>>>(M->mlp, tv, static_cast<unsigned char*>(M->packed));
  ANQS_LAUNCHED("pack_kernel");
  return ANQS_OK;
}

int mlp_tc_status(const anqs_model* M, int* status) {
  int v = 0;
  ANQS_CUDA(cudaMemcpy(&v, static_cast<const unsigned char*>(M->packed) + M->pack_off[M->d.n_orb], sizeof(int),
                       cudaMemcpyDeviceToHost));
  *status = v;
  return ANQS_OK;
}

int launch_mlp_tc_logpsi(const anqs_model* M, const HamView& hv, const uint64_t* x, uint64_t n_x, float* la,
                         float* ph, cudaStream_t s) {
  TileArgs ta{};
  ta.x = x;
  ta.n_rows = n_x;
  ta.la = la;
  ta.ph = ph;
  return launch_mode<MODE_LOGPSI>(M, hv, ta, n_x, s, PROF_TC_PARENT);
}

int launch_mlp_tc_slot_logits(const anqs_model* M, const HamView& hv, int p, const uint64_t* pre,
                              const uint64_t* n_dev, uint64_t max_rows, float* out8, cudaStream_t s) {
  TileArgs ta{};
  ta.x = pre;
  ta.n_rows_dev = n_dev;
  ta.p_single = p;
  ta.logits_out = out8;
  return launch_mode<MODE_LOGITS>(M, hv, ta, max_rows, s, PROF_TC_SLOT);
}

size_t eloc_tc_workspace(const anqs_model* M, const anqs_ham* H, uint64_t n_x) {
  Arena A(nullptr, 0);
  ElocWs w;
  return plan_eloc(H, n_x, A, w);
}

int run_eloc_tc(const anqs_model* M, const anqs_ham* H, const uint64_t* x, uint64_t n_x, double* ere, double* eim,
                void* ws, size_t ws_bytes, cudaStream_t s) {
  Arena A(ws, ws_bytes);
  ElocWs w;
  plan_eloc(H, n_x, A, w);
  if (!A.fits()) return set_error(ANQS_ERR_CAPACITY, "workspace needs %zu bytes", A.off);
  const uint64_t K = H->v.K, m = n_x * K;
  if (m > 0xffffffffull) return set_error(ANQS_ERR_UNSUPPORTED, "more than 2^32 connected determinants per call");
  ANQS_TRY(launch_connected(H->v, x, n_x, w.xp, w.hv, w.js, w.hd, s));
  {
    TileArgs ta{};
    ta.x = x;
    ta.n_rows = n_x;
    ta.la = w.la_x;
    ta.ph = w.ph_x;
    ta.cache_out = w.cache;
    ANQS_TRY(launch_mode<MODE_PARENT>(M, H->v, ta, n_x, s, PROF_TC_PARENT));
  }
  {
    ProfScope ps(PROF_TC_SORT, s);
    ANQS_CUDA(cudaMemsetAsync(w.hist, 0, ANQS_MAX_ORB * sizeof(uint32_t), s));
    unsigned g = unsigned(std::min<uint64_t>((m + 255) / 256, 152 * 4));
    js_hist_kernel<<<g ? g : 1, 256, 0, s>>>(w.js, m, H->v.n, w.hist);
    ANQS_LAUNCHED("js_hist_kernel");
    js_offsets_kernel<<<1, 32, 0, s>>>(w.hist, H->v.n, w.cursor);
    ANQS_LAUNCHED("js_offsets_kernel");
    js_scatter_kernel<<<g ? g : 1, 256, 0, s>>>(w.js, m, w.cursor, w.perm);
    ANQS_LAUNCHED("js_scatter_kernel");
  }
  {
    TileArgs ta{};
    ta.x = w.xp;
    ta.n_rows = m;
    ta.perm = w.perm;
    ta.js = w.js;
    ta.cache = w.cache;
    ta.K = uint32_t(K);
    ta.la = w.la_p;
    ta.ph = w.ph_p;
    ANQS_TRY(launch_mode<MODE_SUFFIX>(M, H->v, ta, m, s, PROF_TC_SUFFIX));
  }
  return launch_eloc_sum(H->v, n_x, w.hv, w.hd, w.la_x, w.ph_x, w.la_p, w.ph_p, ere, eim, s);
}

}  // namespace anqs
