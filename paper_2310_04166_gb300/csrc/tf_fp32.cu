// Plain FP32 form of the causal-transformer ansatz (SIMT, no tensor cores,
// no prefix reuse): log psi of arbitrary determinants and slot logits for the
// sampler.
//
// The network (decoder-only, pre-LayerNorm, eps 1e-5): position t reads the
// start token (t = 0) or the slot value v_{t-1}, h_t = tok[token] + pos[t];
// each block adds causal multi-head attention of LN1(h) and a ReLU FFN
// (hidden 4d) of LN2(h) to the residual stream; the head maps LNf(h_t) to the
// 8 outputs of slot t (modulus logits l_0..l_3, phases phi_0..phi_3), which
// enter the masked slot conditional of Appendix B.1 (f3) with MU masking
// (Sec. III.C) exactly as for the MLP.
//
// A CTA of 256 threads owns a tile of MT rows = S sequences x T positions
// (MT * 6d floats of activations in shared memory: residual h, the LayerNorm
// output / attention output a, and a 4d-wide buffer for q|k|v or the FFN
// hidden layer); weights stream through a staged 32 x 128 shared-memory
// chunk.
#include <cmath>

#include "common.cuh"

namespace anqs {
namespace {

constexpr int NT = 256;
constexpr int KC = 32;   // K depth of a staged weight chunk
constexpr int NCB = 128; // maximum columns of a staged weight chunk
constexpr int WS_FLOATS = KC * (NCB + 1);

template <int D>
struct Cfg {
  static constexpr int MT = D <= 64 ? 128 : (D == 128 ? 64 : 32);  // rows per tile
  static constexpr int RPT = MT / 8;                                 // rows per warp
  static constexpr int CJ = (D >= 128 ? 128 : D) / 32;               // column groups per chunk
  static constexpr int LB = 4 * D + 1;                               // row stride of the 4d buffer
  static constexpr size_t floats = size_t(MT) * (2 * D + LB) + WS_FLOATS + size_t(MT) * 8;
  static constexpr size_t bytes = floats * sizeof(float);
};

// Parameter offsets (floats) of the flat layout documented in anqs.h.
struct TfLayer {
  const float *ln1_g, *ln1_b, *wq, *bq, *wk, *bk, *wv, *bv, *wo, *bo, *ln2_g, *ln2_b, *w1, *b1, *w2, *b2;
};

__device__ __forceinline__ TfLayer tf_layer(const TfView& m, int l) {
  const size_t D = m.d, per = 12 * D * D + 13 * D;
  const float* b = m.params + 5 * D + size_t(m.n) * D + size_t(l) * per;
  TfLayer L;
  L.ln1_g = b;
  L.ln1_b = b + D;
  L.wq = b + 2 * D;
  L.bq = L.wq + D * D;
  L.wk = L.bq + D;
  L.bk = L.wk + D * D;
  L.wv = L.bk + D;
  L.bv = L.wv + D * D;
  L.wo = L.bv + D;
  L.bo = L.wo + D * D;
  L.ln2_g = L.bo + D;
  L.ln2_b = L.ln2_g + D;
  L.w1 = L.ln2_b + D;
  L.b1 = L.w1 + 4 * D * D;
  L.w2 = L.b1 + 4 * D;
  L.b2 = L.w2 + 4 * D * D;
  return L;
}

__device__ __forceinline__ const float* tf_tail(const TfView& m) {
  const size_t D = m.d, per = 12 * D * D + 13 * D;
  return m.params + 5 * D + size_t(m.n) * D + size_t(m.L) * per;  // lnf_g, lnf_b, head_w, head_b
}

// out(r, c) = sum_k A[r][k] W[c][k] for the MT rows and N columns (W row-major
// [N][K], K a multiple of 32); warp w owns rows w + 8 i, lane the columns
// n0 + lane + 32 j of each staged chunk.  epi(r, c, value) stores a result.
template <int D, class Epi>
__device__ __forceinline__ void gemm(const float* A, int lda, int K, const float* __restrict__ W, int N, float* ws,
                                     Epi epi) {
  constexpr int RPT = Cfg<D>::RPT, CJ = Cfg<D>::CJ, NC = 32 * CJ;
  const int lane = threadIdx.x & 31, wg = threadIdx.x >> 5;
  for (int n0 = 0; n0 < N; n0 += NC) {
    float acc[RPT][CJ];
#pragma unroll
    for (int i = 0; i < RPT; ++i)
#pragma unroll
      for (int j = 0; j < CJ; ++j) acc[i][j] = 0.f;
    for (int k0 = 0; k0 < K; k0 += KC) {
      __syncthreads();
      for (int idx = threadIdx.x; idx < NC * KC; idx += NT) {
        const int c = idx / KC, kk = idx % KC;
        ws[kk * (NC + 1) + c] = __ldg(W + size_t(n0 + c) * K + k0 + kk);
      }
      __syncthreads();
#pragma unroll 4
      for (int kk = 0; kk < KC; ++kk) {
        float a[RPT], b[CJ];
#pragma unroll
        for (int i = 0; i < RPT; ++i) a[i] = A[(wg + 8 * i) * lda + k0 + kk];
#pragma unroll
        for (int j = 0; j < CJ; ++j) b[j] = ws[kk * (NC + 1) + lane + 32 * j];
#pragma unroll
        for (int i = 0; i < RPT; ++i)
#pragma unroll
          for (int j = 0; j < CJ; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
      }
    }
#pragma unroll
    for (int i = 0; i < RPT; ++i)
#pragma unroll
      for (int j = 0; j < CJ; ++j) epi(wg + 8 * i, n0 + lane + 32 * j, acc[i][j]);
  }
  __syncthreads();
}

// y[r] = LN(x[r]) * g + b over D features, one warp per row (biased variance)
template <int D>
__device__ __forceinline__ void layer_norm(const float* x, float* y, const float* __restrict__ g,
                                           const float* __restrict__ b) {
  constexpr int MT = Cfg<D>::MT, E = D / 32;
  const int lane = threadIdx.x & 31, wg = threadIdx.x >> 5;
  for (int r = wg; r < MT; r += NT / 32) {
    float v[E], s = 0.f;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      v[e] = x[r * D + lane + 32 * e];
      s += v[e];
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    const float mean = s / float(D);
    float q = 0.f;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      v[e] -= mean;
      q = fmaf(v[e], v[e], q);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
    const float inv = 1.0f / sqrtf(q / float(D) + 1e-5f);
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int c = lane + 32 * e;
      y[r * D + c] = fmaf(v[e] * inv, __ldg(g + c), __ldg(b + c));
    }
  }
  __syncthreads();
}

// Forward of a tile: rows r = s T + t for s < S sequences (determinant or
// prefix xs[s]) and t < T positions.  Leaves the 8 outputs of every row in
// out8[MT][8].
template <int D>
__device__ void tile_forward(const TfView& m, const uint64_t* xs, int S, int T, float* smem) {
  constexpr int MT = Cfg<D>::MT, LB = Cfg<D>::LB;
  float* h = smem;                 // [MT][D] residual stream
  float* a = h + MT * D;           // [MT][D] LayerNorm / attention output
  float* buf = a + MT * D;         // [MT][LB] q|k|v or FFN hidden
  float* ws = buf + MT * LB;       // staged weight chunk
  float* out8 = ws + WS_FLOATS;    // [MT][8]
  const int rows = S * T;
  const float* tok = m.params;
  const float* pos = m.params + 5 * D;
  for (int idx = threadIdx.x; idx < MT * D; idx += NT) {
    const int r = idx / D, c = idx % D;
    float v = 0.f;
    if (r < rows) {
      const int s = r / T, t = r % T;
      const int token = t == 0 ? 4 : int((xs[s] >> (2 * (t - 1))) & 3ull);
      v = __ldg(tok + token * D + c) + __ldg(pos + t * D + c);
    }
    h[idx] = v;
  }
  __syncthreads();
  const int H = m.H, dh = D / H;
  const float scale = 1.0f / sqrtf(float(dh));
  for (int l = 0; l < m.L; ++l) {
    const TfLayer P = tf_layer(m, l);
    layer_norm<D>(h, a, P.ln1_g, P.ln1_b);
    gemm<D>(a, D, D, P.wq, D, ws, [&](int r, int c, float v) { buf[r * LB + c] = v + __ldg(P.bq + c); });
    gemm<D>(a, D, D, P.wk, D, ws, [&](int r, int c, float v) { buf[r * LB + D + c] = v + __ldg(P.bk + c); });
    gemm<D>(a, D, D, P.wv, D, ws, [&](int r, int c, float v) { buf[r * LB + 2 * D + c] = v + __ldg(P.bv + c); });
    // causal attention, one thread per (row, head): two passes over the keys
    for (int task = threadIdx.x; task < MT * H; task += NT) {
      const int r = task / H, hd = task % H;
      const int s = r / T, t = r % T;
      const float* q = buf + r * LB + hd * dh;
      float sc[32];
      float mx = -INFINITY;
#pragma unroll
      for (int u = 0; u < 32; ++u) {
        sc[u] = -INFINITY;
        if (u <= t && r < rows) {
          const float* k = buf + (s * T + u) * LB + D + hd * dh;
          float dot = 0.f;
          for (int e = 0; e < dh; ++e) dot = fmaf(q[e], k[e], dot);
          sc[u] = dot * scale;
          mx = fmaxf(mx, sc[u]);
        }
      }
      float sum = 0.f;
#pragma unroll
      for (int u = 0; u < 32; ++u) {
        const float p = (u <= t && r < rows) ? expf(sc[u] - mx) : 0.f;
        sc[u] = p;
        sum += p;
      }
      const float inv = r < rows ? 1.0f / sum : 0.f;
      for (int e = 0; e < dh; ++e) {
        float o = 0.f;
#pragma unroll
        for (int u = 0; u < 32; ++u)
          if (u <= t && r < rows) o = fmaf(sc[u], buf[(s * T + u) * LB + 2 * D + hd * dh + e], o);
        a[r * D + hd * dh + e] = o * inv;
      }
    }
    __syncthreads();
    gemm<D>(a, D, D, P.wo, D, ws, [&](int r, int c, float v) { h[r * D + c] += v + __ldg(P.bo + c); });
    layer_norm<D>(h, a, P.ln2_g, P.ln2_b);
    gemm<D>(a, D, D, P.w1, 4 * D, ws,
            [&](int r, int c, float v) { buf[r * LB + c] = fmaxf(v + __ldg(P.b1 + c), 0.f); });
    gemm<D>(buf, LB, 4 * D, P.w2, D, ws, [&](int r, int c, float v) { h[r * D + c] += v + __ldg(P.b2 + c); });
  }
  const float* tail = tf_tail(m);
  layer_norm<D>(h, a, tail, tail + D);
  const float* hw = tail + 2 * D;
  const float* hb = hw + 8 * D;
  for (int task = threadIdx.x; task < MT * 8; task += NT) {
    const int r = task >> 3, o = task & 7;
    float acc = __ldg(hb + o);
    const float* wr = hw + o * D;
    for (int k = 0; k < D; ++k) {
      const int kk = (k + r) & (D - 1);  // rotate the start to spread shared-memory banks
      acc = fmaf(a[r * D + kk], __ldg(wr + kk), acc);
    }
    out8[task] = acc;
  }
  __syncthreads();
}

// log-softmax term of the chosen outcome (FP32), as for the MLP: normalised
// over nm, dead when v is not physical
__device__ __forceinline__ void slot_term(const float* o8, unsigned nm, unsigned phys, int v, float& la, float& ph,
                                          bool& dead) {
  const unsigned mask = nm;
  if (!((phys >> v) & 1u)) {
    dead = true;
    return;
  }
  float mx = -INFINITY;
  for (int u = 0; u < 4; ++u)
    if ((mask >> u) & 1u) mx = fmaxf(mx, o8[u]);
  float s = 0.f;
  for (int u = 0; u < 4; ++u)
    if ((mask >> u) & 1u) s += expf(o8[u] - mx);
  la += 0.5f * (o8[v] - mx - logf(s));
  ph += o8[4 + v];
}

template <int D>
__global__ void __launch_bounds__(NT, 1) tf_logpsi_kernel(TfView m, HamView hv, const uint64_t* __restrict__ xs,
                                                          Count n_x_, float* __restrict__ la_out,
                                                          float* __restrict__ ph_out) {
  ANQS_PDL_ENTRY();
  extern __shared__ float smem[];
  constexpr int MT = Cfg<D>::MT;
  __shared__ uint64_t xt[MT];
  float* out8 = smem + Cfg<D>::floats - MT * 8;
  const uint64_t n_x = n_x_.get();
  const int T = m.n, S = MT / T;
  const uint64_t n_tiles = (n_x + S - 1) / S;
  for (uint64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const uint64_t base = tile * S;
    const int ns = int(n_x - base < uint64_t(S) ? n_x - base : uint64_t(S));
    if (threadIdx.x < S) xt[threadIdx.x] = threadIdx.x < ns ? xs[base + threadIdx.x] : 0ull;
    __syncthreads();
    tile_forward<D>(m, xt, ns, T, smem);
    if (threadIdx.x < ns) {
      const int s = threadIdx.x;
      const uint64_t x = xt[s];
      float la = 0.f, ph = 0.f;
      bool dead = false;
      int ca = 0, cb = 0;
      for (int p = 0; p < T; ++p) {
        const int v = int((x >> (2 * p)) & 3ull);
        const unsigned pm = slot_mask(hv, p, ca, cb, x);
        slot_term(out8 + (s * T + p) * 8, norm_mask(hv, p, pm), pm, v, la, ph, dead);
        ca += v & 1;
        cb += v >> 1;
      }
      const bool out_of_sector = dead || (hv.n < 32 && (x >> (2 * hv.n)) != 0);
      la_out[base + s] = out_of_sector ? -INFINITY : la;
      ph_out[base + s] = ph;
    }
    __syncthreads();
  }
}

template <int D>
__global__ void __launch_bounds__(NT, 1) tf_slot_logits_kernel(TfView m, int p, const uint64_t* __restrict__ pre,
                                                               const uint64_t* __restrict__ n_rows_dev,
                                                               float* __restrict__ out) {
  ANQS_PDL_ENTRY();
  extern __shared__ float smem[];
  constexpr int MT = Cfg<D>::MT;
  __shared__ uint64_t xt[MT];
  float* out8 = smem + Cfg<D>::floats - MT * 8;
  const uint64_t n_rows = *n_rows_dev;
  const int T = p + 1, S = MT / T;
  const uint64_t n_tiles = (n_rows + S - 1) / S;
  for (uint64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const uint64_t base = tile * S;
    const int ns = int(n_rows - base < uint64_t(S) ? n_rows - base : uint64_t(S));
    if (threadIdx.x < S) xt[threadIdx.x] = threadIdx.x < ns ? pre[base + threadIdx.x] : 0ull;
    __syncthreads();
    tile_forward<D>(m, xt, ns, T, smem);
    for (int idx = threadIdx.x; idx < ns * 8; idx += NT)
      out[(base + (idx >> 3)) * 8 + (idx & 7)] = out8[((idx >> 3) * T + T - 1) * 8 + (idx & 7)];
    __syncthreads();
  }
}

template <int D>
int logpsi_d(const TfView& m, const HamView& hv, const uint64_t* x, Count n_x, float* la, float* ph,
             cudaStream_t s) {
  const int S = Cfg<D>::MT / m.n;
  const uint64_t tiles = (n_x.n + S - 1) / S;
  const unsigned grid = unsigned(tiles < 152 ? (tiles ? tiles : 1) : 152);
  ANQS_CUDA(cudaFuncSetAttribute(tf_logpsi_kernel<D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 int(Cfg<D>::bytes)));
  ProfScope ps(PROF_TF, s);
  ANQS_CUDA_LAUNCH("tf_logpsi_kernel",
                   launch_k(tf_logpsi_kernel<D>, dim3(grid), dim3(NT), Cfg<D>::bytes, s, m, hv, x, n_x, la, ph));
  return ANQS_OK;
}

template <int D>
int logits_d(const TfView& m, int p, const uint64_t* pre, const uint64_t* nr, uint64_t max_rows, float* out,
             cudaStream_t s) {
  const int S = Cfg<D>::MT / (p + 1);
  const uint64_t tiles = (max_rows + S - 1) / S;
  const unsigned grid = unsigned(tiles < 152 ? (tiles ? tiles : 1) : 152);
  ANQS_CUDA(cudaFuncSetAttribute(tf_slot_logits_kernel<D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 int(Cfg<D>::bytes)));
  ProfScope ps(PROF_TF, s);
  ANQS_CUDA_LAUNCH("tf_slot_logits_kernel",
                   launch_k(tf_slot_logits_kernel<D>, dim3(grid), dim3(NT), Cfg<D>::bytes, s, m, p, pre, nr, out));
  return ANQS_OK;
}

}  // namespace

int launch_tf_fp32_logpsi(const TfView& m, const HamView& hv, const uint64_t* x, Count n_x, float* la, float* ph,
                          cudaStream_t s) {
  if (n_x.n == 0) return ANQS_OK;
  switch (m.d) {
    case 32: return logpsi_d<32>(m, hv, x, n_x, la, ph, s);
    case 64: return logpsi_d<64>(m, hv, x, n_x, la, ph, s);
    case 128: return logpsi_d<128>(m, hv, x, n_x, la, ph, s);
    case 256: return logpsi_d<256>(m, hv, x, n_x, la, ph, s);
  }
  return set_error(ANQS_ERR_UNSUPPORTED, "d_model %d", m.d);
}

int launch_tf_fp32_slot_logits(const TfView& m, int p, const uint64_t* pre, const uint64_t* nr, uint64_t max_rows,
                               float* out, cudaStream_t s) {
  switch (m.d) {
    case 32: return logits_d<32>(m, p, pre, nr, max_rows, out, s);
    case 64: return logits_d<64>(m, p, pre, nr, max_rows, out, s);
    case 128: return logits_d<128>(m, p, pre, nr, max_rows, out, s);
    case 256: return logits_d<256>(m, p, pre, nr, max_rows, out, s);
  }
  return set_error(ANQS_ERR_UNSUPPORTED, "d_model %d", m.d);
}

}  // namespace anqs
