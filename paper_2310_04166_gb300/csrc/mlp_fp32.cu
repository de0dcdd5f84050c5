// Plain FP32 form of the per-slot MLP ansatz (SIMT, no tensor cores, no
// prefix reuse): log psi of arbitrary determinants, slot logits for the
// sampler, and the hand-written adjoint for the VMC gradient.
//
// Slot p's network (Appendix B.1 layout with one network per spatial
// orbital): h_1 = tanh(b_1 + sum_{q<p} W_1[:, 4q + v_q]) (the one-hot input
// is a column gather), h_k = tanh(W_k h_{k-1} + b_k) for k = 2..L, and the
// head out = W_{L+1} h_L + b_{L+1} = (l_0..l_3, phi_0..phi_3).  The slot
// conditional is the masked softmax of l over the allowed outcomes
// (activation f3 of Appendix B.1 with MU masking, Sec. III.C).
//
// A CTA of 256 threads owns a tile of R = 32 rows; activations stay in
// shared memory, weights stream through a padded shared-memory chunk.
#include <algorithm>
#include <cmath>

#include "common.cuh"

namespace anqs {
namespace {

constexpr int R = 32;    // rows per CTA tile (log psi and slot logits)
// rows per CTA tile of the adjoint: the smallest of 16, 24, 32 whose tiles fit
// in one wave of CTAs (rg_for)
constexpr int NT = 256;  // threads per CTA
constexpr int KC = 32;   // weight chunk depth

struct MlpPtr {
  const float* W1;  // [w][4p] (absent for p = 0)
  const float* b1;  // [w]
  const float* Wk;  // first hidden-to-hidden matrix
  const float* Wh;  // head [8][w]
  const float* bh;  // [8]
};

__device__ __forceinline__ MlpPtr slot_ptrs(const MlpView& m, int p) {
  MlpPtr r;
  const int w = m.width;
  r.W1 = m.params + m.slot_off[p];
  r.b1 = r.W1 + size_t(w) * 4 * p;
  r.Wk = r.b1 + w;
  r.Wh = r.Wk + size_t(m.n_hidden - 1) * (size_t(w) * w + w);
  r.bh = r.Wh + 8 * w;
  return r;
}

// out[r][c] = sum_k in[r][k] * B(k, c), B(k, c) = W[c][k] (forward) or W[k][c]
// (adjoint).  Each warp owns R/8 rows, each lane W/32 columns.  With wres
// the matrix is already resident in shared memory (row stride W + 1, so
// that both access patterns are free of bank conflicts) and no chunk is
// staged; otherwise 32-row chunks of W stream through ws.
template <int W, bool ADJ, int RR = R>
__device__ __forceinline__ void tile_gemm(const float* in, const float* __restrict__ Wg, float* ws,
                                          float (&acc)[RR / 8][W / 32], const float* wres = nullptr) {
  constexpr int RPT = RR / 8, CPT = W / 32;
  const int lane = threadIdx.x & 31, wg = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < RPT; ++i)
#pragma unroll
    for (int j = 0; j < CPT; ++j) acc[i][j] = 0.f;
  if (wres) {
    __syncthreads();  // `in` was written by other threads
#pragma unroll 4
    for (int k = 0; k < W; ++k) {
      float a[RPT], b[CPT];
#pragma unroll
      for (int i = 0; i < RPT; ++i) a[i] = in[(wg * RPT + i) * W + k];
#pragma unroll
      for (int j = 0; j < CPT; ++j)
        b[j] = ADJ ? wres[k * (W + 1) + lane + 32 * j] : wres[(lane + 32 * j) * (W + 1) + k];
#pragma unroll
      for (int i = 0; i < RPT; ++i)
#pragma unroll
        for (int j = 0; j < CPT; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    return;
  }
  for (int k0 = 0; k0 < W; k0 += KC) {
    __syncthreads();
    for (int idx = threadIdx.x; idx < KC * W; idx += NT) {
      int c, kk;
      float val;
      if (!ADJ) {
        c = idx / KC;
        kk = idx % KC;
        val = __ldg(Wg + size_t(c) * W + k0 + kk);
      } else {
        kk = idx / W;
        c = idx % W;
        val = __ldg(Wg + size_t(k0 + kk) * W + c);
      }
      ws[kk * (W + 1) + c] = val;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < KC; ++kk) {
      float a[RPT], b[CPT];
#pragma unroll
      for (int i = 0; i < RPT; ++i) a[i] = in[(wg * RPT + i) * W + k0 + kk];
#pragma unroll
      for (int j = 0; j < CPT; ++j) b[j] = ws[kk * (W + 1) + lane + 32 * j];
#pragma unroll
      for (int i = 0; i < RPT; ++i)
#pragma unroll
        for (int j = 0; j < CPT; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
  }
}

template <int W, int RR = R>
struct Smem {
  static constexpr size_t ws_floats = KC * (W + 1);
  static size_t bytes(int n_act) { return (size_t(n_act) * RR * W + ws_floats + RR * 8) * sizeof(float); }
};

// Forward of slot p for the R rows whose determinants are xs[0..R) (rows
// >= nrows are computed on garbage-free zeros and ignored).  act holds
// n_keep activation buffers [R][W]: with n_keep == L every layer's output is
// kept (for the adjoint), with n_keep == 2 they ping-pong.  Leaves the head
// outputs in out8[R][8] and returns the index of the last hidden buffer.
template <int W, int RR = R>
__device__ int slot_forward(const MlpView& m, int p, const uint64_t* xs, int nrows, float* act, int n_keep,
                            float* ws, float* out8, const float* wres = nullptr) {
  const MlpPtr P = slot_ptrs(m, p);
  for (int idx = threadIdx.x; idx < RR * W; idx += NT) {
    int r = idx / W, o = idx % W;
    float acc = __ldg(P.b1 + o);
    if (r < nrows) {
      uint64_t x = xs[r];
      const float* wrow = P.W1 + size_t(o) * 4 * p;
      for (int q = 0; q < p; ++q) acc += __ldg(wrow + 4 * q + int((x >> (2 * q)) & 3ull));
    }
    act[idx] = tanhf(acc);
  }
  int cur = 0;
  const float* Wk = P.Wk;
  constexpr int RPT = RR / 8, CPT = W / 32;
  const int lane = threadIdx.x & 31, wg = threadIdx.x >> 5;
  for (int k = 2; k <= m.n_hidden; ++k) {
    const float* bk = Wk + size_t(W) * W;
    float acc[RPT][CPT];
    tile_gemm<W, false, RR>(act + size_t(cur) * RR * W, Wk, ws, acc,
                            wres ? wres + size_t(k - 2) * W * (W + 1) : nullptr);
    int nxt = (n_keep == 2) ? (cur ^ 1) : (cur + 1);
    float* o = act + size_t(nxt) * RR * W;
#pragma unroll
    for (int i = 0; i < RPT; ++i)
#pragma unroll
      for (int j = 0; j < CPT; ++j) {
        int c = lane + 32 * j;
        o[(wg * RPT + i) * W + c] = tanhf(acc[i][j] + __ldg(bk + c));
      }
    cur = nxt;
    Wk = bk + W;
  }
  __syncthreads();
  {
    const float* h = act + size_t(cur) * RR * W;
    int r = threadIdx.x >> 3, o = threadIdx.x & 7;
    if (r < RR) {
      float acc = __ldg(P.bh + o);
      const float* wr = P.Wh + size_t(o) * W;
      for (int k = 0; k < W; ++k) acc = fmaf(h[r * W + ((k + r) & (W - 1))], __ldg(wr + ((k + r) & (W - 1))), acc);
      out8[r * 8 + o] = acc;
    }
  }
  __syncthreads();
  return cur;
}

// log-softmax term of the chosen outcome (FP32): normalised over nm, zero
// amplitude (dead) when v is not physical
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

template <int W>
__global__ void __launch_bounds__(NT) logpsi_kernel(MlpView m, HamView hv, const uint64_t* __restrict__ xs,
                                                    Count n_x_, float* __restrict__ la_out,
                                                    float* __restrict__ ph_out) {
  ANQS_PDL_ENTRY();
  const uint64_t n_x = n_x_.get();
  extern __shared__ float smem[];
  float* act = smem;
  float* ws = act + 2 * R * W;
  float* out8 = ws + Smem<W>::ws_floats;
  __shared__ uint64_t xt[R];
  __shared__ float la[R], ph[R];
  __shared__ int ca[R], cb[R], dead[R];
  const uint64_t n_tiles = (n_x + R - 1) / R;
  for (uint64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const uint64_t base = tile * R;
    const int nrows = int(n_x - base < uint64_t(R) ? n_x - base : uint64_t(R));
    if (threadIdx.x < R) {
      xt[threadIdx.x] = threadIdx.x < nrows ? xs[base + threadIdx.x] : 0ull;
      la[threadIdx.x] = 0.f;
      ph[threadIdx.x] = 0.f;
      ca[threadIdx.x] = cb[threadIdx.x] = dead[threadIdx.x] = 0;
    }
    __syncthreads();
    for (int p = 0; p < m.n; ++p) {
      slot_forward<W>(m, p, xt, nrows, act, 2, ws, out8);
      if (threadIdx.x < nrows) {
        int r = threadIdx.x;
        int v = int((xt[r] >> (2 * p)) & 3ull);
        unsigned mk = slot_mask(hv, p, ca[r], cb[r], xt[r]);
        bool dd = dead[r];
        slot_term(out8 + r * 8, norm_mask(hv, p, mk), mk, v, la[r], ph[r], dd);
        dead[r] = dd;
        ca[r] += v & 1;
        cb[r] += v >> 1;
      }
      __syncthreads();
    }
    if (threadIdx.x < nrows) {
      int r = threadIdx.x;
      bool out_of_sector = dead[r] || (hv.n < 32 && (xt[r] >> (2 * hv.n)) != 0);
      la_out[base + r] = out_of_sector ? -INFINITY : la[r];
      ph_out[base + r] = ph[r];
    }
    __syncthreads();
  }
}

template <int W>
__global__ void __launch_bounds__(NT) slot_logits_kernel(MlpView m, int p, const uint64_t* __restrict__ prefixes,
                                                         const uint64_t* __restrict__ n_rows_dev,
                                                         float* __restrict__ out) {
  ANQS_PDL_ENTRY();
  extern __shared__ float smem[];
  float* act = smem;
  float* ws = act + 2 * R * W;
  float* out8 = ws + Smem<W>::ws_floats;
  __shared__ uint64_t xt[R];
  const uint64_t n_rows = *n_rows_dev;
  const uint64_t n_tiles = (n_rows + R - 1) / R;
  for (uint64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const uint64_t base = tile * R;
    const int nrows = int(n_rows - base < uint64_t(R) ? n_rows - base : uint64_t(R));
    if (threadIdx.x < R) xt[threadIdx.x] = threadIdx.x < nrows ? prefixes[base + threadIdx.x] : 0ull;
    __syncthreads();
    slot_forward<W>(m, p, xt, nrows, act, 2, ws, out8);
    int r = threadIdx.x >> 3, o = threadIdx.x & 7;
    if (r < nrows) out[(base + r) * 8 + o] = out8[r * 8 + o];
    __syncthreads();
  }
}

// Adjoint of sum_l [cot_la_l log|psi(x_l)| + cot_ph_l arg psi(x_l)] with
// respect to slot p's parameters, for one tile of rows; partial sums over
// the tile are added to grad with atomics.
// PARTIAL: each (tile, slot) CTA stores its sums, without atomics, into the
// tile's own copy of the gradient (grad + tile * n_params); a second kernel
// adds the copies.  Otherwise the sums go to grad with atomics.
template <int W, bool PARTIAL>
__device__ __forceinline__ void gacc(float* p, float v) {
  if (PARTIAL) *p = v;
  else atomicAdd(p, v);
}

// gW[o][i] (+)= sum_r dz[r][o] h[r][i] over the R rows of the tile, with
// register blocking: a 16 x 16 grid of threads, each owning a block of
// W/16 x W/16 outputs (W = 256 in two column halves), float4 shared loads.
template <int W, bool PARTIAL, int RR>
__device__ __forceinline__ void outer_accumulate(const float* dz, const float* h, float* gW) {
  constexpr int B = (W >= 128) ? 8 : W / 16;  // outputs per thread along o and along i
  constexpr int COLS = 16 * B;                 // columns covered per pass
  const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
  for (int c0 = 0; c0 < W; c0 += COLS) {
    float acc[B][B];
#pragma unroll
    for (int a = 0; a < B; ++a)
#pragma unroll
      for (int b = 0; b < B; ++b) acc[a][b] = 0.f;
    const int o0 = ty * B * (W / (16 * B)), i0 = c0 + tx * B;
    for (int ob = 0; ob < W / (16 * B); ++ob) {
      const int oo = o0 + ob * B;
      if (ob > 0) {
#pragma unroll
        for (int a = 0; a < B; ++a)
#pragma unroll
          for (int b = 0; b < B; ++b) acc[a][b] = 0.f;
      }
#pragma unroll 4
      for (int r = 0; r < RR; ++r) {
        float zo[B], hi[B];
#pragma unroll
        for (int a = 0; a < B; a += 4) {
          const float4 z4 = *reinterpret_cast<const float4*>(dz + r * W + oo + a);
          zo[a] = z4.x;
          zo[a + 1] = z4.y;
          zo[a + 2] = z4.z;
          zo[a + 3] = z4.w;
          const float4 h4 = *reinterpret_cast<const float4*>(h + r * W + i0 + a);
          hi[a] = h4.x;
          hi[a + 1] = h4.y;
          hi[a + 2] = h4.z;
          hi[a + 3] = h4.w;
        }
#pragma unroll
        for (int a = 0; a < B; ++a)
#pragma unroll
          for (int b = 0; b < B; ++b) acc[a][b] = fmaf(zo[a], hi[b], acc[a][b]);
      }
#pragma unroll
      for (int a = 0; a < B; ++a)
#pragma unroll
        for (int b = 0; b < B; ++b) gacc<W, PARTIAL>(gW + size_t(oo + a) * W + i0 + b, acc[a][b]);
    }
  }
}

template <int W, int RG, bool PARTIAL, bool RESIDENT>
__global__ void __launch_bounds__(NT) grad_kernel(MlpView m, HamView hv, const uint64_t* __restrict__ xs,
                                                  Count n_x_, CotSrc cot, float* __restrict__ grad,
                                                  uint64_t n_params) {
  extern __shared__ float smem[];
  const int L = m.n_hidden;
  float* act = smem;                       // L buffers [RG][W]: h_1..h_L
  float* ws = act + size_t(L) * RG * W;     // weight chunk
  float* out8 = ws + Smem<W, RG>::ws_floats;   // head outputs, then their adjoint
  float* dh = out8 + RG * 8;                // [RG][W] adjoint of the current layer output
  __shared__ uint64_t xt[RG];
  __shared__ float cl[RG], cp[RG];
  const int p = blockIdx.y;
  // Prologue, before the wait on the previous kernel: the hidden matrices of
  // slot p into shared memory (row stride W + 1).  No library kernel writes
  // the parameters, so their last update has completed before any library
  // kernel can let this one start; rows, counts and energies are read after
  // the wait.
  float* wres = RESIDENT ? dh + RG * W : nullptr;
  if (RESIDENT) {
    const MlpPtr Pw = slot_ptrs(m, p);
    for (int l = 0; l < L - 1; ++l) {
      const float* src = Pw.Wk + size_t(l) * (size_t(W) * W + W);
      float* dst = wres + size_t(l) * W * (W + 1);
      for (int idx = threadIdx.x; idx < W * W; idx += NT) dst[(idx / W) * (W + 1) + idx % W] = __ldg(src + idx);
    }
  }
  ANQS_PDL_WAIT();
  ANQS_PDL_TRIGGER();
  const uint64_t n_x = n_x_.get();
  const uint64_t base = uint64_t(blockIdx.x) * RG;
  if (base >= n_x) return;
  const int nrows = int(n_x - base < uint64_t(RG) ? n_x - base : uint64_t(RG));
  if (threadIdx.x < RG) {
    bool ok = threadIdx.x < nrows;
    xt[threadIdx.x] = ok ? xs[base + threadIdx.x] : 0ull;
    float a = 0.f, b = 0.f;
    if (ok) cot_of(cot, base + threadIdx.x, a, b);
    cl[threadIdx.x] = a;
    cp[threadIdx.x] = b;
  }
  __syncthreads();
  const int last = slot_forward<W, RG>(m, p, xt, nrows, act, L, ws, out8, wres);
  const MlpPtr P = slot_ptrs(m, p);
  float* gbase = grad + (P.W1 - m.params) + (PARTIAL ? uint64_t(blockIdx.x) * n_params : 0ull);
  // d out: d l_u = cot_la * 1/2 (delta_uv - p~_u) over allowed u, d phi_u = cot_ph delta_uv
  if (threadIdx.x < RG) {
    int r = threadIdx.x;
    float d[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (r < nrows) {
      uint64_t x = xt[r];
      int a = 0, b = 0;
      for (int q = 0; q < p; ++q) {
        int vq = int((x >> (2 * q)) & 3ull);
        a += vq & 1;
        b += vq >> 1;
      }
      const unsigned pm = slot_mask(hv, p, a, b, x), mk = norm_mask(hv, p, pm);
      int v = int((x >> (2 * p)) & 3ull);
      if ((pm >> v) & 1u) {
        const float* o8 = out8 + r * 8;
        float mx = -INFINITY;
        for (int u = 0; u < 4; ++u)
          if ((mk >> u) & 1u) mx = fmaxf(mx, o8[u]);
        float e[4], s = 0.f;
        for (int u = 0; u < 4; ++u) {
          e[u] = ((mk >> u) & 1u) ? expf(o8[u] - mx) : 0.f;
          s += e[u];
        }
        for (int u = 0; u < 4; ++u) d[u] = 0.5f * cl[r] * ((u == v ? 1.f : 0.f) - e[u] / s);
        d[4 + v] = cp[r];
      }
    }
    for (int u = 0; u < 8; ++u) out8[r * 8 + u] = d[u];
  }
  __syncthreads();
  // head: dW_h[o][k] += sum_r d[r][o] h_L[r][k]; db_h[o] += sum_r d[r][o]; dh_L = W_h^T d
  {
    const float* hL = act + size_t(last) * RG * W;
    float* gWh = gbase + (P.Wh - P.W1);
    float* gbh = gbase + (P.bh - P.W1);
    for (int idx = threadIdx.x; idx < 8 * W; idx += NT) {
      int o = idx / W, k = idx % W;
      float s = 0.f;
      for (int r = 0; r < RG; ++r) s = fmaf(out8[r * 8 + o], hL[r * W + k], s);
      gacc<W, PARTIAL>(gWh + idx, s);
    }
    if (threadIdx.x < 8) {
      float s = 0.f;
      for (int r = 0; r < RG; ++r) s += out8[r * 8 + threadIdx.x];
      gacc<W, PARTIAL>(gbh + threadIdx.x, s);
    }
    for (int idx = threadIdx.x; idx < RG * W; idx += NT) {
      int r = idx / W, k = idx % W;
      float s = 0.f;
      for (int o = 0; o < 8; ++o) s = fmaf(__ldg(P.Wh + o * W + k), out8[r * 8 + o], s);
      // through tanh: dz = dh (1 - h^2)
      float hv_ = hL[idx];
      dh[idx] = s * (1.f - hv_ * hv_);
    }
  }
  __syncthreads();
  // hidden layers L..2 (dh holds dz_k of layer k)
  constexpr int RPT = RG / 8, CPT = W / 32;
  const int lane = threadIdx.x & 31, wg = threadIdx.x >> 5;
  for (int k = L; k >= 2; --k) {
    const float* Wk = P.Wk + size_t(k - 2) * (size_t(W) * W + W);
    float* gW = gbase + (Wk - P.W1);
    float* gb = gW + size_t(W) * W;
    const float* hprev = act + size_t(k - 2) * RG * W;  // h_{k-1}
    outer_accumulate<W, PARTIAL, RG>(dh, hprev, gW);
    for (int o = threadIdx.x; o < W; o += NT) {
      float s = 0.f;
      for (int r = 0; r < RG; ++r) s += dh[r * W + o];
      gacc<W, PARTIAL>(gb + o, s);
    }
    float acc[RPT][CPT];
    tile_gemm<W, true, RG>(dh, Wk, ws, acc, RESIDENT ? wres + size_t(k - 2) * W * (W + 1) : nullptr);  // W_k^T dz_k
    __syncthreads();
#pragma unroll
    for (int i = 0; i < RPT; ++i)
#pragma unroll
      for (int j = 0; j < CPT; ++j) {
        int r = wg * RPT + i, c = lane + 32 * j;
        float hv_ = hprev[r * W + c];
        dh[r * W + c] = acc[i][j] * (1.f - hv_ * hv_);
      }
    __syncthreads();
  }
  // layer 1: dW_1[o][4q + v_q] += sum_r dz_1[r][o]; db_1 += sum_r dz_1
  {
    float* gW1 = gbase;
    float* gb1 = gbase + size_t(W) * 4 * p;
    for (int o = threadIdx.x; o < W; o += NT) {
      float s = 0.f;
      for (int r = 0; r < nrows; ++r) s += dh[r * W + o];
      gacc<W, PARTIAL>(gb1 + o, s);
      for (int q = 0; q < p; ++q) {
        float c4[4] = {0.f, 0.f, 0.f, 0.f};
        for (int r = 0; r < nrows; ++r) c4[int((xt[r] >> (2 * q)) & 3ull)] += dh[r * W + o];
        for (int u = 0; u < 4; ++u)
          if (PARTIAL || c4[u] != 0.f) gacc<W, PARTIAL>(gW1 + size_t(o) * 4 * p + 4 * q + u, c4[u]);
      }
    }
  }
}

// grad[i] = sum over the tiles of the per-tile copies (only tiles holding rows)
__global__ void partial_sum_kernel(const float* __restrict__ part, Count n_x_, uint64_t n_params, int rg,
                                   float* __restrict__ grad) {
  ANQS_PDL_ENTRY();
  const uint64_t tiles = (n_x_.get() + rg - 1) / rg;
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < n_params;
       i += uint64_t(gridDim.x) * blockDim.x) {
    // four tiles' loads in flight at a time, added in tile order
    float s = 0.f;
    uint64_t t = 0;
    for (; t + 4 <= tiles; t += 4) {
      const float a0 = part[t * n_params + i], a1 = part[(t + 1) * n_params + i],
                  a2 = part[(t + 2) * n_params + i], a3 = part[(t + 3) * n_params + i];
      s += a0;
      s += a1;
      s += a2;
      s += a3;
    }
    for (; t < tiles; ++t) s += part[t * n_params + i];
    grad[i] = s;
  }
}

// the smallest tile height (16, 24 or 32 rows) whose tiles of all slots fit
// in one wave of (one per SM) CTAs, else 32
int rg_for(const MlpView& m, uint64_t n_x) {
  for (int rg : {16, 24})
    if (((n_x + rg - 1) / rg) * uint64_t(m.n) <= 152) return rg;
  return 32;
}

template <class F>
int set_smem(F* f, size_t bytes) {
  ANQS_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes)));
  return ANQS_OK;
}

unsigned grid_for(uint64_t tiles, unsigned cap) { return unsigned(tiles < cap ? (tiles ? tiles : 1) : cap); }

template <int W>
int logpsi_w(const MlpView& m, const HamView& hv, const uint64_t* x, Count n_x, float* la, float* ph,
             cudaStream_t s) {
  size_t sm = Smem<W>::bytes(2);
  ANQS_TRY(set_smem(logpsi_kernel<W>, sm));
  ProfScope ps(PROF_MLP_FP32_LOGPSI, s);
  ANQS_CUDA_LAUNCH("mlp logpsi_kernel", launch_k(logpsi_kernel<W>, dim3(grid_for((n_x.n + R - 1) / R, 152 * 8)), dim3(NT), sm, s, m, hv, x, n_x, la, ph));
  return ANQS_OK;
}

template <int W>
int logits_w(const MlpView& m, int p, const uint64_t* pre, const uint64_t* nr, uint64_t max_rows, float* out,
             cudaStream_t s) {
  size_t sm = Smem<W>::bytes(2);
  ANQS_TRY(set_smem(slot_logits_kernel<W>, sm));
  ProfScope ps(PROF_MLP_FP32_SLOT, s);
  ANQS_CUDA_LAUNCH("mlp slot_logits_kernel", launch_k(slot_logits_kernel<W>, dim3(grid_for((max_rows + R - 1) / R, 152 * 8)), dim3(NT), sm, s, m, p, pre, nr, out));
  return ANQS_OK;
}

template <int W, int RG, bool RES>
int grad_launch(const MlpView& m, const HamView& hv, const uint64_t* x, Count n_x, const CotSrc& cot, float* g,
                float* part, uint64_t n_params, size_t sm, cudaStream_t s) {
  dim3 grid(unsigned(std::max<uint64_t>((n_x.n + RG - 1) / RG, 1)), unsigned(m.n));
  if (part) {
    ANQS_TRY(set_smem(grad_kernel<W, RG, true, RES>, sm));
    {
      ProfScope ps(PROF_MLP_FP32_GRAD, s);
      ANQS_CUDA_LAUNCH("mlp grad_kernel", launch_k(grad_kernel<W, RG, true, RES>, dim3(grid), dim3(NT), sm, s, m, hv,
                                                   x, n_x, cot, part, n_params));
    }
    ProfScope ps(PROF_GRAD_REDUCE, s);
    ANQS_CUDA_LAUNCH("mlp partial_sum_kernel",
                     launch_k(partial_sum_kernel, dim3(unsigned(std::min<uint64_t>((n_params + 255) / 256, 152 * 8))),
                              dim3(256), 0, s, part, n_x, n_params, RG, g));
  } else {
    ANQS_TRY(set_smem(grad_kernel<W, RG, false, RES>, sm));
    ProfScope ps(PROF_MLP_FP32_GRAD, s);
    ANQS_CUDA_LAUNCH("mlp grad_kernel", launch_k(grad_kernel<W, RG, false, RES>, dim3(grid), dim3(NT), sm, s, m, hv,
                                                 x, n_x, cot, g, n_params));
  }
  return ANQS_OK;
}

// The slot's hidden matrices stay in shared memory when they fit next to the
// activations (widths 64 and 128); otherwise they stream in chunks.
template <int W, int RG>
int grad_rg(const MlpView& m, const HamView& hv, const uint64_t* x, Count n_x, const CotSrc& cot, float* g,
            float* part, uint64_t n_params, cudaStream_t s) {
  const size_t sm = Smem<W, RG>::bytes(m.n_hidden + 1);
  const size_t res = sm + size_t(m.n_hidden - 1) * W * (W + 1) * sizeof(float);
  if (res <= 227 * 1024) return grad_launch<W, RG, true>(m, hv, x, n_x, cot, g, part, n_params, res, s);
  if (sm > 227 * 1024)
    return set_error(ANQS_ERR_UNSUPPORTED, "FP32 MLP adjoint needs %zu bytes of shared memory", sm);
  return grad_launch<W, RG, false>(m, hv, x, n_x, cot, g, part, n_params, sm, s);
}

template <int W>
int grad_w(const MlpView& m, const HamView& hv, const uint64_t* x, Count n_x, const CotSrc& cot, float* g,
           float* part, uint64_t n_params, cudaStream_t s) {
  switch (rg_for(m, n_x.n)) {
    case 16: return grad_rg<W, 16>(m, hv, x, n_x, cot, g, part, n_params, s);
    case 24: return grad_rg<W, 24>(m, hv, x, n_x, cot, g, part, n_params, s);
  }
  return grad_rg<W, 32>(m, hv, x, n_x, cot, g, part, n_params, s);
}

}  // namespace

int launch_mlp_fp32_logpsi(const MlpView& m, const HamView& hv, const uint64_t* x, Count n_x, float* la,
                           float* ph, cudaStream_t s) {
  switch (m.width) {
    case 64: return logpsi_w<64>(m, hv, x, n_x, la, ph, s);
    case 128: return logpsi_w<128>(m, hv, x, n_x, la, ph, s);
    case 256: return logpsi_w<256>(m, hv, x, n_x, la, ph, s);
  }
  return set_error(ANQS_ERR_UNSUPPORTED, "width %d", m.width);
}

int launch_mlp_fp32_slot_logits(const MlpView& m, int p, const uint64_t* pre, const uint64_t* nr,
                                uint64_t max_rows, float* out, cudaStream_t s) {
  switch (m.width) {
    case 64: return logits_w<64>(m, p, pre, nr, max_rows, out, s);
    case 128: return logits_w<128>(m, p, pre, nr, max_rows, out, s);
    case 256: return logits_w<256>(m, p, pre, nr, max_rows, out, s);
  }
  return set_error(ANQS_ERR_UNSUPPORTED, "width %d", m.width);
}

int launch_grad_partial_sum(const float* part, Count n_x, uint64_t n_params, int rows_per_tile, float* g,
                            cudaStream_t s) {
  ProfScope ps(PROF_GRAD_REDUCE, s);
  ANQS_CUDA_LAUNCH("mlp partial_sum_kernel",
                   launch_k(partial_sum_kernel, dim3(unsigned(std::min<uint64_t>((n_params + 255) / 256, 152 * 8))),
                            dim3(256), 0, s, part, n_x, n_params, rows_per_tile, g));
  return ANQS_OK;
}

size_t mlp_fp32_grad_partial_floats(const MlpView& m, uint64_t n_x) {
  const int rg = rg_for(m, n_x);
  return size_t((n_x + rg - 1) / rg) * m.slot_off[m.n];
}

int launch_mlp_fp32_grad(const MlpView& m, const HamView& hv, const uint64_t* x, Count n_x, const CotSrc& cot,
                         float* g, float* part, cudaStream_t s) {
  if ((n_x.n + 15) / 16 > 0x7fffffffull) return set_error(ANQS_ERR_UNSUPPORTED, "too many rows");
  const uint64_t np = m.slot_off[m.n];
  switch (m.width) {
    case 64: return grad_w<64>(m, hv, x, n_x, cot, g, part, np, s);
    case 128: return grad_w<128>(m, hv, x, n_x, cot, g, part, np, s);
    case 256: return grad_w<256>(m, hv, x, n_x, cot, g, part, np, s);
  }
  return set_error(ANQS_ERR_UNSUPPORTED, "width %d", m.width);
}

}  // namespace anqs
