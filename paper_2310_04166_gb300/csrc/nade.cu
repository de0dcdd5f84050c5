// FP32 form of the paper's own ansatz, the per-qubit complex NADE of
// Appendix B.1: qubit i (0-based, i = 0..2n-1) has a complex MLP reading the
// i previous bits, z1 = W1 x_<i + b1, h1 = tanh z1 (complex), z2 = W2 h1 + b2,
// h2 = LeReLU(Re z2) + i LeReLU(Im z2) (leaky ReLU, 0.01 x below zero), z3 =
// W3 h2 + b3 (2 outputs) and f3(z) = z - 1/2 LSE(2 Re z): log psi_i(x_i | x_<i)
// = f3(z3)_{x_i}.
//
// Slot p groups qubits 2p (alpha) and 2p+1 (beta): psi_slot(a + 2b) =
// psi_2p(a) psi_2p+1(b | a), so qubit 2p's network runs once and qubit 2p+1's
// twice (a = 0, 1) per prefix.  MU masking (Sec. III.C) acts on each binary
// conditional: qubit 2p's allowed values are the a with an allowed (a, b) in
// the slot mask, qubit 2p+1's the b with (a, b) allowed; the modulus is
// renormalised over them, the phases kept; DU slots of an MU-d strategy mask
// nothing.  The slot's 8 values l_v = log |psi_slot(v)|^2, phi_v =
// arg psi_slot(v) are already a normalised distribution, so the slot-level
// machinery (masked log-softmax, sampler, local energy) applies unchanged.
//
// A CTA of 256 threads holds 256 / W rows; thread (r, u) owns hidden unit u of
// row r (complex values in shared memory between the layers).
#include <cmath>

#include "common.cuh"

namespace anqs {
namespace {

constexpr int NT = 256;
enum { NADE_LOGPSI = 0, NADE_LOGITS = 1 };

// tanh(a + ib) = (sinh a cosh a + i sin b cos b) / (sinh^2 a + cos^2 b), for
// z = (ah + al) + i (bh + bl) given as float-float pairs.  The denominator
// is a sum of squares (no cancellation), and it vanishes at the poles
// z = i pi (k + 1/2) where tanh is ill-conditioned; the low parts enter
// through first-order corrections of sinh a, cosh a, sin b and cos b, so that
// near a pole the result is not spoiled by the rounding of z to float.  For
// |a| > 9, tanh z = sign(a) + i sin 2b * 2 e^{-2|a|} to float precision.
__device__ __forceinline__ float2 ctanh(float ah, float al, float bh, float bl) {
  if (fabsf(ah) > 9.f) return make_float2(copysignf(1.f, ah), 2.f * sinf(2.f * bh) * expf(-2.f * fabsf(ah)));
  float sa = sinhf(ah);
  float ca = sqrtf(1.f + sa * sa);
  float sb, cb;
  sincosf(bh, &sb, &cb);
  const float sa1 = fmaf(ca, al, sa), ca1 = fmaf(sa, al, ca);
  const float sb1 = fmaf(cb, bl, sb), cb1 = fmaf(-sb, bl, cb);
  const float den = fmaf(sa1, sa1, cb1 * cb1);
  return make_float2(sa1 * ca1 / den, sb1 * cb1 / den);
}

// s + e = a + b exactly (Knuth's TwoSum)
__device__ __forceinline__ float two_sum(float a, float b, float& e) {
  const float s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
  return s;
}

__device__ __forceinline__ float lerelu(float x) { return x >= 0.f ? x : 0.01f * x; }

struct QubitPtr {
  const float2 *W1, *b1, *W2, *b2, *W3, *b3;
};

__device__ __forceinline__ QubitPtr qubit_ptrs(const NadeView& m, int i) {
  const int w = m.w;
  QubitPtr q;
  q.W1 = reinterpret_cast<const float2*>(m.params + m.qoff[i]);
  q.b1 = q.W1 + size_t(w) * i;
  q.W2 = q.b1 + w;
  q.b2 = q.W2 + size_t(w) * w;
  q.W3 = q.b2 + w;
  q.b3 = q.W3 + 2 * w;
  return q;
}

__device__ __forceinline__ float2 cmul(float2 x, float2 y) { return make_float2(x.x * y.x - x.y * y.y, x.x * y.y + x.y * y.x); }

// Qubit i's network for the R rows of the tile: bits k < i of row r are the
// bits of x[r] below bit min(i, 2p), and bit 2p (when i = 2p + 1) is `a`.
// Writes f3(z3) (unmasked log psi_i(0), log psi_i(1)) to lq[r][0..1].
template <int W>
__device__ void qubit_forward(const NadeView& m, int i, int p, int a, const uint64_t* xs, float2* h1, float2* h2,
                              float2* lq) {
  const int r = threadIdx.x / W, u = threadIdx.x % W;
  const QubitPtr q = qubit_ptrs(m, i);
  const uint64_t x = xs[r];
  // z1 as a float-float pair: the sum of the selected W1 columns is exact to
  // about u^2, which matters only next to a pole of tanh
  float2 z = __ldg(q.b1 + u), lo = make_float2(0.f, 0.f);
  for (int k = 0; k < i; ++k) {
    const int bit = k < 2 * p ? int((x >> k) & 1ull) : a;
    if (bit) {
      const float2 wv = __ldg(q.W1 + size_t(u) * i + k);
      float ex, ey;
      z.x = two_sum(z.x, wv.x, ex);
      z.y = two_sum(z.y, wv.y, ey);
      lo.x += ex;
      lo.y += ey;
    }
  }
  h1[r * W + u] = ctanh(z.x, lo.x, z.y, lo.y);
  __syncthreads();
  z = __ldg(q.b2 + u);
  for (int k = 0; k < W; ++k) {
    const float2 t = cmul(__ldg(q.W2 + size_t(u) * W + k), h1[r * W + k]);
    z.x += t.x;
    z.y += t.y;
  }
  h2[r * W + u] = make_float2(lerelu(z.x), lerelu(z.y));
  __syncthreads();
  if (u < 2) {
    z = __ldg(q.b3 + u);
    for (int k = 0; k < W; ++k) {
      const float2 t = cmul(__ldg(q.W3 + size_t(u) * W + k), h2[r * W + k]);
      z.x += t.x;
      z.y += t.y;
    }
    lq[r * 2 + u] = z;
  }
  __syncthreads();
  if (u == 0) {  // f3: log-normalise the two outputs
    const float2 z0 = lq[r * 2], z1 = lq[r * 2 + 1];
    const float mx = fmaxf(2.f * z0.x, 2.f * z1.x);
    const float lse = 0.5f * (mx + logf(expf(2.f * z0.x - mx) + expf(2.f * z1.x - mx)));
    lq[r * 2] = make_float2(z0.x - lse, z0.y);
    lq[r * 2 + 1] = make_float2(z1.x - lse, z1.y);
  }
  __syncthreads();
}

// renormalise the modulus of a binary conditional over the allowed values
__device__ __forceinline__ void mask2(float2& l0, float2& l1, unsigned allowed) {
  const float r0 = (allowed & 1u) ? l0.x : -INFINITY;
  const float r1 = (allowed & 2u) ? l1.x : -INFINITY;
  const float mx = fmaxf(r0, r1);
  float lse = 0.f;
  if (mx > -INFINITY) lse = mx + 0.5f * logf(expf(2.f * (r0 - mx)) + expf(2.f * (r1 - mx)));
  l0.x = r0 - lse;
  l1.x = r1 - lse;
}

// prefix (slots < p) electron counts and the slot mask of row x
__device__ __forceinline__ unsigned prefix_mask(const HamView& hv, int p, uint64_t x) {
  const uint64_t pm = (1ull << (2 * p)) - 1ull;  // p < 32
  return slot_mask(hv, p, __popcll(x & pm & 0x5555555555555555ull), __popcll(x & pm & 0xAAAAAAAAAAAAAAAAull), x);
}

// The 8 slot values of slot p for the tile's rows (into o8[r][8]).
template <int W>
__device__ void nade_slot(const NadeView& m, const HamView& hv, int p, const uint64_t* xs, float2* h1, float2* h2,
                          float2* lq, float* o8) {
  constexpr int R = NT / W;
  float2* lq0 = lq;          // [R][2]
  float2* lq1 = lq + 2 * R;  // [2][R][2]: a = 0, 1
  qubit_forward<W>(m, 2 * p, p, 0, xs, h1, h2, lq0);
  qubit_forward<W>(m, 2 * p + 1, p, 0, xs, h1, h2, lq1);
  qubit_forward<W>(m, 2 * p + 1, p, 1, xs, h1, h2, lq1 + 2 * R);
  if (threadIdx.x < R) {
    const int r = threadIdx.x;
    const unsigned pm = prefix_mask(hv, p, xs[r]);
    float2 a0 = lq0[r * 2], a1 = lq0[r * 2 + 1];                  // qubit 2p: a = 0, 1
    float2 b00 = lq1[r * 2], b01 = lq1[r * 2 + 1];                // qubit 2p+1 given a = 0: b = 0, 1
    float2 b10 = lq1[2 * R + r * 2], b11 = lq1[2 * R + r * 2 + 1];  // given a = 1
    if (p < hv.mu_lv) {
      // v = a + 2b: a allowed if (a, 0) or (a, 1) is; b given a if (a, b) is
      mask2(a0, a1, ((pm | (pm >> 2)) & 1u) | (((pm >> 1) | (pm >> 3)) & 1u) << 1);
      mask2(b00, b01, (pm & 1u) | ((pm >> 2) & 1u) << 1);
      mask2(b10, b11, ((pm >> 1) & 1u) | ((pm >> 3) & 1u) << 1);
    }
    const float2 t[4] = {make_float2(a0.x + b00.x, a0.y + b00.y), make_float2(a1.x + b10.x, a1.y + b10.y),
                         make_float2(a0.x + b01.x, a0.y + b01.y), make_float2(a1.x + b11.x, a1.y + b11.y)};
    for (int v = 0; v < 4; ++v) {
      o8[r * 8 + v] = 2.f * t[v].x;
      o8[r * 8 + 4 + v] = t[v].y;
    }
  }
  __syncthreads();
}

// NADE_LOGPSI: log psi of rows x (masked log-softmax over each slot's
// normalising set, -inf outside the sector); NADE_LOGITS: the 8 values of
// slot p for the sampler's prefixes.
template <int W>
__global__ void __launch_bounds__(NT) nade_kernel(NadeView m, HamView hv, const uint64_t* __restrict__ xs, Count rows_,
                                                  int mode, int p_one, float* __restrict__ la_out,
                                                  float* __restrict__ ph_out, float* __restrict__ out8) {
  ANQS_PDL_ENTRY();
  constexpr int R = NT / W;
  __shared__ float2 h1[R * W], h2[R * W], lq[6 * R];
  __shared__ float o8[R * 8];
  __shared__ uint64_t xt[R];
  const uint64_t rows = rows_.get();
  for (uint64_t base = uint64_t(blockIdx.x) * R; base < rows; base += uint64_t(gridDim.x) * R) {
    if (threadIdx.x < R) xt[threadIdx.x] = base + threadIdx.x < rows ? xs[base + threadIdx.x] : 0ull;
    __syncthreads();
    if (mode == NADE_LOGITS) {
      nade_slot<W>(m, hv, p_one, xt, h1, h2, lq, o8);
      if (threadIdx.x < R * 8 && base + threadIdx.x / 8 < rows) out8[base * 8 + threadIdx.x] = o8[threadIdx.x];
      __syncthreads();
      continue;
    }
    float la = 0.f, ph = 0.f;
    bool dead = false;
    for (int p = 0; p < m.n; ++p) {
      nade_slot<W>(m, hv, p, xt, h1, h2, lq, o8);
      if (threadIdx.x < R) {
        const uint64_t x = xt[threadIdx.x];
        const unsigned pm = prefix_mask(hv, p, x);
        const unsigned nm = norm_mask(hv, p, pm);
        const int v = int((x >> (2 * p)) & 3ull);
        const float* o = o8 + threadIdx.x * 8;
        if (!((pm >> v) & 1u)) {
          dead = true;
        } else {
          float mx = -INFINITY;
          for (int u = 0; u < 4; ++u)
            if ((nm >> u) & 1u) mx = fmaxf(mx, o[u]);
          float s = 0.f;
          for (int u = 0; u < 4; ++u)
            if ((nm >> u) & 1u) s += expf(o[u] - mx);
          la += 0.5f * (o[v] - mx - logf(s));
        }
        ph += o[4 + v];
      }
      __syncthreads();
    }
    if (threadIdx.x < R && base + threadIdx.x < rows) {
      const uint64_t x = xt[threadIdx.x];
      const bool out = dead || (hv.n < 32 && (x >> (2 * hv.n)) != 0);
      la_out[base + threadIdx.x] = out ? -INFINITY : la;
      ph_out[base + threadIdx.x] = ph;
    }
    __syncthreads();
  }
}

template <int W>
int launch_w(const NadeView& m, const HamView& hv, const uint64_t* x, Count rows, int mode, int p, float* la,
             float* ph, float* out8, cudaStream_t s) {
  constexpr int R = NT / W;
  uint64_t blocks = (rows.n + R - 1) / R;
  if (blocks > 152ull * 8) blocks = 152ull * 8;
  ProfScope ps(PROF_NADE, s);
  ANQS_CUDA_LAUNCH("nade_kernel", launch_k(nade_kernel<W>, dim3(unsigned(blocks ? blocks : 1)), dim3(NT), 0, s, m, hv,
                                           x, rows, mode, p, la, ph, out8));
  return ANQS_OK;
}

int launch(const NadeView& m, const HamView& hv, const uint64_t* x, Count rows, int mode, int p, float* la, float* ph,
           float* out8, cudaStream_t s) {
  switch (m.w) {
    case 32: return launch_w<32>(m, hv, x, rows, mode, p, la, ph, out8, s);
    case 64: return launch_w<64>(m, hv, x, rows, mode, p, la, ph, out8, s);
    case 128: return launch_w<128>(m, hv, x, rows, mode, p, la, ph, out8, s);
  }
  return set_error(ANQS_ERR_UNSUPPORTED, "NADE width %d", m.w);
}

}  // namespace

int launch_nade_logpsi(const NadeView& m, const HamView& hv, const uint64_t* x, Count n_x, float* la, float* ph,
                       cudaStream_t s) {
  if (n_x.n == 0) return ANQS_OK;
  return launch(m, hv, x, n_x, NADE_LOGPSI, 0, la, ph, nullptr, s);
}

int launch_nade_slot_logits(const NadeView& m, const HamView& hv, int p, const uint64_t* pre, const uint64_t* n_dev,
                            uint64_t max_rows, float* out8, cudaStream_t s) {
  return launch(m, hv, pre, Count{max_rows, n_dev, 1}, NADE_LOGITS, p, nullptr, nullptr, out8, s);
}

// ---------------------------------------------------------------------------
// Adjoint (vector-Jacobian product of the masked log psi).
//
// The masked NADE is normalised slot by slot on MU and DU levels alike, so the
// slot log-softmax of the forward is identically zero and
// log psi(x) = sum_i [Re z3_i(x_i) - LSE_{A_i}(2 Re z3_i) / 2 + i Im z3_i(x_i)],
// with A_i qubit i's allowed values on the path x (both values on DU slots).
// Only the branch a = x_2p of qubit 2p+1 enters.  For L = cl la + cp ph the
// gradient of the complex output z3_i(k), as (dL/dRe, dL/dIm), is
// (cl (delta_k,x_i - pi_k), cp delta_k,x_i) with pi the softmax of 2 Re z3 over
// A_i; it is pulled back through the complex layers (W^H g for a linear map,
// conj(1 - h1^2) g for tanh, the 1 / 0.01 slope per part for LeReLU) and the
// parameter gradients are g conj(input) (the real bits for W1).
//
// CTA (g, i) handles qubit i for the row tiles g, g + G, ... and accumulates
// qubit i's whole parameter block in shared memory (each entry owned by one
// thread, rows in tile order: deterministic); with G > 1 the blocks go to a
// per-g partial buffer that a second kernel sums in a fixed order.
// ---------------------------------------------------------------------------
namespace {

__host__ __device__ inline uint32_t qubit_floats(uint32_t w, uint32_t i) { return 2u * (w * i + w + w * w + w + 2u * w + 2u); }

template <int W>
__global__ void __launch_bounds__(NT) nade_grad_kernel(NadeView m, HamView hv, const uint64_t* __restrict__ xs,
                                                       Count rows_, const float* __restrict__ cl,
                                                       const float* __restrict__ cp, float* __restrict__ out,
                                                       uint64_t out_stride) {
  ANQS_PDL_ENTRY();
  constexpr int R = NT / W;
  extern __shared__ float2 acc[];  // qubit i's parameter block (complex entries)
  __shared__ float2 h1[R * W], h2[R * W], gz1[R * W], gz2[R * W], z3[R * 2], g3[R * 2];
  __shared__ uint64_t xt[R];
  const int i = blockIdx.y, p = i >> 1, sigma = i & 1;
  const int r = threadIdx.x / W, u = threadIdx.x % W;
  const uint32_t nc = qubit_floats(W, i) / 2;  // complex entries of the block
  const uint32_t oW1 = 0, ob1 = W * i, oW2 = ob1 + W, ob2 = oW2 + W * W, oW3 = ob2 + W, ob3 = oW3 + 2 * W;
  for (uint32_t e = threadIdx.x; e < nc; e += NT) acc[e] = make_float2(0.f, 0.f);
  const QubitPtr q = qubit_ptrs(m, i);
  const uint64_t rows = rows_.get();
  for (uint64_t base = uint64_t(blockIdx.x) * R; base < rows; base += uint64_t(gridDim.x) * R) {
    if (threadIdx.x < R) xt[threadIdx.x] = base + threadIdx.x < rows ? xs[base + threadIdx.x] : 0ull;
    __syncthreads();
    const uint64_t x = xt[r];
    // forward of qubit i on the path (bits x_<i of row r)
    float2 z = __ldg(q.b1 + u), lo = make_float2(0.f, 0.f);
    for (int k = 0; k < i; ++k) {
      if ((x >> k) & 1ull) {
        const float2 wv = __ldg(q.W1 + size_t(u) * i + k);
        float ex, ey;
        z.x = two_sum(z.x, wv.x, ex);
        z.y = two_sum(z.y, wv.y, ey);
        lo.x += ex;
        lo.y += ey;
      }
    }
    h1[r * W + u] = ctanh(z.x, lo.x, z.y, lo.y);
    __syncthreads();
    z = __ldg(q.b2 + u);
    for (int k = 0; k < W; ++k) {
      const float2 t = cmul(__ldg(q.W2 + size_t(u) * W + k), h1[r * W + k]);
      z.x += t.x;
      z.y += t.y;
    }
    h2[r * W + u] = make_float2(lerelu(z.x), lerelu(z.y));
    __syncthreads();
    if (u < 2) {
      z = __ldg(q.b3 + u);
      for (int k = 0; k < W; ++k) {
        const float2 t = cmul(__ldg(q.W3 + size_t(u) * W + k), h2[r * W + k]);
        z.x += t.x;
        z.y += t.y;
      }
      z3[r * 2 + u] = z;
    }
    __syncthreads();
    if (u == 0) {  // cotangent of z3: allowed values of qubit i on the path, softmax of 2 Re z3 over them
      unsigned allowed = 3u;
      if (p < hv.mu_lv) {
        const unsigned pm = prefix_mask(hv, p, x);
        if (sigma == 0) {
          allowed = ((pm | (pm >> 2)) & 1u) | (((pm >> 1) | (pm >> 3)) & 1u) << 1;
        } else {
          const int a = int((x >> (2 * p)) & 1ull);
          allowed = ((pm >> a) & 1u) | ((pm >> (a + 2)) & 1u) << 1;
        }
      }
      const int xi = int((x >> i) & 1ull);
      float2 g0 = make_float2(0.f, 0.f), g1 = g0;
      if (base + r < rows && ((allowed >> xi) & 1u)) {
        const float r0 = (allowed & 1u) ? 2.f * z3[r * 2].x : -INFINITY;
        const float r1 = (allowed & 2u) ? 2.f * z3[r * 2 + 1].x : -INFINITY;
        const float mx = fmaxf(r0, r1);
        const float e0 = expf(r0 - mx), e1 = expf(r1 - mx);
        const float pi0 = e0 / (e0 + e1), pi1 = e1 / (e0 + e1);
        const float c_l = cl[base + r], c_p = cp[base + r];
        g0 = make_float2(c_l * ((xi == 0 ? 1.f : 0.f) - pi0), xi == 0 ? c_p : 0.f);
        g1 = make_float2(c_l * ((xi == 1 ? 1.f : 0.f) - pi1), xi == 1 ? c_p : 0.f);
      }
      g3[r * 2] = g0;
      g3[r * 2 + 1] = g1;
    }
    __syncthreads();
    {  // z2 cotangent: conj(W3)^T g3, then the LeReLU slope of each part (sign of h2 = sign of z2)
      const float2 w0 = __ldg(q.W3 + u), w1 = __ldg(q.W3 + W + u);
      const float2 ga = g3[r * 2], gb = g3[r * 2 + 1];
      const float gr = w0.x * ga.x + w0.y * ga.y + w1.x * gb.x + w1.y * gb.y;
      const float gi = w0.x * ga.y - w0.y * ga.x + w1.x * gb.y - w1.y * gb.x;
      const float2 hh = h2[r * W + u];
      gz2[r * W + u] = make_float2(hh.x >= 0.f ? gr : 0.01f * gr, hh.y >= 0.f ? gi : 0.01f * gi);
    }
    __syncthreads();
    {  // z1 cotangent: conj(W2)^T gz2, then tanh: conj(1 - h1^2) g
      float gr = 0.f, gi = 0.f;
      for (int j = 0; j < W; ++j) {
        const float2 w = __ldg(q.W2 + size_t(j) * W + u);
        const float2 g = gz2[r * W + j];
        gr += w.x * g.x + w.y * g.y;
        gi += w.x * g.y - w.y * g.x;
      }
      const float2 h = h1[r * W + u];
      const float dr = 1.f - (h.x * h.x - h.y * h.y), di = -2.f * h.x * h.y;
      gz1[r * W + u] = make_float2(dr * gr + di * gi, dr * gi - di * gr);
    }
    __syncthreads();
    // parameter gradients of the tile's rows: g conj(input) per weight, g per bias
    for (uint32_t e = threadIdx.x; e < nc; e += NT) {
      float2 s = acc[e];
      if (e < ob1) {  // W1[v][k]: real input bits
        const uint32_t v = e / uint32_t(i), k = e % uint32_t(i);
        for (int rr = 0; rr < R; ++rr)
          if ((xt[rr] >> k) & 1ull) {
            s.x += gz1[rr * W + v].x;
            s.y += gz1[rr * W + v].y;
          }
      } else if (e < oW2) {  // b1
        for (int rr = 0; rr < R; ++rr) {
          s.x += gz1[rr * W + (e - ob1)].x;
          s.y += gz1[rr * W + (e - ob1)].y;
        }
      } else if (e < ob2) {  // W2[v][k]
        const uint32_t v = (e - oW2) / W, k = (e - oW2) % W;
        for (int rr = 0; rr < R; ++rr) {
          const float2 g = gz2[rr * W + v], h = h1[rr * W + k];
          s.x += g.x * h.x + g.y * h.y;
          s.y += g.y * h.x - g.x * h.y;
        }
      } else if (e < oW3) {  // b2
        for (int rr = 0; rr < R; ++rr) {
          s.x += gz2[rr * W + (e - ob2)].x;
          s.y += gz2[rr * W + (e - ob2)].y;
        }
      } else if (e < ob3) {  // W3[k][j]
        const uint32_t k = (e - oW3) / W, j = (e - oW3) % W;
        for (int rr = 0; rr < R; ++rr) {
          const float2 g = g3[rr * 2 + k], h = h2[rr * W + j];
          s.x += g.x * h.x + g.y * h.y;
          s.y += g.y * h.x - g.x * h.y;
        }
      } else {  // b3
        for (int rr = 0; rr < R; ++rr) {
          s.x += g3[rr * 2 + (e - ob3)].x;
          s.y += g3[rr * 2 + (e - ob3)].y;
        }
      }
      acc[e] = s;
    }
    __syncthreads();
  }
  (void)oW1;
  float2* o = reinterpret_cast<float2*>(out + blockIdx.x * out_stride + m.qoff[i]);
  for (uint32_t e = threadIdx.x; e < nc; e += NT) o[e] = acc[e];
}

__global__ void nade_partial_sum_kernel(const float* __restrict__ part, int G, uint64_t n, float* __restrict__ grad) {
  ANQS_PDL_ENTRY();
  for (uint64_t j = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < n; j += uint64_t(gridDim.x) * blockDim.x) {
    float s = 0.f;
    for (int g = 0; g < G; ++g) s += part[uint64_t(g) * n + j];
    grad[j] = s;
  }
}

// CTAs per qubit: about two CTAs per SM over all 2n qubits, at most one per row tile
int grad_groups(const NadeView& m, uint64_t n_x) {
  const uint64_t tiles = (n_x + (NT / m.w) - 1) / (NT / m.w);
  uint64_t g = (2 * 152) / uint64_t(2 * m.n);
  if (g < 1) g = 1;
  if (g > tiles) g = tiles;
  return int(g < 1 ? 1 : g);
}

template <int W>
int grad_w(const NadeView& m, const HamView& hv, const uint64_t* x, Count n_x, const float* cl, const float* cp,
           float* grad, uint64_t n_params, float* part, cudaStream_t s) {
  const int G = grad_groups(m, n_x.n);
  const size_t smem = size_t(qubit_floats(W, 2 * m.n - 1)) * sizeof(float);
  ANQS_CUDA(cudaFuncSetAttribute(nade_grad_kernel<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
  float* out = G > 1 ? part : grad;
  if (G > 1 && !part) return set_error(ANQS_ERR_CAPACITY, "NADE adjoint needs its partial-sum workspace");
  ProfScope ps(PROF_NADE_GRAD, s);
  ANQS_CUDA_LAUNCH("nade_grad_kernel", launch_k(nade_grad_kernel<W>, dim3(G, 2 * m.n), dim3(NT), smem, s, m, hv, x,
                                                n_x, cl, cp, out, G > 1 ? n_params : uint64_t(0)));
  if (G > 1) {
    uint64_t blocks = (n_params + 255) / 256;
    if (blocks > 152 * 4) blocks = 152 * 4;
    ANQS_CUDA_LAUNCH("nade_partial_sum_kernel", launch_k(nade_partial_sum_kernel, dim3(unsigned(blocks)), dim3(256), 0,
                                                         s, static_cast<const float*>(part), G, n_params, grad));
  }
  return ANQS_OK;
}

}  // namespace

size_t nade_grad_partial_floats(const NadeView& m, uint64_t n_params, uint64_t n_x) {
  const int G = grad_groups(m, n_x);
  return G > 1 ? size_t(G) * n_params : 0;
}

int launch_nade_grad(const NadeView& m, const HamView& hv, const uint64_t* x, Count n_x, const float* cl,
                     const float* cp, float* grad, uint64_t n_params, float* part, cudaStream_t s) {
  if (n_x.n == 0) return ANQS_OK;
  switch (m.w) {
    case 32: return grad_w<32>(m, hv, x, n_x, cl, cp, grad, n_params, part, s);
    case 64: return grad_w<64>(m, hv, x, n_x, cl, cp, grad, n_params, part, s);
    case 128: return grad_w<128>(m, hv, x, n_x, cl, cp, grad, n_params, part, s);
  }
  return set_error(ANQS_ERR_UNSUPPORTED, "NADE width %d", m.w);
}

}  // namespace anqs
