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

}  // namespace anqs
