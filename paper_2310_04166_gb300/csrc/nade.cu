// FP32 form of the paper's own ansatz, the per-qubit complex NADE of
// Appendix B.1: qubit i (0-based, i = 0..2n-1) has a complex MLP reading the
// i previous bits, z1 = W1 x_<i + b1, h1 = tanh z1 (complex), z2 = W2 h1 + b2,
// h2 = LeReLU(Re z2) + i LeReLU(Im z2) (leaky ReLU, 0.01 x below zero), z3 =
// W3 h2 + b3 (2 outputs) and f3(z) = z - 1/2 LSE(2 Re z): log psi_i(x_i | x_<i)
// = f3(z3)_{x_i}.
//
// Slot p groups qubits 2p (alpha) and 2p+1 (beta): psi_slot(a + 2b) =
// psi_2p(a) psi_2p+1(b | a).  MU masking (Sec. III.C) acts on each binary
// conditional: qubit 2p's allowed values are the a with an allowed (a, b) in
// the slot mask, qubit 2p+1's the b with (a, b) allowed; the modulus is
// renormalised over them, the phases kept; DU slots of an MU-d strategy mask
// nothing.  A slot's 8 values l_v = log |psi_slot(v)|^2, phi_v =
// arg psi_slot(v) are thus already a normalised distribution, and log psi(x)
// is the sum over the qubits of x's own path of the masked qubit terms
// Re z3_i(x_i) - LSE_{A_i}(2 Re z3_i) / 2 + i Im z3_i(x_i) (A_i the allowed
// values): one evaluation per qubit, where the slot values need three per
// slot (qubit 2p+1 for both values of qubit 2p).
//
// Tile engine: a CTA of 256 threads evaluates one qubit for a tile of
// TR = RJ * 1024 / W rows.  The W2 product, the bulk of the work, is a complex
// GEMM [TR x W] x [W x W]^T run from shared memory (W2 with row stride W + 1,
// h1 transposed with row stride TR + 1) with a register tile of RJ rows x 4
// units per thread; the input layer, tanh, LeReLU and the 2-output head are
// elementwise or short reductions around it.  RJ = 4 for launches with
// enough rows to fill the GPU, RJ = 1 (4x smaller tiles, 4x more CTAs) for
// the latency-bound small ones (sampler levels, parent passes).
//
// Modes: LOGPSI (log psi of rows, path qubits only), RAW (the 8 slot values
// of every slot of every row: the parent pass of the local energy), SUFFIX
// (for each connected x', sorted by its first differing slot j, the path terms
// of the slots p > j: prefix reuse, the slots <= j come from the parent), and
// LOGITS (slot p's 8 values for the sampler's prefixes).
#include <cmath>

#include <cooperative_groups.h>

#include "common.cuh"

namespace anqs {
namespace {

constexpr int NT = 256;

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
  const float inv = __frcp_rn(fmaf(sa1, sa1, cb1 * cb1));
  return make_float2(sa1 * ca1 * inv, sb1 * cb1 * inv);
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

// allowed values (bit b = value b) of qubit i on the path x: from the slot
// mask pm of slot p = i / 2 on MU slots, both values on DU slots
__device__ __forceinline__ unsigned qubit_allowed(const HamView& hv, int i, uint64_t x, unsigned pm) {
  const int p = i >> 1;
  if (p >= hv.mu_lv) return 3u;
  if ((i & 1) == 0) return ((pm | (pm >> 2)) & 1u) | (((pm >> 1) | (pm >> 3)) & 1u) << 1;
  const int a = int((x >> (2 * p)) & 1ull);
  return ((pm >> a) & 1u) | ((pm >> (a + 2)) & 1u) << 1;
}

// acc += w h (complex)
__device__ __forceinline__ void cmac(float2& acc, float2 w, float2 h) {
  acc.x = fmaf(w.x, h.x, acc.x);
  acc.x = fmaf(-w.y, h.y, acc.x);
  acc.y = fmaf(w.x, h.y, acc.y);
  acc.y = fmaf(w.y, h.x, acc.y);
}

// h1 = tanh z1 of one hidden unit: z1 = b1 + the sum of the W1 columns k < i
// whose input bit is set (w1 = the unit's row of W1).  The sum is
// Kahan-compensated: z + c carries it to about u^2, which matters only next
// to a pole of tanh.  The loop runs over all k < i so that lanes sharing the
// unit load each W1 entry together.
__device__ __forceinline__ float2 input_layer(const float2* __restrict__ w1, float2 b1, uint64_t bits, int i) {
  float2 z = b1, c = make_float2(0.f, 0.f);
  for (int k = 0; k < i; ++k) {
    if (!((bits >> k) & 1ull)) continue;
    const float2 wv = __ldg(w1 + k);
    const float yx = wv.x - c.x, yy = wv.y - c.y;
    const float tx = z.x + yx, ty = z.y + yy;
    c.x = (tx - z.x) - yx;
    c.y = (ty - z.y) - yy;
    z.x = tx;
    z.y = ty;
  }
  return ctanh(z.x, -c.x, z.y, -c.y);
}

// ---------------------------------------------------------------------------
// Tile engine
// ---------------------------------------------------------------------------
template <int W, int RJ>
struct Tile {
  static constexpr int NTX = W / 4;      // GEMM thread grid: NTX x NTY threads, 4 units x RJ rows each
  static constexpr int NTY = NT / NTX;
  static constexpr int TR = NTY * RJ;    // rows per tile
  static constexpr int WS = W + 1;       // W2 row stride (float2)
  static constexpr int HS = TR + 4;      // h row stride (floats; real and imaginary planes)
  static constexpr int KP = 128 / TR;    // k-parts of the head reduction
  static constexpr int NZ = 1;           // z3 tiles kept (one evaluation per CTA)
  static constexpr size_t w2_bytes = size_t(W) * WS * sizeof(float2);
  static constexpr size_t h_bytes = 2 * size_t(W) * HS * sizeof(float);
  static constexpr size_t smem_bytes = w2_bytes + h_bytes + (size_t(KP) * TR * 2 + size_t(NZ) * TR * 2) * sizeof(float2);
  static_assert(NTX * NTY == NT && NT % TR == 0 && W % KP == 0 && TR % 4 == 0, "tile shape");
};

// asynchronous global -> shared copy of 8 bytes (both 8-byte aligned)
__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gmem_src) {
  const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(smem_dst));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

struct TileSmem {
  float2* W2;        // [W][WS]: W2[u][k] at u * WS + k
  float *Hr, *Hi;    // [W][HS]: h[r][k] at k * HS + r
  float2 *Z3p, *Z3;
};

template <int W, int RJ>
__device__ __forceinline__ TileSmem tile_smem(float2* base) {
  using T = Tile<W, RJ>;
  TileSmem s;
  char* p = reinterpret_cast<char*>(base);
  s.W2 = reinterpret_cast<float2*>(p);
  s.Hr = reinterpret_cast<float*>(p + T::w2_bytes);
  s.Hi = s.Hr + size_t(W) * T::HS;
  s.Z3p = reinterpret_cast<float2*>(s.Hi + size_t(W) * T::HS);
  s.Z3 = s.Z3p + size_t(T::KP) * T::TR * 2;
  return s;
}

// z3 of qubit i for the tile's rows into z3out[r][2].  Bit k < i of row r is
// bit k of xt[r] for k < kx and `a` for k = kx (kx = i: all bits from x).
// `staged` is the qubit whose W2 is in shared memory or on its way there
// (`pending`: asynchronous copies in flight), uniform over the CTA.  With
// next >= 0, qubit next's W2 is copied in asynchronously as soon as this
// evaluation's GEMM is done with the buffer, so the copy overlaps the head,
// the caller's row work and the next evaluation's input layer.
// Starts and ends with the CTA synchronised.
template <int W, int RJ>
__device__ void eval_qubit(const NadeView& m, int i, int kx, int a, const uint64_t* xt, const TileSmem& S,
                           float2* z3out, int& staged, bool& pending, int next) {
  using T = Tile<W, RJ>;
  constexpr int TR = T::TR, WS = T::WS, HS = T::HS, NTX = T::NTX;
  const int tid = threadIdx.x;
  const QubitPtr q = qubit_ptrs(m, i);
  if (pending) {  // this thread's copies land before the barrier that ends the input layer
    cp_async_wait_all();
    pending = false;
  }
  if (staged != i) {  // W2 [u][k] -> shared [u][k] (coalesced, conflict-free)
    for (int e = tid; e < W * W; e += NT) S.W2[(e / W) * WS + (e % W)] = __ldg(q.W2 + e);
    staged = i;
  }
  {  // z1 and tanh: lanes of a warp take consecutive rows of one unit
    const int r = tid % TR;
    const uint64_t xr = xt[r];
    // the input bits x_<i of the row: x's bits below kx, then a at kx
    const uint64_t bits0 = (kx >= 64 ? xr : (xr & ((1ull << kx) - 1ull))) | (kx < i && a ? (1ull << kx) : 0ull);
    for (int u = tid / TR; u < W; u += NT / TR) {
      const float2 h = input_layer(q.W1 + size_t(u) * i, __ldg(q.b1 + u), bits0, i);
      S.Hr[u * HS + r] = h.x;
      S.Hi[u * HS + r] = h.y;
    }
  }
  __syncthreads();
  // z2[r][u] = sum_k W2[u][k] h1[r][k]: thread (tx, ty) owns units tx + NTX c and rows RJ ty + j
  const int tx = tid % NTX, ty = tid / NTX;
  float2 z2[RJ][4];
#pragma unroll
  for (int j = 0; j < RJ; ++j)
#pragma unroll
    for (int c = 0; c < 4; ++c) z2[j][c] = make_float2(0.f, 0.f);
#pragma unroll 2
  for (int k = 0; k < W; ++k) {
    float2 w[4], h[RJ];
#pragma unroll
    for (int c = 0; c < 4; ++c) w[c] = S.W2[(tx + NTX * c) * WS + k];
    if constexpr (RJ % 4 == 0) {
#pragma unroll
      for (int j = 0; j < RJ; j += 4) {
        const float4 a4 = *reinterpret_cast<const float4*>(S.Hr + k * HS + RJ * ty + j);
        const float4 b4 = *reinterpret_cast<const float4*>(S.Hi + k * HS + RJ * ty + j);
        h[j] = make_float2(a4.x, b4.x);
        h[j + 1] = make_float2(a4.y, b4.y);
        h[j + 2] = make_float2(a4.z, b4.z);
        h[j + 3] = make_float2(a4.w, b4.w);
      }
    } else {
#pragma unroll
      for (int j = 0; j < RJ; ++j) h[j] = make_float2(S.Hr[k * HS + RJ * ty + j], S.Hi[k * HS + RJ * ty + j]);
    }
#pragma unroll
    for (int j = 0; j < RJ; ++j)
#pragma unroll
      for (int c = 0; c < 4; ++c) cmac(z2[j][c], w[c], h[j]);
  }
  __syncthreads();  // h1 fully consumed: h2 overwrites it; W2 no longer read
  if (next >= 0 && next != i) {
    const float2* src = qubit_ptrs(m, next).W2;
    for (int e = tid; e < W * W; e += NT) cp_async8(S.W2 + (e / W) * WS + (e % W), src + e);
    cp_async_commit();
    staged = next;
    pending = true;
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int u = tx + NTX * c;
    const float2 b = __ldg(q.b2 + u);
#pragma unroll
    for (int j = 0; j < RJ; ++j) {
      S.Hr[u * HS + RJ * ty + j] = lerelu(z2[j][c].x + b.x);
      S.Hi[u * HS + RJ * ty + j] = lerelu(z2[j][c].y + b.y);
    }
  }
  __syncthreads();
  {  // head: z3[r][o] = b3[o] + sum_k W3[o][k] h2[r][k], the k range in KP parts
    constexpr int KL = W / T::KP;
    const int r = tid % TR, g = tid / TR, o = g & 1, part = g >> 1;
    float2 z = make_float2(0.f, 0.f);
    for (int k = part * KL; k < (part + 1) * KL; ++k)
      cmac(z, __ldg(q.W3 + o * W + k), make_float2(S.Hr[k * HS + r], S.Hi[k * HS + r]));
    S.Z3p[(part * TR + r) * 2 + o] = z;
  }
  __syncthreads();
  if (tid < 2 * TR) {
    const int r = tid >> 1, o = tid & 1;
    float2 z = __ldg(q.b3 + o);
    for (int part = 0; part < T::KP; ++part) {
      const float2 t = S.Z3p[(part * TR + r) * 2 + o];
      z.x += t.x;
      z.y += t.y;
    }
    z3out[r * 2 + o] = z;
  }
  __syncthreads();
}

// Masked path term of qubit i of row x from its z3 = (z0, z1): (Re, Im) of
// log psi_i(x_i | x_<i) after masking; false when x_i (or, at the slot's
// second qubit, the slot outcome) is not allowed.
__device__ __forceinline__ bool path_term(const HamView& hv, int i, uint64_t x, float2 z0, float2 z1, float& tre,
                                          float& tim) {
  const int p = i >> 1, xi = int((x >> i) & 1ull);
  const unsigned pm = prefix_mask(hv, p, x);
  const unsigned allowed = qubit_allowed(hv, i, x, pm);
  tim = xi ? z1.y : z0.y;
  if (!((allowed >> xi) & 1u)) return false;
  if ((i & 1) && !((pm >> int((x >> (2 * p)) & 3ull)) & 1u)) return false;
  const float r0 = (allowed & 1u) ? 2.f * z0.x : -INFINITY;
  const float r1 = (allowed & 2u) ? 2.f * z1.x : -INFINITY;
  const float mx = fmaxf(r0, r1);
  tre = (xi ? z1.x : z0.x) - 0.5f * (mx + logf(expf(r0 - mx) + expf(r1 - mx)));
  return true;
}

// The 8 values of slot p for row r from the three evaluations z[e] ([TR][2]
// each: qubit 2p, qubit 2p+1 given a = 0, given a = 1).
__device__ void slot_values(const HamView& hv, int p, uint64_t x, const float2* const (&z)[3], int r, float* o8) {
  float2 l[3][2];
#pragma unroll
  for (int e = 0; e < 3; ++e) {  // f3
    const float2 z0 = z[e][r * 2], z1 = z[e][r * 2 + 1];
    const float mx = fmaxf(2.f * z0.x, 2.f * z1.x);
    const float lse = 0.5f * (mx + logf(expf(2.f * z0.x - mx) + expf(2.f * z1.x - mx)));
    l[e][0] = make_float2(z0.x - lse, z0.y);
    l[e][1] = make_float2(z1.x - lse, z1.y);
  }
  if (p < hv.mu_lv) {  // v = a + 2b: a allowed if (a, 0) or (a, 1) is; b given a if (a, b) is
    const unsigned pm = prefix_mask(hv, p, x);
    mask2(l[0][0], l[0][1], ((pm | (pm >> 2)) & 1u) | (((pm >> 1) | (pm >> 3)) & 1u) << 1);
    mask2(l[1][0], l[1][1], (pm & 1u) | ((pm >> 2) & 1u) << 1);
    mask2(l[2][0], l[2][1], ((pm >> 1) & 1u) | ((pm >> 3) & 1u) << 1);
  }
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    const int a = v & 1, b = v >> 1;
    o8[v] = 2.f * (l[0][a].x + l[1 + a][b].x);
    o8[4 + v] = l[0][a].y + l[1 + a][b].y;
  }
}

enum { MODE_LOGPSI = 0, MODE_RAW = 1, MODE_SUFFIX = 2, MODE_LOGITS = 3 };

struct FwdArgs {
  const uint64_t* x;        // rows (LOGPSI, RAW, LOGITS) or connected determinants (SUFFIX)
  Count rows;               // row count (SUFFIX: bound on the connected rows; the count is offsets[n - 1])
  int p;                    // LOGITS: the slot
  float *la, *ph;           // LOGPSI: outputs
  float* out8;              // RAW: [row][n][8]; LOGITS: [row][8]
  const uint8_t* js;        // SUFFIX: first differing slot of each connected row
  const uint32_t* perm;     // SUFFIX: connected rows in ascending js
  const uint32_t* offsets;  // SUFFIX: offsets[p] = rows with js < p
  float2* T;                // SUFFIX: [row][n] path terms of the slots > js
};

template <int W, int RJ, int MODE>
__global__ void __launch_bounds__(NT) nade_fwd_kernel(NadeView m, HamView hv, FwdArgs A) {
  ANQS_PDL_ENTRY();
  constexpr int TR = Tile<W, RJ>::TR;
  extern __shared__ float2 dsm[];
  const TileSmem S = tile_smem<W, RJ>(dsm);
  __shared__ uint64_t xt[TR];
  __shared__ float la[TR], ph[TR], t0r[TR], t0i[TR];
  __shared__ int dead[TR], jr[TR];
  __shared__ uint32_t rid[TR];
  const int n = m.n, tid = threadIdx.x;
  const uint64_t rows = MODE == MODE_SUFFIX ? uint64_t(A.offsets[n - 1]) : A.rows.get();
  int staged = -1;
  bool pending = false;
  for (uint64_t base = uint64_t(blockIdx.x) * TR; base < rows; base += uint64_t(gridDim.x) * TR) {
    if (tid < TR) {
      const uint64_t l = base + tid;
      const bool valid = l < rows;
      if (MODE == MODE_SUFFIX) {
        const uint32_t row = valid ? A.perm[l] : 0u;
        rid[tid] = row;
        jr[tid] = valid ? int(A.js[row]) : n;  // j = n: no slot of the row is written
        xt[tid] = valid ? A.x[row] : 0ull;
      } else {
        xt[tid] = valid ? A.x[l] : 0ull;
      }
      la[tid] = 0.f;
      ph[tid] = 0.f;
      dead[tid] = 0;
    }
    __syncthreads();
    if (MODE == MODE_LOGPSI) {
      for (int i = 0; i < 2 * n; ++i) {
        eval_qubit<W, RJ>(m, i, i, 0, xt, S, S.Z3, staged, pending, i + 1 < 2 * n ? i + 1 : -1);
        if (tid < TR) {
          float tr = 0.f, ti;
          if (path_term(hv, i, xt[tid], S.Z3[tid * 2], S.Z3[tid * 2 + 1], tr, ti)) la[tid] += tr;
          else dead[tid] = 1;
          ph[tid] += ti;
        }
      }
      __syncthreads();
      if (tid < TR && base + tid < rows) {
        const uint64_t x = xt[tid];
        const bool out = dead[tid] || (n < 32 && (x >> (2 * n)) != 0);
        A.la[base + tid] = out ? -INFINITY : la[tid];
        A.ph[base + tid] = ph[tid];
      }
    } else if (MODE == MODE_SUFFIX) {
      // rows are in ascending j: the tile's first row has the smallest, and
      // every row needs the slots above its own j only
      for (int i = 2 * (jr[0] + 1); i < 2 * n; ++i) {
        eval_qubit<W, RJ>(m, i, i, 0, xt, S, S.Z3, staged, pending, i + 1 < 2 * n ? i + 1 : -1);
        const int p = i >> 1;
        if (tid < TR && p > jr[tid]) {
          float tr = 0.f, ti;
          const bool ok = path_term(hv, i, xt[tid], S.Z3[tid * 2], S.Z3[tid * 2 + 1], tr, ti);
          if ((i & 1) == 0) {
            t0r[tid] = ok ? tr : -INFINITY;
            t0i[tid] = ti;
          } else {
            A.T[uint64_t(rid[tid]) * n + p] = make_float2(ok ? t0r[tid] + tr : -INFINITY, t0i[tid] + ti);
          }
        }
      }
    } else {
      // RAW (slot blockIdx.y / 3), LOGITS (slot A.p): the three evaluations
      // of the slot run in the three CTAs of a cluster (CTA e = blockIdx.y %
      // 3: qubit 2p, qubit 2p+1 given a = 0, given a = 1); after a cluster
      // barrier CTA 0 reads the other two z3 tiles from their shared memory
      cooperative_groups::cluster_group cl = cooperative_groups::this_cluster();
      const int e = int(blockIdx.y % 3);
      const int p = MODE == MODE_RAW ? int(blockIdx.y / 3) : A.p;
      eval_qubit<W, RJ>(m, e == 0 ? 2 * p : 2 * p + 1, 2 * p, e == 2 ? 1 : 0, xt, S, S.Z3, staged, pending, -1);
      cl.sync();
      if (e == 0 && tid < TR && base + tid < rows) {
        const float2* const z[3] = {S.Z3, cl.map_shared_rank(S.Z3, cl.block_rank() + 1),
                                    cl.map_shared_rank(S.Z3, cl.block_rank() + 2)};
        float o8[8];
        slot_values(hv, p, xt[tid], z, tid, o8);
        float* dst = MODE == MODE_RAW ? A.out8 + ((base + tid) * n + p) * 8 : A.out8 + (base + tid) * 8;
#pragma unroll
        for (int v = 0; v < 8; ++v) dst[v] = o8[v];
      }
      cl.sync();  // the peers' z3 stay until CTA 0 has read them
    }
    __syncthreads();
  }
  if (pending) cp_async_wait_all();  // no copy outlives the CTA
}

// Grid: ny slots (RAW: one per slot) x row tiles, at most one wave of
// resident CTAs.  RJ = 4 when its tiles fill a wave, else RJ = 1.
// CTAs along y: RAW 3 per slot, LOGITS 3 (clusters of three, one per
// evaluation of the slot), else 1
template <int MODE>
constexpr bool clustered() { return MODE == MODE_RAW || MODE == MODE_LOGITS; }

template <int W, int RJ, int MODE>
int fwd_launch(const NadeView& m, const HamView& hv, const FwdArgs& a, uint64_t max_rows, int prof, cudaStream_t s) {
  constexpr int TR = Tile<W, RJ>::TR;
  const size_t smem = Tile<W, RJ>::smem_bytes;
  auto kern = nade_fwd_kernel<W, RJ, MODE>;
  ANQS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
  int occ = 0;
  ANQS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NT, smem));
  const uint64_t ny = MODE == MODE_RAW ? 3ull * uint64_t(m.n) : (clustered<MODE>() ? 3ull : 1ull);
  uint64_t cap = 152ull * uint64_t(occ > 0 ? occ : 1) / ny;
  if (cap < 1) cap = 1;
  uint64_t blocks = (max_rows + TR - 1) / TR;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  ProfScope ps(prof, s);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(blocks), unsigned(ny));
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  attr[1].id = cudaLaunchAttributeClusterDimension;
  attr[1].val.clusterDim.x = 1;
  attr[1].val.clusterDim.y = clustered<MODE>() ? 3 : 1;
  attr[1].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  note_launch();
  ANQS_CUDA_LAUNCH("nade_fwd_kernel", cudaLaunchKernelEx(&cfg, kern, m, hv, a));
  return ANQS_OK;
}

template <int W, int MODE>
int fwd_w(const NadeView& m, const HamView& hv, const FwdArgs& a, uint64_t max_rows, int prof, cudaStream_t s) {
  const uint64_t ny = MODE == MODE_RAW ? 3ull * uint64_t(m.n) : (clustered<MODE>() ? 3ull : 1ull);
  const uint64_t big_tiles = (max_rows + Tile<W, 4>::TR - 1) / Tile<W, 4>::TR;
  if (big_tiles * ny >= 152) return fwd_launch<W, 4, MODE>(m, hv, a, max_rows, prof, s);
  return fwd_launch<W, 1, MODE>(m, hv, a, max_rows, prof, s);
}

template <int MODE>
int fwd(const NadeView& m, const HamView& hv, const FwdArgs& a, uint64_t max_rows, int prof, cudaStream_t s) {
  switch (m.w) {
    case 32: return fwd_w<32, MODE>(m, hv, a, max_rows, prof, s);
    case 64: return fwd_w<64, MODE>(m, hv, a, max_rows, prof, s);
    case 128: return fwd_w<128, MODE>(m, hv, a, max_rows, prof, s);
  }
  return set_error(ANQS_ERR_UNSUPPORTED, "NADE width %d", m.w);
}

// workspace of the local energy with prefix reuse
struct NadeElocWs {
  uint64_t* xp;
  double *hv, *hd;
  uint8_t* js;
  float *la_x, *ph_x, *raw, *cache;
  float2* T;
  uint32_t *perm, *hist, *cursor, *offsets, *ticket;
};

size_t plan_eloc(const anqs_ham* H, uint64_t n_x, Arena& A, NadeElocWs& w) {
  const uint64_t m = n_x * H->v.K, n = uint64_t(H->v.n);
  w.xp = A.take<uint64_t>(m);
  w.hv = A.take<double>(m);
  w.js = A.take<uint8_t>(m);
  w.hd = A.take<double>(n_x);
  w.la_x = A.take<float>(n_x);
  w.ph_x = A.take<float>(n_x);
  w.raw = A.take<float>(n_x * n * 8);
  w.cache = A.take<float>(n_x * n * TC_CACHE_F);
  w.T = A.take<float2>(m * n);
  w.perm = A.take<uint32_t>(m);
  w.cursor = A.take<uint32_t>(ANQS_MAX_ORB);
  w.offsets = A.take<uint32_t>(ANQS_MAX_ORB + 1);
  w.hist = A.take<uint32_t>(TC_CTL_WORDS);
  w.ticket = w.hist + TC_CTL_STATS_TICKET;
  return A.off;
}

}  // namespace

int launch_nade_logpsi(const NadeView& m, const HamView& hv, const uint64_t* x, Count n_x, float* la, float* ph,
                       cudaStream_t s) {
  if (n_x.n == 0) return ANQS_OK;
  FwdArgs a{};
  a.x = x;
  a.rows = n_x;
  a.la = la;
  a.ph = ph;
  return fwd<MODE_LOGPSI>(m, hv, a, n_x.n, PROF_NADE, s);
}

int launch_nade_slot_logits(const NadeView& m, const HamView& hv, int p, const uint64_t* pre, const uint64_t* n_dev,
                            uint64_t max_rows, float* out8, cudaStream_t s) {
  FwdArgs a{};
  a.x = pre;
  a.rows = Count{max_rows, n_dev, 1};
  a.p = p;
  a.out8 = out8;
  return fwd<MODE_LOGITS>(m, hv, a, max_rows, PROF_NADE_SLOT, s);
}

size_t nade_eloc_workspace(const anqs_ham* H, uint64_t n_x) {
  Arena A(nullptr, 0);
  NadeElocWs w;
  return plan_eloc(H, n_x, A, w);
}

// Local energy with prefix reuse: the parents' slot values (RAW) give log psi(x)
// and, per slot, the prefix sums and the slot's masked terms; each connected
// x' then needs only the path terms of the slots above its first differing
// slot j (SUFFIX, rows sorted by j); the assembly adds them up and sums
// H_xx' psi(x')/psi(x) in FP64.
int run_eloc_nade(const anqs_model* M, const anqs_ham* H, const uint64_t* x, Count n_x, double* ere, double* eim,
                  const uint64_t* counts, double* stats, void* ws, size_t ws_bytes, cudaStream_t s) {
  Arena A(ws, ws_bytes);
  NadeElocWs w;
  plan_eloc(H, n_x.n, A, w);
  if (!A.fits() || !ws) return set_error(ANQS_ERR_CAPACITY, "workspace needs %zu bytes", A.off);
  const uint64_t K = H->v.K;
  const Count mc = scaled(n_x, K);
  if (mc.n > 0xffffffffull) return set_error(ANQS_ERR_UNSUPPORTED, "more than 2^32 connected determinants per call");
  ANQS_TRY(launch_connected(H->v, x, n_x, w.xp, w.hv, w.js, w.hd, s, w.hist));
  {
    FwdArgs a{};
    a.x = x;
    a.rows = n_x;
    a.out8 = w.raw;
    ANQS_TRY(fwd<MODE_RAW>(M->nade, H->v, a, n_x.n, PROF_NADE_PARENT, s));
    ProfScope ps(PROF_TC_FINALIZE, s);
    ANQS_TRY(launch_tc_finalize(H->v, x, n_x, w.raw, w.la_x, w.ph_x, w.cache, s));
  }
  {
    ProfScope ps(PROF_TC_SORT, s);
    ANQS_TRY(launch_js_sort(w.js, mc, H->v.n, w.hist, w.cursor, w.offsets, w.perm, s));
  }
  {
    FwdArgs a{};
    a.x = w.xp;
    a.rows = mc;
    a.js = w.js;
    a.perm = w.perm;
    a.offsets = w.offsets;
    a.T = w.T;
    ANQS_TRY(fwd<MODE_SUFFIX>(M->nade, H->v, a, mc.n, PROF_NADE_SUFFIX, s));
  }
  ProfScope ps(PROF_TC_ELOC, s);
  return launch_eloc_assemble(H->v.n, uint32_t(K), n_x, w.xp, w.js, w.cache, w.T, w.hv, w.hd, w.la_x, w.ph_x, ere, eim,
                              StatsOut{counts, stats, w.ticket}, s);
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
                                                       Count rows_, CotSrc cot, float* __restrict__ out,
                                                       uint64_t out_stride) {
  ANQS_PDL_ENTRY();
  constexpr int R = NT / W;
  extern __shared__ float2 acc[];  // qubit i's parameter block (complex entries)
  __shared__ float2 h1[R * W], h2[R * W], gz1[R * W], gz2[R * W], z3[R * 2], g3[R * 2];
  __shared__ uint64_t xt[R];
  const int i = blockIdx.y, p = i >> 1;
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
    h1[r * W + u] = input_layer(q.W1 + size_t(u) * i, __ldg(q.b1 + u), x, i);
    __syncthreads();
    float2 z = __ldg(q.b2 + u);
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
      const unsigned allowed = qubit_allowed(hv, i, x, prefix_mask(hv, p, x));
      const int xi = int((x >> i) & 1ull);
      float2 g0 = make_float2(0.f, 0.f), g1 = g0;
      if (base + r < rows && ((allowed >> xi) & 1u)) {
        const float r0 = (allowed & 1u) ? 2.f * z3[r * 2].x : -INFINITY;
        const float r1 = (allowed & 2u) ? 2.f * z3[r * 2 + 1].x : -INFINITY;
        const float mx = fmaxf(r0, r1);
        const float e0 = expf(r0 - mx), e1 = expf(r1 - mx);
        const float pi0 = e0 / (e0 + e1), pi1 = e1 / (e0 + e1);
        float c_l, c_p;
        cot_of(cot, base + r, c_l, c_p);
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

// Tiled adjoint (widths 32 and 64): CTA (g, i) takes qubit i for the row
// tiles g, g + G, ... of TR = 4096 / W rows.  The qubit's W2 is staged in
// shared memory once; per tile the forward keeps h1 and h2 (real and
// imaginary planes [unit][row]), and the backward runs the two W x W
// contractions of the adjoint, gh1 = W2^H gz2 and dW2 += gz2^T conj(h1), with
// register tiles.  The qubit's parameter block accumulates in shared memory,
// every entry owned by one thread and the rows taken in tile order
// (deterministic), as in the kernel above.
__device__ __forceinline__ void cmac_conj(float2& acc, float2 a, float2 b) {  // acc += conj(a) b
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(-a.y, b.x, acc.y);
}

template <int W>
struct GradTile {
  using T = Tile<W, 4>;
  static constexpr int TR = T::TR, WS = T::WS, HS = T::HS, KP = T::KP;
  static constexpr int UK = W / 16;  // dW2 register tile: UK units x UK inputs per thread (16 x 16 threads)
  static size_t smem_bytes(int n) {
    return size_t(W) * WS * sizeof(float2) + 4 * size_t(W) * HS * sizeof(float) +
           size_t(KP) * TR * 2 * sizeof(float2) + size_t(qubit_floats(W, 2 * n - 1)) * sizeof(float);
  }
};

template <int W>
__global__ void __launch_bounds__(NT) nade_grad_tile_kernel(NadeView m, HamView hv, const uint64_t* __restrict__ xs,
                                                            Count rows_, CotSrc cot, float* __restrict__ out,
                                                            uint64_t out_stride) {
  using G = GradTile<W>;
  constexpr int TR = G::TR, WS = G::WS, HS = G::HS, KP = G::KP, NTX = W / 4, UK = G::UK;
  extern __shared__ float4 dsm4[];
  float2* W2s = reinterpret_cast<float2*>(dsm4);  // [W][WS]
  float* H1r = reinterpret_cast<float*>(W2s + size_t(W) * WS);
  float* H1i = H1r + W * HS;                       // h1 planes [W][HS]
  float* Gr = H1i + W * HS;
  float* Gi = Gr + W * HS;                         // h2, then gz2, then gz1
  float2* Z3p = reinterpret_cast<float2*>(Gi + W * HS);
  float2* acc = Z3p + KP * TR * 2;                 // the qubit's parameter block (complex entries)
  __shared__ uint64_t xt[TR];
  __shared__ float2 z3[TR * 2], g3[TR * 2];
  const int i = blockIdx.y, p = i >> 1, tid = threadIdx.x;
  const QubitPtr q = qubit_ptrs(m, i);
  const uint32_t nc = qubit_floats(W, i) / 2;
  const uint32_t ob1 = W * i, oW2 = ob1 + W, ob2 = oW2 + W * W, oW3 = ob2 + W;  // b3 follows W3 at oW3 + 2W
  // prologue: the parameters are written before any library kernel runs
  for (uint32_t e = tid; e < nc; e += NT) acc[e] = make_float2(0.f, 0.f);
  for (int e = tid; e < W * W; e += NT) W2s[(e / W) * WS + (e % W)] = __ldg(q.W2 + e);
  ANQS_PDL_WAIT();
  ANQS_PDL_TRIGGER();
  const uint64_t rows = rows_.get();
  const int tx = tid % NTX, ty = tid / NTX;
  for (uint64_t base = uint64_t(blockIdx.x) * TR; base < rows; base += uint64_t(gridDim.x) * TR) {
    if (tid < TR) xt[tid] = base + tid < rows ? xs[base + tid] : 0ull;
    __syncthreads();
    {  // h1 = tanh(z1) of the path x_<i
      const int r = tid % TR;
      for (int u = tid / TR; u < W; u += NT / TR) {
        const float2 h = input_layer(q.W1 + size_t(u) * i, __ldg(q.b1 + u), xt[r], i);
        H1r[u * HS + r] = h.x;
        H1i[u * HS + r] = h.y;
      }
    }
    __syncthreads();
    {  // z2 = W2 h1 + b2, h2 = LeReLU parts -> G planes
      float2 z2[4][4];
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int c = 0; c < 4; ++c) z2[j][c] = make_float2(0.f, 0.f);
#pragma unroll 2
      for (int k = 0; k < W; ++k) {
        float2 w[4], h[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) w[c] = W2s[(tx + NTX * c) * WS + k];
        const float4 a4 = *reinterpret_cast<const float4*>(H1r + k * HS + 4 * ty);
        const float4 b4 = *reinterpret_cast<const float4*>(H1i + k * HS + 4 * ty);
        h[0] = make_float2(a4.x, b4.x);
        h[1] = make_float2(a4.y, b4.y);
        h[2] = make_float2(a4.z, b4.z);
        h[3] = make_float2(a4.w, b4.w);
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
          for (int c = 0; c < 4; ++c) cmac(z2[j][c], w[c], h[j]);
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int u = tx + NTX * c;
        const float2 b = __ldg(q.b2 + u);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          Gr[u * HS + 4 * ty + j] = lerelu(z2[j][c].x + b.x);
          Gi[u * HS + 4 * ty + j] = lerelu(z2[j][c].y + b.y);
        }
      }
    }
    __syncthreads();
    {  // head: z3[r][o] = b3[o] + sum_k W3[o][k] h2[r][k]
      constexpr int KL = W / KP;
      const int r = tid % TR, g = tid / TR, o = g & 1, part = g >> 1;
      float2 z = make_float2(0.f, 0.f);
      for (int k = part * KL; k < (part + 1) * KL; ++k)
        cmac(z, __ldg(q.W3 + o * W + k), make_float2(Gr[k * HS + r], Gi[k * HS + r]));
      Z3p[(part * TR + r) * 2 + o] = z;
    }
    __syncthreads();
    if (tid < 2 * TR) {
      const int r = tid >> 1, o = tid & 1;
      float2 z = __ldg(q.b3 + o);
      for (int part = 0; part < KP; ++part) {
        const float2 t = Z3p[(part * TR + r) * 2 + o];
        z.x += t.x;
        z.y += t.y;
      }
      z3[r * 2 + o] = z;
    }
    __syncthreads();
    if (tid < TR) {  // cotangent of z3: the path's masked softmax (see the kernel above)
      const int r = tid;
      const uint64_t x = xt[r];
      const unsigned allowed = qubit_allowed(hv, i, x, prefix_mask(hv, p, x));
      const int xi = int((x >> i) & 1ull);
      float2 g0 = make_float2(0.f, 0.f), g1 = g0;
      if (base + r < rows && ((allowed >> xi) & 1u)) {
        const float r0 = (allowed & 1u) ? 2.f * z3[r * 2].x : -INFINITY;
        const float r1 = (allowed & 2u) ? 2.f * z3[r * 2 + 1].x : -INFINITY;
        const float mx = fmaxf(r0, r1);
        const float e0 = expf(r0 - mx), e1 = expf(r1 - mx);
        const float pi0 = e0 / (e0 + e1), pi1 = e1 / (e0 + e1);
        float c_l, c_p;
        cot_of(cot, base + r, c_l, c_p);
        g0 = make_float2(c_l * ((xi == 0 ? 1.f : 0.f) - pi0), xi == 0 ? c_p : 0.f);
        g1 = make_float2(c_l * ((xi == 1 ? 1.f : 0.f) - pi1), xi == 1 ? c_p : 0.f);
      }
      g3[r * 2] = g0;
      g3[r * 2 + 1] = g1;
    }
    __syncthreads();
    // W3, b3: sum_r g3[r][o] conj(h2[r][j]), sum_r g3[r][o]
    if (tid < 2 * W + 2) {
      float2 sacc = acc[oW3 + tid];
      if (tid < 2 * W) {
        const int o = tid / W, j = tid % W;
        for (int r = 0; r < TR; ++r) cmac_conj(sacc, make_float2(Gr[j * HS + r], Gi[j * HS + r]), g3[r * 2 + o]);
      } else {
        for (int r = 0; r < TR; ++r) {
          sacc.x += g3[r * 2 + (tid - 2 * W)].x;
          sacc.y += g3[r * 2 + (tid - 2 * W)].y;
        }
      }
      acc[oW3 + tid] = sacc;
    }
    __syncthreads();
    // gz2 = LeReLU'(z2) (conj(W3)^T g3), in place of h2 (sign of h2 = sign of z2)
    for (int e = tid; e < TR * W; e += NT) {
      const int u = e / TR, r = e % TR;
      const float2 w0 = __ldg(q.W3 + u), w1 = __ldg(q.W3 + W + u);
      const float2 ga = g3[r * 2], gb = g3[r * 2 + 1];
      const float gr = w0.x * ga.x + w0.y * ga.y + w1.x * gb.x + w1.y * gb.y;
      const float gi = w0.x * ga.y - w0.y * ga.x + w1.x * gb.y - w1.y * gb.x;
      Gr[u * HS + r] = Gr[u * HS + r] >= 0.f ? gr : 0.01f * gr;
      Gi[u * HS + r] = Gi[u * HS + r] >= 0.f ? gi : 0.01f * gi;
    }
    __syncthreads();
    if (tid < W) {  // b2
      float2 sacc = acc[ob2 + tid];
      for (int r = 0; r < TR; ++r) {
        sacc.x += Gr[tid * HS + r];
        sacc.y += Gi[tid * HS + r];
      }
      acc[ob2 + tid] = sacc;
    }
    {  // W2[u][k] += sum_r gz2[r][u] conj(h1[r][k]): thread owns a UK x UK block of (u, k)
      const int u0 = (tid / 16) * UK, k0 = (tid % 16) * UK;
      float2 s[UK][UK];
#pragma unroll
      for (int a = 0; a < UK; ++a)
#pragma unroll
        for (int b = 0; b < UK; ++b) s[a][b] = make_float2(0.f, 0.f);
      for (int r = 0; r < TR; r += 2) {
        float2 gr2[UK], gi2[UK], hr2[UK], hi2[UK];
#pragma unroll
        for (int a = 0; a < UK; ++a) {
          gr2[a] = *reinterpret_cast<const float2*>(Gr + (u0 + a) * HS + r);
          gi2[a] = *reinterpret_cast<const float2*>(Gi + (u0 + a) * HS + r);
          hr2[a] = *reinterpret_cast<const float2*>(H1r + (k0 + a) * HS + r);
          hi2[a] = *reinterpret_cast<const float2*>(H1i + (k0 + a) * HS + r);
        }
#pragma unroll
        for (int a = 0; a < UK; ++a)
#pragma unroll
          for (int b = 0; b < UK; ++b) {
            cmac_conj(s[a][b], make_float2(hr2[b].x, hi2[b].x), make_float2(gr2[a].x, gi2[a].x));
            cmac_conj(s[a][b], make_float2(hr2[b].y, hi2[b].y), make_float2(gr2[a].y, gi2[a].y));
          }
      }
#pragma unroll
      for (int a = 0; a < UK; ++a)
#pragma unroll
        for (int b = 0; b < UK; ++b) {
          float2& d = acc[oW2 + (u0 + a) * W + k0 + b];
          d.x += s[a][b].x;
          d.y += s[a][b].y;
        }
    }
    // gh1[r][k] = sum_u conj(W2[u][k]) gz2[r][u]: thread (tx, ty) owns inputs tx + NTX c, rows 4 ty + j
    float2 gh[4][4];
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int c = 0; c < 4; ++c) gh[j][c] = make_float2(0.f, 0.f);
#pragma unroll 2
    for (int u = 0; u < W; ++u) {
      float2 w[4], g[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) w[c] = W2s[u * WS + tx + NTX * c];
      const float4 a4 = *reinterpret_cast<const float4*>(Gr + u * HS + 4 * ty);
      const float4 b4 = *reinterpret_cast<const float4*>(Gi + u * HS + 4 * ty);
      g[0] = make_float2(a4.x, b4.x);
      g[1] = make_float2(a4.y, b4.y);
      g[2] = make_float2(a4.z, b4.z);
      g[3] = make_float2(a4.w, b4.w);
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int c = 0; c < 4; ++c) cmac_conj(gh[j][c], w[c], g[j]);
    }
    __syncthreads();  // gz2 and the b2 sums are done with the G planes
    // gz1 = conj(1 - h1^2) gh1 -> G planes
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int k = tx + NTX * c, r = 4 * ty + j;
        const float hr = H1r[k * HS + r], hi = H1i[k * HS + r];
        const float dr = 1.f - (hr * hr - hi * hi), di = -2.f * hr * hi;
        const float2 g = gh[j][c];
        Gr[k * HS + r] = dr * g.x + di * g.y;
        Gi[k * HS + r] = dr * g.y - di * g.x;
      }
    __syncthreads();
    // W1[u][k] (real input bits) and b1[u]: sums of gz1 over the rows
    for (uint32_t e = tid; e < uint32_t(W) * (i + 1); e += NT) {
      float2 sacc = acc[e];
      if (e < ob1) {
        const uint32_t u = e / uint32_t(i), k = e % uint32_t(i);
        for (int r = 0; r < TR; ++r)
          if ((xt[r] >> k) & 1ull) {
            sacc.x += Gr[u * HS + r];
            sacc.y += Gi[u * HS + r];
          }
      } else {
        const uint32_t u = e - ob1;
        for (int r = 0; r < TR; ++r) {
          sacc.x += Gr[u * HS + r];
          sacc.y += Gi[u * HS + r];
        }
      }
      acc[e] = sacc;
    }
    __syncthreads();
  }
  float2* o = reinterpret_cast<float2*>(out + blockIdx.x * out_stride + m.qoff[i]);
  for (uint32_t e = tid; e < nc; e += NT) o[e] = acc[e];
}

__global__ void nade_partial_sum_kernel(const float* __restrict__ part, int G, uint64_t n, float* __restrict__ grad) {
  ANQS_PDL_ENTRY();
  for (uint64_t j = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < n; j += uint64_t(gridDim.x) * blockDim.x) {
    float s = 0.f;
    for (int g = 0; g < G; ++g) s += part[uint64_t(g) * n + j];
    grad[j] = s;
  }
}

// CTAs per qubit: over all 2n qubits about one CTA per SM for the tiled
// adjoint (widths 32, 64; tiles of 4096 / W rows), two for the one of width
// 128 (tiles of 256 / W rows); at most one per row tile
int grad_groups(const NadeView& m, uint64_t n_x) {
  const bool tiled = m.w <= 64;
  const uint64_t tr = tiled ? uint64_t(4096 / m.w) : uint64_t(NT / m.w);
  const uint64_t tiles = (n_x + tr - 1) / tr;
  uint64_t g = (tiled ? 152 : 2 * 152) / uint64_t(2 * m.n);
  if (g < 1) g = 1;
  if (g > tiles) g = tiles;
  return int(g < 1 ? 1 : g);
}

template <int W>
int grad_w(const NadeView& m, const HamView& hv, const uint64_t* x, Count n_x, const CotSrc& cot, float* grad,
           uint64_t n_params, float* part, cudaStream_t s) {
  const int G = grad_groups(m, n_x.n);
  float* out = G > 1 ? part : grad;
  if (G > 1 && !part) return set_error(ANQS_ERR_CAPACITY, "NADE adjoint needs its partial-sum workspace");
  ProfScope ps(PROF_NADE_GRAD, s);
  if constexpr (W <= 64) {
    const size_t smem = GradTile<W>::smem_bytes(m.n);
    ANQS_CUDA(cudaFuncSetAttribute(nade_grad_tile_kernel<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
    ANQS_CUDA_LAUNCH("nade_grad_tile_kernel", launch_k(nade_grad_tile_kernel<W>, dim3(G, 2 * m.n), dim3(NT), smem, s, m,
                                                       hv, x, n_x, cot, out, G > 1 ? n_params : uint64_t(0)));
  } else {
    const size_t smem = size_t(qubit_floats(W, 2 * m.n - 1)) * sizeof(float);
    ANQS_CUDA(cudaFuncSetAttribute(nade_grad_kernel<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
    ANQS_CUDA_LAUNCH("nade_grad_kernel", launch_k(nade_grad_kernel<W>, dim3(G, 2 * m.n), dim3(NT), smem, s, m, hv, x,
                                                  n_x, cot, out, G > 1 ? n_params : uint64_t(0)));
  }
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

int launch_nade_grad(const NadeView& m, const HamView& hv, const uint64_t* x, Count n_x, const CotSrc& cot,
                     float* grad, uint64_t n_params, float* part, cudaStream_t s) {
  if (n_x.n == 0) return ANQS_OK;
  switch (m.w) {
    case 32: return grad_w<32>(m, hv, x, n_x, cot, grad, n_params, part, s);
    case 64: return grad_w<64>(m, hv, x, n_x, cot, grad, n_params, part, s);
    case 128: return grad_w<128>(m, hv, x, n_x, cot, grad, n_params, part, s);
  }
  return set_error(ANQS_ERR_UNSUPPORTED, "NADE width %d", m.w);
}

}  // namespace anqs
