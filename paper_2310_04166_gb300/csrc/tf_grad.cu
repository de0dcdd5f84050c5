// Hand-written adjoint of the masked log psi for the causal-transformer
// ansatz (FP32): the VMC gradient of Eq. grad_def is the vector-Jacobian
// product of sum_l [cot_la_l log|psi(x_l)| + cot_ph_l arg psi(x_l)] with the
// cotangents 2 w_l Re(E_loc,l - E) and 2 w_l Im(E_loc,l - E).
//
// The unique samples are few (thousands) while each has n positions, so the
// adjoint runs as batched passes over all R = n_x * n rows (sample,
// position) with every activation of the forward stored in the workspace
// (or, when the workspace is too small for that, only the block inputs, each
// block's activations being recomputed from its input before its backward):
// embedding; per block LN1, q|k|v, causal attention (probabilities kept),
// output projection + residual, LN2, FFN (pre-activation kept) + residual;
// final LN and head.  The backward walks the same steps in reverse.  Matrix
// products go through one tiled SGEMM kernel (operands normal or transposed,
// optional bias, residual input, ReLU on an operand, ReLU'-mask of the
// result); weight gradients are products over the R rows, split along R
// across CTAs and accumulated with atomics into the flat gradient.
#include <cmath>

#include "common.cuh"

namespace anqs {
namespace {

constexpr int BM = 64, BN = 64, BK = 16, GT = 256;

struct Gm {
  const float* A;
  int lda;
  const float* B;
  int ldb;
  float* C;
  int ldc;
  const float* Cin;  // residual input (may alias C), or null
  int ldcin;
  const float* bias;  // per column, or null
  const float* mask;  // result zeroed where mask <= 0, or null
  int ldmask;
  Count M, K;  // M (rows) and K may be device counts
  int N;
  int relu_a, relu_b, atomic;
  uint64_t k_chunk;  // split-K: K range per blockIdx.z
};

// C[m][n] = sum_k opA(m, k) opB(k, n), opA(m, k) = A[m][k] (TA: A[k][m]),
// opB(k, n) = B[k][n] (TB: B[n][k]).  64 x 64 tile per CTA, 4 x 4 per thread.
template <bool TA, bool TB>
__global__ void __launch_bounds__(GT) sgemm_kernel(Gm g) {
  ANQS_PDL_ENTRY();
  __shared__ __align__(16) float As[BK][BM + 4];
  __shared__ __align__(16) float Bs[BK][BN + 4];
  const uint64_t M = g.M.get(), K = g.K.get();
  const uint64_t m0 = uint64_t(blockIdx.y) * BM;
  const int n0 = blockIdx.x * BN;
  if (m0 >= M) return;
  const uint64_t k_lo = uint64_t(blockIdx.z) * g.k_chunk;
  if (k_lo >= K && !(k_lo == 0)) return;
  const uint64_t k_hi = k_lo + g.k_chunk < K ? k_lo + g.k_chunk : K;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  float acc[4][4] = {};
  for (uint64_t k0 = k_lo; k0 < k_hi; k0 += BK) {
    // A tile: BM x BK elements, 4 per thread
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int e = threadIdx.x + GT * i;
      int mm, kk;
      if (TA) {  // consecutive threads along m
        mm = e % BM;
        kk = e / BM;
      } else {  // consecutive threads along k
        kk = e % BK;
        mm = e / BK;
      }
      const uint64_t m = m0 + mm, k = k0 + kk;
      float v = 0.f;
      if (m < M && k < k_hi) v = TA ? g.A[k * g.lda + m] : g.A[m * g.lda + k];
      if (g.relu_a) v = fmaxf(v, 0.f);
      As[kk][mm] = v;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int e = threadIdx.x + GT * i;
      int nn, kk;
      if (TB) {  // B[n][k]: consecutive threads along k
        kk = e % BK;
        nn = e / BK;
      } else {  // B[k][n]: consecutive threads along n
        nn = e % BN;
        kk = e / BN;
      }
      const int n = n0 + nn;
      const uint64_t k = k0 + kk;
      float v = 0.f;
      if (n < g.N && k < k_hi) v = TB ? g.B[uint64_t(n) * g.ldb + k] : g.B[k * g.ldb + n];
      if (g.relu_b) v = fmaxf(v, 0.f);
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      const float4 a = *reinterpret_cast<const float4*>(&As[kk][ty * 4]);
      const float4 b = *reinterpret_cast<const float4*>(&Bs[kk][tx * 4]);
      const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const uint64_t m = m0 + ty * 4 + i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx * 4 + j;
      if (n >= g.N) continue;
      float v = acc[i][j];
      if (g.atomic) {
        atomicAdd(g.C + m * g.ldc + n, v);
        continue;
      }
      if (g.bias) v += g.bias[n];
      if (g.Cin) v += g.Cin[m * g.ldcin + n];
      if (g.mask && !(g.mask[m * g.ldmask + n] > 0.f)) v = 0.f;
      g.C[m * g.ldc + n] = v;
    }
  }
}

// h0[r] = tok[token(r)] + pos[t], r = s n + t
__global__ void embed_kernel(TfView m, const uint64_t* __restrict__ x, Count rows_, float* __restrict__ h0) {
  ANQS_PDL_ENTRY();
  const uint64_t rows = rows_.get();
  const int D = m.d, n = m.n;
  const float* tok = m.params;
  const float* pos = m.params + 5 * size_t(D);
  for (uint64_t idx = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; idx < rows * D;
       idx += uint64_t(gridDim.x) * blockDim.x) {
    const uint64_t r = idx / D;
    const int c = int(idx % D), t = int(r % n);
    const uint64_t s = r / n;
    const int token = t == 0 ? 4 : int((x[s] >> (2 * (t - 1))) & 3ull);
    h0[idx] = tok[token * D + c] + pos[t * D + c];
  }
}

// y = xhat * g + b, xhat = (x - mean) rs, one warp per row; keeps xhat and rs
template <int D>
__global__ void ln_fwd_kernel(const float* __restrict__ X, const float* __restrict__ gam,
                              const float* __restrict__ bet, float* __restrict__ Xh, float* __restrict__ Y,
                              float* __restrict__ RS, Count rows_) {
  ANQS_PDL_ENTRY();
  constexpr int E = D / 32;
  const uint64_t rows = rows_.get();
  const int lane = threadIdx.x & 31;
  for (uint64_t r = (blockIdx.x * uint64_t(blockDim.x) + threadIdx.x) >> 5; r < rows;
       r += (uint64_t(gridDim.x) * blockDim.x) >> 5) {
    float v[E], s = 0.f;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      v[e] = X[r * D + lane + 32 * e];
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
    const float rs = 1.0f / sqrtf(q / float(D) + 1e-5f);
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int c = lane + 32 * e;
      const float xh = v[e] * rs;
      Xh[r * D + c] = xh;
      Y[r * D + c] = fmaf(xh, gam[c], bet[c]);
    }
    if (lane == 0) RS[r] = rs;
  }
}

// dX = dRes + rs (gy - mean(gy) - xhat mean(gy xhat)), gy = dY * g (dRes may
// alias dX or be null); dg += sum_r dY xhat, db += sum_r dY
template <int D>
__global__ void __launch_bounds__(256) ln_bwd_kernel(const float* __restrict__ dY, const float* __restrict__ Xh,
                                                     const float* __restrict__ gam, const float* __restrict__ RS,
                                                     const float* dRes, float* dX, float* __restrict__ dg,
                                                     float* __restrict__ db, Count rows_) {
  ANQS_PDL_ENTRY();
  constexpr int E = D / 32;
  __shared__ float s_dg[D], s_db[D];
  for (int c = threadIdx.x; c < D; c += blockDim.x) s_dg[c] = s_db[c] = 0.f;
  __syncthreads();
  const uint64_t rows = rows_.get();
  const int lane = threadIdx.x & 31;
  float pg[E] = {}, pb[E] = {};
  for (uint64_t r = (blockIdx.x * uint64_t(blockDim.x) + threadIdx.x) >> 5; r < rows;
       r += (uint64_t(gridDim.x) * blockDim.x) >> 5) {
    float dy[E], xh[E], gy[E], s1 = 0.f, s2 = 0.f;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int c = lane + 32 * e;
      dy[e] = dY[r * D + c];
      xh[e] = Xh[r * D + c];
      gy[e] = dy[e] * gam[c];
      s1 += gy[e];
      s2 = fmaf(gy[e], xh[e], s2);
      pg[e] = fmaf(dy[e], xh[e], pg[e]);
      pb[e] += dy[e];
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      s1 += __shfl_xor_sync(0xffffffffu, s1, o);
      s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    const float m1 = s1 / float(D), m2 = s2 / float(D), rs = RS[r];
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int c = lane + 32 * e;
      float v = rs * (gy[e] - m1 - xh[e] * m2);
      if (dRes) v += dRes[r * D + c];
      dX[r * D + c] = v;
    }
  }
#pragma unroll
  for (int e = 0; e < E; ++e) {
    atomicAdd(&s_dg[lane + 32 * e], pg[e]);
    atomicAdd(&s_db[lane + 32 * e], pb[e]);
  }
  __syncthreads();
  for (int c = threadIdx.x; c < D; c += blockDim.x) {
    atomicAdd(dg + c, s_dg[c]);
    atomicAdd(db + c, s_db[c]);
  }
}

// out[c] += sum_r X[r][c] for c < N
__global__ void __launch_bounds__(256) colsum_kernel(const float* __restrict__ X, int N, Count rows_,
                                                     float* __restrict__ out) {
  ANQS_PDL_ENTRY();
  const uint64_t rows = rows_.get();
  for (int c0 = 0; c0 < N; c0 += 256) {
    const int c = c0 + threadIdx.x;
    if (c >= N) break;
    float s = 0.f;
    for (uint64_t r = blockIdx.x; r < rows; r += gridDim.x) s += X[r * N + c];
    atomicAdd(out + c, s);
  }
}

// causal attention of one (sample, head, query t) per thread; keeps the
// probabilities P[s][h][t][u] (zero for u > t)
__global__ void attn_fwd_kernel(const float* __restrict__ Q, const float* __restrict__ Kt,
                                const float* __restrict__ V, float* __restrict__ P, float* __restrict__ O, int n,
                                int D, int H, Count nx_) {
  ANQS_PDL_ENTRY();
  const uint64_t nx = nx_.get();
  const int dh = D / H;
  const float scale = 1.0f / sqrtf(float(dh));
  for (uint64_t task = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; task < nx * H * n;
       task += uint64_t(gridDim.x) * blockDim.x) {
    const int t = int(task % n), hd = int((task / n) % H);
    const uint64_t s = task / (uint64_t(n) * H);
    const float* q = Q + (s * n + t) * D + hd * dh;
    float* prow = P + task * n;
    float mx = -INFINITY;
    for (int u = 0; u <= t; ++u) {
      const float* k = Kt + (s * n + u) * D + hd * dh;
      float dot = 0.f;
      for (int e = 0; e < dh; ++e) dot = fmaf(q[e], k[e], dot);
      prow[u] = dot * scale;
      mx = fmaxf(mx, dot * scale);
    }
    float sum = 0.f;
    for (int u = 0; u <= t; ++u) {
      const float p = expf(prow[u] - mx);
      prow[u] = p;
      sum += p;
    }
    const float inv = 1.0f / sum;
    for (int u = 0; u < n; ++u) prow[u] = u <= t ? prow[u] * inv : 0.f;
    float* o = O + (s * n + t) * D + hd * dh;
    for (int e = 0; e < dh; ++e) {
      float a = 0.f;
      for (int u = 0; u <= t; ++u) a = fmaf(prow[u], V[(s * n + u) * D + hd * dh + e], a);
      o[e] = a;
    }
  }
}

// backward of the attention of one (sample, head): dQ, dK, dV (written)
__global__ void attn_bwd_kernel(const float* __restrict__ Q, const float* __restrict__ Kt,
                                const float* __restrict__ V, const float* __restrict__ P,
                                const float* __restrict__ dO, float* __restrict__ dQ, float* __restrict__ dK,
                                float* __restrict__ dV, int n, int D, int H, Count nx_) {
  ANQS_PDL_ENTRY();
  const uint64_t nx = nx_.get();
  const int dh = D / H;
  const float scale = 1.0f / sqrtf(float(dh));
  for (uint64_t task = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; task < nx * H;
       task += uint64_t(gridDim.x) * blockDim.x) {
    const int hd = int(task % H);
    const uint64_t s = task / H;
    const uint64_t rb = s * n;
    for (int u = 0; u < n; ++u)
      for (int e = 0; e < dh; ++e) {
        dK[(rb + u) * D + hd * dh + e] = 0.f;
        dV[(rb + u) * D + hd * dh + e] = 0.f;
      }
    for (int t = 0; t < n; ++t) {
      const float* prow = P + (task * n + t) * n;
      const float* go = dO + (rb + t) * D + hd * dh;
      // dP_u = dO_t . V_u ; dS_u = P_u (dP_u - sum_u' P_u' dP_u')
      float dp[32];
      float dot = 0.f;
      for (int u = 0; u <= t; ++u) {
        float a = 0.f;
        for (int e = 0; e < dh; ++e) a = fmaf(go[e], V[(rb + u) * D + hd * dh + e], a);
        dp[u] = a;
        dot = fmaf(prow[u], a, dot);
      }
      const float* q = Q + (rb + t) * D + hd * dh;
      float* gq = dQ + (rb + t) * D + hd * dh;
      for (int e = 0; e < dh; ++e) gq[e] = 0.f;
      for (int u = 0; u <= t; ++u) {
        const float ds = prow[u] * (dp[u] - dot) * scale;
        const float* k = Kt + (rb + u) * D + hd * dh;
        float* gk = dK + (rb + u) * D + hd * dh;
        float* gv = dV + (rb + u) * D + hd * dh;
        for (int e = 0; e < dh; ++e) {
          gq[e] = fmaf(ds, k[e], gq[e]);
          gk[e] = fmaf(ds, q[e], gk[e]);
          gv[e] = fmaf(prow[u], go[e], gv[e]);
        }
      }
    }
  }
}

// head cotangents: d out8[r] from the masked log-softmax of every slot
__global__ void head_dout_kernel(HamView hv, const uint64_t* __restrict__ x, Count nx_,
                                 const float* __restrict__ out8, const float* __restrict__ cl,
                                 const float* __restrict__ cp, float* __restrict__ dout8, int n) {
  ANQS_PDL_ENTRY();
  const uint64_t nx = nx_.get();
  for (uint64_t s = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; s < nx; s += uint64_t(gridDim.x) * blockDim.x) {
    const uint64_t xs = x[s];
    bool dead = hv.n < 32 && (xs >> (2 * hv.n)) != 0;
    int ca = 0, cb = 0;
    for (int p = 0; p < n; ++p) {
      const int v = int((xs >> (2 * p)) & 3ull);
      if (!((slot_mask(hv, p, ca, cb, xs) >> v) & 1u)) dead = true;
      ca += v & 1;
      cb += v >> 1;
    }
    ca = cb = 0;
    for (int p = 0; p < n; ++p) {
      const int v = int((xs >> (2 * p)) & 3ull);
      const unsigned mk = norm_mask(hv, p, slot_mask(hv, p, ca, cb, xs));
      const float* o = out8 + (s * n + p) * 8;
      float* d = dout8 + (s * n + p) * 8;
      float mx = -INFINITY;
      for (int u = 0; u < 4; ++u)
        if ((mk >> u) & 1u) mx = fmaxf(mx, o[u]);
      float e[4], sum = 0.f;
      for (int u = 0; u < 4; ++u) {
        e[u] = ((mk >> u) & 1u) ? expf(o[u] - mx) : 0.f;
        sum += e[u];
      }
      for (int u = 0; u < 4; ++u) {
        const float pu = e[u] / sum;
        d[u] = dead ? 0.f : 0.5f * cl[s] * ((u == v ? 1.f : 0.f) - pu);
        d[4 + u] = (dead || u != v) ? 0.f : cp[s];
      }
      ca += v & 1;
      cb += v >> 1;
    }
  }
}

// gtok[token(r)] += dH0[r], gpos[t] += dH0[r]
__global__ void embed_bwd_kernel(TfView m, const uint64_t* __restrict__ x, Count rows_, const float* __restrict__ dh0,
                                 float* __restrict__ gtok, float* __restrict__ gpos) {
  ANQS_PDL_ENTRY();
  const uint64_t rows = rows_.get();
  const int D = m.d, n = m.n;
  for (uint64_t idx = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; idx < rows * D;
       idx += uint64_t(gridDim.x) * blockDim.x) {
    const uint64_t r = idx / D;
    const int c = int(idx % D), t = int(r % n);
    const int token = t == 0 ? 4 : int((x[r / n] >> (2 * (t - 1))) & 3ull);
    const float v = dh0[idx];
    atomicAdd(gtok + token * D + c, v);
    atomicAdd(gpos + t * D + c, v);
  }
}

// ---- host side ----------------------------------------------------------------

struct LayerOff {  // float offsets of one block's parameters within the flat layout
  size_t ln1_g, ln1_b, wq, bq, wk, bk, wv, bv, wo, bo, ln2_g, ln2_b, w1, b1, w2, b2;
};

LayerOff layer_off(const TfView& m, int l) {
  const size_t D = m.d, per = 12 * D * D + 13 * D;
  LayerOff o;
  o.ln1_g = 5 * D + size_t(m.n) * D + size_t(l) * per;
  o.ln1_b = o.ln1_g + D;
  o.wq = o.ln1_b + D;
  o.bq = o.wq + D * D;
  o.wk = o.bq + D;
  o.bk = o.wk + D * D;
  o.wv = o.bk + D;
  o.bv = o.wv + D * D;
  o.wo = o.bv + D;
  o.bo = o.wo + D * D;
  o.ln2_g = o.bo + D;
  o.ln2_b = o.ln2_g + D;
  o.w1 = o.ln2_b + D;
  o.b1 = o.w1 + 4 * D * D;
  o.w2 = o.b1 + 4 * D;
  o.b2 = o.w2 + 4 * D * D;
  return o;
}

struct Acts {
  float *H[17], *Xh1[16], *A1[16], *RS1[16], *Q[16], *K[16], *V[16], *P[16], *O[16], *Hm[16], *Xh2[16],
      *A2[16], *RS2[16], *F[16];
  float *Xhf, *Af, *RSf, *out8, *dout8, *dH, *dA, *dHm, *dF, *dQ, *dK, *dV, *dO;
};

// Full storage keeps every block's activations; with `ckpt` (activation
// recomputation) only the block inputs H[l] are kept and one set of block
// activations is shared by all blocks: the backward recomputes block l's
// forward from H[l] just before its own backward.
size_t plan(const TfView& m, uint64_t nx, Arena& Ar, Acts& a, bool ckpt = false) {
  const uint64_t R = nx * m.n, D = m.d;
  for (int l = 0; l <= m.L; ++l) a.H[l] = Ar.take<float>(R * D);
  for (int l = 0; l < (ckpt ? 1 : m.L); ++l) {
    a.Xh1[l] = Ar.take<float>(R * D);
    a.A1[l] = Ar.take<float>(R * D);
    a.RS1[l] = Ar.take<float>(R);
    a.Q[l] = Ar.take<float>(R * D);
    a.K[l] = Ar.take<float>(R * D);
    a.V[l] = Ar.take<float>(R * D);
    a.P[l] = Ar.take<float>(R * m.H * m.n);
    a.O[l] = Ar.take<float>(R * D);
    a.Hm[l] = Ar.take<float>(R * D);
    a.Xh2[l] = Ar.take<float>(R * D);
    a.A2[l] = Ar.take<float>(R * D);
    a.RS2[l] = Ar.take<float>(R);
    a.F[l] = Ar.take<float>(R * 4 * D);
  }
  for (int l = 1; ckpt && l < m.L; ++l) {
    a.Xh1[l] = a.Xh1[0], a.A1[l] = a.A1[0], a.RS1[l] = a.RS1[0], a.Q[l] = a.Q[0], a.K[l] = a.K[0];
    a.V[l] = a.V[0], a.P[l] = a.P[0], a.O[l] = a.O[0], a.Hm[l] = a.Hm[0], a.Xh2[l] = a.Xh2[0];
    a.A2[l] = a.A2[0], a.RS2[l] = a.RS2[0], a.F[l] = a.F[0];
  }
  a.Xhf = Ar.take<float>(R * D);
  a.Af = Ar.take<float>(R * D);
  a.RSf = Ar.take<float>(R);
  a.out8 = Ar.take<float>(R * 8);
  a.dout8 = Ar.take<float>(R * 8);
  a.dH = Ar.take<float>(R * D);
  a.dA = Ar.take<float>(R * D);
  a.dHm = Ar.take<float>(R * D);
  a.dF = Ar.take<float>(R * 4 * D);
  a.dQ = Ar.take<float>(R * D);
  a.dK = Ar.take<float>(R * D);
  a.dV = Ar.take<float>(R * D);
  a.dO = Ar.take<float>(R * D);
  return Ar.off;
}

unsigned grid_for(uint64_t work, int threads, uint64_t cap) {
  uint64_t b = (work + threads - 1) / threads;
  if (b > cap) b = cap;
  return unsigned(b ? b : 1);
}

// C (M x N) = op(A) op(B) with the options of Gm; M a row count (device or
// host), K given by Kc.  Weight products (atomic) split K over CTAs.
template <bool TA, bool TB>
int gemm(Gm g, uint64_t M_host, uint64_t K_host, cudaStream_t s) {
  const unsigned gx = unsigned((g.N + BN - 1) / BN), gy = unsigned((M_host + BM - 1) / BM);
  unsigned gz = 1;
  g.k_chunk = K_host ? K_host : 1;
  if (g.atomic) {
    const uint64_t tiles = uint64_t(gx) * gy;
    uint64_t want = (152 * 4 + tiles - 1) / tiles;
    const uint64_t max_split = (K_host + 255) / 256;  // at least 256 rows per split
    if (want > max_split) want = max_split;
    if (want < 1) want = 1;
    gz = unsigned(want);
    g.k_chunk = ((K_host + gz - 1) / gz + BK - 1) / BK * BK;
  }
  if (gy > 65535u) return set_error(ANQS_ERR_UNSUPPORTED, "too many rows for the transformer adjoint");
  ANQS_CUDA_LAUNCH("tf sgemm_kernel", launch_k(sgemm_kernel<TA, TB>, dim3(gx, gy, gz), dim3(GT), 0, s, g));
  return ANQS_OK;
}

int gemm_nt(const Gm& g, uint64_t M, uint64_t K, cudaStream_t s) { return gemm<false, true>(g, M, K, s); }
int gemm_nn(const Gm& g, uint64_t M, uint64_t K, cudaStream_t s) { return gemm<false, false>(g, M, K, s); }
int gemm_tn(const Gm& g, uint64_t M, uint64_t K, cudaStream_t s) { return gemm<true, false>(g, M, K, s); }

Gm mk(const float* A, int lda, const float* B, int ldb, float* C, int ldc, Count M, Count K, int N) {
  Gm g = {};
  g.A = A;
  g.lda = lda;
  g.B = B;
  g.ldb = ldb;
  g.C = C;
  g.ldc = ldc;
  g.M = M;
  g.K = K;
  g.N = N;
  return g;
}

template <int D>
int run(const TfView& m, const HamView& hv, const uint64_t* x, Count nx, const float* cl, const float* cp,
        float* grad, void* ws, size_t ws_bytes, cudaStream_t s) {
  Arena Ar(ws, ws_bytes);
  Acts a;
  plan(m, nx.n, Ar, a);
  bool ckpt = false;
  if (!Ar.fits()) {  // too little workspace for every activation: recompute each block's
    Arena Ac(ws, ws_bytes);
    plan(m, nx.n, Ac, a, true);
    if (!Ac.fits())
      return set_error(ANQS_ERR_CAPACITY, "transformer adjoint workspace needs %zu bytes (%zu with recomputation)",
                       Ar.off, Ac.off);
    ckpt = true;
  }
  const int n = m.n, L = m.L, H = m.H;
  const Count rows = scaled(nx, n);
  const uint64_t R = rows.n;
  const Count kD = host_count(D), k4D = host_count(4 * D), k8 = host_count(8);
  const float* P = m.params;
  ProfScope ps(PROF_TF_GRAD, s);
  const unsigned eg = grid_for(R * D, 256, 152 * 16), lg = grid_for(R * 32, 256, 152 * 16);
  ANQS_CUDA_LAUNCH("tf embed_kernel", launch_k(embed_kernel, dim3(eg), dim3(256), 0, s, m, x, rows, a.H[0]));
  // forward of block l from H[l]: its activations and H[l + 1] (deterministic,
  // so a recomputation reproduces them bit for bit)
  auto fwd_block = [&](int l) -> int {
    const LayerOff o = layer_off(m, l);
    ANQS_CUDA_LAUNCH("tf ln_fwd_kernel", launch_k(ln_fwd_kernel<D>, dim3(lg), dim3(256), 0, s, a.H[l], P + o.ln1_g,
                                                  P + o.ln1_b, a.Xh1[l], a.A1[l], a.RS1[l], rows));
    const float* Wqkv[3] = {P + o.wq, P + o.wk, P + o.wv};
    const float* bqkv[3] = {P + o.bq, P + o.bk, P + o.bv};
    float* qkv[3] = {a.Q[l], a.K[l], a.V[l]};
    for (int i = 0; i < 3; ++i) {
      Gm g = mk(a.A1[l], D, Wqkv[i], D, qkv[i], D, rows, kD, D);
      g.bias = bqkv[i];
      ANQS_TRY(gemm_nt(g, R, D, s));
    }
    ANQS_CUDA_LAUNCH("tf attn_fwd_kernel",
                     launch_k(attn_fwd_kernel, dim3(grid_for(nx.n * H * n, 128, 152 * 16)), dim3(128), 0, s,
                              a.Q[l], a.K[l], a.V[l], a.P[l], a.O[l], n, D, H, nx));
    {
      Gm g = mk(a.O[l], D, P + o.wo, D, a.Hm[l], D, rows, kD, D);
      g.bias = P + o.bo;
      g.Cin = a.H[l];
      g.ldcin = D;
      ANQS_TRY(gemm_nt(g, R, D, s));
    }
    ANQS_CUDA_LAUNCH("tf ln_fwd_kernel", launch_k(ln_fwd_kernel<D>, dim3(lg), dim3(256), 0, s, a.Hm[l], P + o.ln2_g,
                                                  P + o.ln2_b, a.Xh2[l], a.A2[l], a.RS2[l], rows));
    {
      Gm g = mk(a.A2[l], D, P + o.w1, D, a.F[l], 4 * D, rows, kD, 4 * D);
      g.bias = P + o.b1;
      ANQS_TRY(gemm_nt(g, R, D, s));
    }
    {
      Gm g = mk(a.F[l], 4 * D, P + o.w2, 4 * D, a.H[l + 1], D, rows, k4D, D);
      g.relu_a = 1;
      g.bias = P + o.b2;
      g.Cin = a.Hm[l];
      g.ldcin = D;
      ANQS_TRY(gemm_nt(g, R, 4 * D, s));
    }
    return ANQS_OK;
  };
  for (int l = 0; l < L; ++l) ANQS_TRY(fwd_block(l));
  const size_t tail = 5 * size_t(D) + size_t(n) * D + size_t(L) * (12 * size_t(D) * D + 13 * size_t(D));
  const size_t lnf_g = tail, lnf_b = tail + D, head_w = tail + 2 * D, head_b = tail + 10 * D;
  ANQS_CUDA_LAUNCH("tf ln_fwd_kernel", launch_k(ln_fwd_kernel<D>, dim3(lg), dim3(256), 0, s, a.H[L], P + lnf_g,
                                                P + lnf_b, a.Xhf, a.Af, a.RSf, rows));
  {
    Gm g = mk(a.Af, D, P + head_w, D, a.out8, 8, rows, kD, 8);
    g.bias = P + head_b;
    ANQS_TRY(gemm_nt(g, R, D, s));
  }
  ANQS_CUDA_LAUNCH("tf head_dout_kernel", launch_k(head_dout_kernel, dim3(grid_for(nx.n, 128, 152 * 8)), dim3(128), 0,
                                                   s, hv, x, nx, a.out8, cl, cp, a.dout8, n));
  // ---- backward ----
  const unsigned cg = grid_for(R, 64, 152 * 4);
  auto wgrad = [&](const float* dY, int ldy, const float* X, int ldx, int Mo, int Ni, float* gW, int relu_x) -> int {
    Gm g = mk(dY, ldy, X, ldx, gW, Ni, host_count(Mo), rows, Ni);
    g.relu_b = relu_x;
    g.atomic = 1;
    return gemm_tn(g, Mo, R, s);
  };
  auto colsum = [&](const float* X, int N, float* out) -> int {
    ANQS_CUDA_LAUNCH("tf colsum_kernel", launch_k(colsum_kernel, dim3(cg), dim3(256), 0, s, X, N, rows, out));
    return ANQS_OK;
  };
  ANQS_TRY(wgrad(a.dout8, 8, a.Af, D, 8, D, grad + head_w, 0));
  ANQS_TRY(colsum(a.dout8, 8, grad + head_b));
  {
    Gm g = mk(a.dout8, 8, P + head_w, D, a.dA, D, rows, k8, D);
    ANQS_TRY(gemm_nn(g, R, 8, s));
  }
  ANQS_CUDA_LAUNCH("tf ln_bwd_kernel",
                   launch_k(ln_bwd_kernel<D>, dim3(lg), dim3(256), 0, s, a.dA, a.Xhf, P + lnf_g, a.RSf,
                            (const float*)nullptr, a.dH, grad + lnf_g, grad + lnf_b, rows));
  for (int l = L - 1; l >= 0; --l) {
    const LayerOff o = layer_off(m, l);
    if (ckpt && l + 1 < L) ANQS_TRY(fwd_block(l));  // the shared activations hold block L-1's after the forward
    ANQS_TRY(wgrad(a.dH, D, a.F[l], 4 * D, D, 4 * D, grad + o.w2, 1));
    ANQS_TRY(colsum(a.dH, D, grad + o.b2));
    {
      Gm g = mk(a.dH, D, P + o.w2, 4 * D, a.dF, 4 * D, rows, kD, 4 * D);
      g.mask = a.F[l];
      g.ldmask = 4 * D;
      ANQS_TRY(gemm_nn(g, R, D, s));
    }
    ANQS_TRY(wgrad(a.dF, 4 * D, a.A2[l], D, 4 * D, D, grad + o.w1, 0));
    ANQS_TRY(colsum(a.dF, 4 * D, grad + o.b1));
    {
      Gm g = mk(a.dF, 4 * D, P + o.w1, D, a.dA, D, rows, k4D, D);
      ANQS_TRY(gemm_nn(g, R, 4 * D, s));
    }
    ANQS_CUDA_LAUNCH("tf ln_bwd_kernel", launch_k(ln_bwd_kernel<D>, dim3(lg), dim3(256), 0, s, a.dA, a.Xh2[l],
                                                  P + o.ln2_g, a.RS2[l], (const float*)a.dH, a.dHm, grad + o.ln2_g,
                                                  grad + o.ln2_b, rows));
    ANQS_TRY(wgrad(a.dHm, D, a.O[l], D, D, D, grad + o.wo, 0));
    ANQS_TRY(colsum(a.dHm, D, grad + o.bo));
    {
      Gm g = mk(a.dHm, D, P + o.wo, D, a.dO, D, rows, kD, D);
      ANQS_TRY(gemm_nn(g, R, D, s));
    }
    ANQS_CUDA_LAUNCH("tf attn_bwd_kernel",
                     launch_k(attn_bwd_kernel, dim3(grid_for(nx.n * H, 64, 152 * 16)), dim3(64), 0, s, a.Q[l], a.K[l],
                              a.V[l], a.P[l], a.dO, a.dQ, a.dK, a.dV, n, D, H, nx));
    const float* dqkv[3] = {a.dQ, a.dK, a.dV};
    const size_t wo3[3] = {o.wq, o.wk, o.wv}, bo3[3] = {o.bq, o.bk, o.bv};
    for (int i = 0; i < 3; ++i) {
      ANQS_TRY(wgrad(dqkv[i], D, a.A1[l], D, D, D, grad + wo3[i], 0));
      ANQS_TRY(colsum(dqkv[i], D, grad + bo3[i]));
      Gm g = mk(dqkv[i], D, P + wo3[i], D, a.dA, D, rows, kD, D);
      if (i) {
        g.Cin = a.dA;
        g.ldcin = D;
      }
      ANQS_TRY(gemm_nn(g, R, D, s));
    }
    ANQS_CUDA_LAUNCH("tf ln_bwd_kernel", launch_k(ln_bwd_kernel<D>, dim3(lg), dim3(256), 0, s, a.dA, a.Xh1[l],
                                                  P + o.ln1_g, a.RS1[l], (const float*)a.dHm, a.dH, grad + o.ln1_g,
                                                  grad + o.ln1_b, rows));
  }
  ANQS_CUDA_LAUNCH("tf embed_bwd_kernel", launch_k(embed_bwd_kernel, dim3(eg), dim3(256), 0, s, m, x, rows, a.dH,
                                                   grad, grad + 5 * size_t(D)));
  return ANQS_OK;
}

}  // namespace

size_t tf_grad_workspace(const TfView& m, uint64_t n_x, bool recompute) {
  Arena Ar(nullptr, 0);
  Acts a;
  return plan(m, n_x, Ar, a, recompute);
}

int launch_tf_fp32_grad(const TfView& m, const HamView& hv, const uint64_t* x, Count n_x, const float* cl,
                        const float* cp, float* grad, void* ws, size_t ws_bytes, cudaStream_t s) {
  if (n_x.n == 0) return ANQS_OK;
  if (m.n > 32) return set_error(ANQS_ERR_UNSUPPORTED, "n_orb %d", m.n);
  switch (m.d) {
    case 32: return run<32>(m, hv, x, n_x, cl, cp, grad, ws, ws_bytes, s);
    case 64: return run<64>(m, hv, x, n_x, cl, cp, grad, ws, ws_bytes, s);
    case 128: return run<128>(m, hv, x, n_x, cl, cp, grad, ws, ws_bytes, s);
    case 256: return run<256>(m, hv, x, n_x, cl, cp, grad, ws, ws_bytes, s);
  }
  return set_error(ANQS_ERR_UNSUPPORTED, "d_model %d", m.d);
}

}  // namespace anqs
