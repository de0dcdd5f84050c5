// Connected set of a determinant: single and double excitations that keep
// N_alpha and N_beta, with Jordan-Wigner signs and Slater-Condon elements
// (Eq. local_energy_def, Eq. sq_hamiltonian, Sec. IV.A).
//
// One thread per (determinant l, excitation k).  The excitation index k is
// unranked directly into the fixed order (alpha singles, beta singles,
// alpha-alpha doubles, beta-beta doubles, alpha-beta doubles), so that the
// output needs no sort and every row has the same length K.  Integer work
// (x', sign, first slot) is exact; matrix elements are FP64.
#include "common.cuh"

namespace anqs {
namespace {

__device__ __forceinline__ uint32_t spin_occ(uint64_t x, int s, int n) {
  uint32_t m = 0;
  for (int p = 0; p < n; ++p) m |= uint32_t((x >> (2 * p + s)) & 1ull) << p;
  return m;
}

// position of the r-th (0-based) set bit of m
__device__ __forceinline__ int nth_bit(uint32_t m, int r) {
  for (int i = 0; i < r; ++i) m &= m - 1;
  return __ffs(m) - 1;
}

// parity of the occupied spin-orbitals below q
__device__ __forceinline__ int par_below(uint64_t x, int q) {
  return __popcll(x & ((1ull << q) - 1ull)) & 1;
}

// unrank a pair (i < j) of an m-element list in lexicographic order
__device__ __forceinline__ void unrank_pair(uint32_t idx, int m, int& i, int& j) {
  i = 0;
  while (idx >= uint32_t(m - 1 - i)) {
    idx -= uint32_t(m - 1 - i);
    ++i;
  }
  j = i + 1 + int(idx);
}

__device__ __forceinline__ double G(const HamView& hv, int p, int q, int r, int s) {
  int n = hv.n;
  return __ldg(hv.g + ((size_t(p) * n + q) * n + r) * n + s);
}

// blocks bid = 0..nb-1 of a grid-stride loop over the (sample, excitation)
// pairs
__device__ __forceinline__ void connected_body(const HamView& hv, const uint64_t* __restrict__ xs, Count n_x,
                                               uint64_t* __restrict__ xp_out, double* __restrict__ h_out,
                                               uint8_t* __restrict__ j_out, uint64_t bid, uint64_t nb) {
  const uint64_t K = hv.K;
  const uint64_t total = n_x.get() * K;
  const int n = hv.n;
  for (uint64_t t = bid * blockDim.x + threadIdx.x; t < total; t += nb * blockDim.x) {
    uint64_t l;
    uint32_t k;
    if (total <= 0xffffffffull) {  // the usual case: a 32-bit division instead of a 64-bit one
      const uint32_t t32 = uint32_t(t), l32 = t32 / uint32_t(K);
      l = l32;
      k = t32 - l32 * uint32_t(K);
    } else {
      l = t / K;
      k = uint32_t(t - l * K);
    }
    uint64_t x = __ldg(xs + l);
    uint32_t oa = spin_occ(x, 0, n), ob = spin_occ(x, 1, n);
    uint32_t full = (n == 32) ? 0xffffffffu : ((1u << n) - 1u);
    bool ok = (__popc(oa) == hv.na) && (__popc(ob) == hv.nb) && (n == 32 || (x >> (2 * n)) == 0);
    if (!ok) {
      xp_out[t] = x;
      h_out[t] = __longlong_as_double(0x7ff8000000000000ll);
      if (j_out) j_out[t] = 255;
      continue;
    }
    uint32_t va = full & ~oa, vb = full & ~ob;
    uint64_t xn;
    double val;
    int jfirst;
    if (k < hv.nsa + hv.nsb) {
      // single I -> A of spin s: (h_ai + sum_{J occ} ([AI|JJ] - [AJ|JI])) <x'|a+_A a_I|x>
      int s = k < hv.nsa ? 0 : 1;
      uint32_t idx = s ? k - hv.nsa : k;
      int nv = n - (s ? hv.nb : hv.na);
      int i = nth_bit(s ? ob : oa, int(idx / nv));
      int a = nth_bit(s ? vb : va, int(idx % nv));
      int I = 2 * i + s, A = 2 * a + s;
      xn = x ^ (1ull << I) ^ (1ull << A);
      int lo = min(I, A), hi = max(I, A);
      uint64_t between = ((1ull << hi) - 1ull) & ~((2ull << lo) - 1ull);
      int sign = __popcll(x & between) & 1;
      double v = __ldg(hv.h + a * n + i);
      for (int t2 = 0; t2 < 2; ++t2)
        for (uint32_t m = t2 ? ob : oa; m; m &= m - 1) {
          int jj = __ffs(m) - 1;
          v += G(hv, a, i, jj, jj);
          if (t2 == s) v -= G(hv, a, jj, jj, i);
        }
      val = sign ? -v : v;
      jfirst = min(i, a);
    } else {
      uint32_t r = k - hv.nsa - hv.nsb;
      int I, J, A, B;
      double v;
      int i, j, a, b;
      if (r < hv.ndaa + hv.ndbb) {
        // same-spin double I<J -> A<B: [AI|BJ] - [AJ|BI]
        int s = r < hv.ndaa ? 0 : 1;
        uint32_t idx = s ? r - hv.ndaa : r;
        int ne = s ? hv.nb : hv.na, nv = n - ne;
        uint32_t nvp = uint32_t(nv) * (nv - 1) / 2;
        int ri, rj, ra, rb;
        unrank_pair(idx / nvp, ne, ri, rj);
        unrank_pair(idx % nvp, nv, ra, rb);
        uint32_t om = s ? ob : oa, vm = s ? vb : va;
        i = nth_bit(om, ri);
        j = nth_bit(om, rj);
        a = nth_bit(vm, ra);
        b = nth_bit(vm, rb);
        I = 2 * i + s;
        J = 2 * j + s;
        A = 2 * a + s;
        B = 2 * b + s;
        v = G(hv, a, i, b, j) - G(hv, a, j, b, i);
      } else {
        // opposite-spin double (I_a, A_a, I_b, A_b): [AI|BJ] (exchange term vanishes by spin)
        uint32_t idx = r - hv.ndaa - hv.ndbb;
        int nva = n - hv.na, nvb = n - hv.nb;
        int rab = int(idx % nvb);
        idx /= nvb;
        int rib = int(idx % hv.nb);
        idx /= hv.nb;
        int raa = int(idx % nva);
        int ria = int(idx / nva);
        i = nth_bit(oa, ria);
        a = nth_bit(va, raa);
        j = nth_bit(ob, rib);
        b = nth_bit(vb, rab);
        I = 2 * i;
        A = 2 * a;
        J = 2 * j + 1;
        B = 2 * b + 1;
        v = G(hv, a, i, b, j);
      }
      // sign of <x'| a+_A a+_B a_J a_I |x>, operators applied right to left
      uint64_t y = x;
      int sg = par_below(y, I);
      y ^= 1ull << I;
      sg ^= par_below(y, J);
      y ^= 1ull << J;
      sg ^= par_below(y, B);
      y ^= 1ull << B;
      sg ^= par_below(y, A);
      y ^= 1ull << A;
      xn = y;
      val = sg ? -v : v;
      jfirst = min(min(i, j), min(a, b));
    }
    xp_out[t] = xn;
    h_out[t] = val;
    if (j_out) j_out[t] = uint8_t(jfirst);
  }
}

// The tensor-core local energy's control words (TC_CTL_WORDS, optional) are
// zeroed by block 0 of the call's first kernel, on the stream of the kernels
// that use them (sort histogram, statistics ticket).
__device__ __forceinline__ void zero_ctl(uint32_t* ctl) {
  if (ctl && blockIdx.x == 0 && threadIdx.x < TC_CTL_WORDS) ctl[threadIdx.x] = 0u;
}

__global__ void connected_kernel(HamView hv, const uint64_t* __restrict__ xs, Count n_x,
                                 uint64_t* __restrict__ xp_out, double* __restrict__ h_out,
                                 uint8_t* __restrict__ j_out, uint32_t* __restrict__ ctl) {
  ANQS_PDL_ENTRY();
  zero_ctl(ctl);
  connected_body(hv, xs, n_x, xp_out, h_out, j_out, blockIdx.x, gridDim.x);
}

// <x|H|x> = E_nuc + sum_I h_ii + 1/2 sum_{I,J occ} ([II|JJ] - [IJ|JI]).
// One warp per determinant: lane i takes the occupied spin-orbital pairs
// (I, J) with I*N_occ + J = i mod 32, then the FP64 partial sums are reduced.
// one warp per sample, blocks bid = 0..nb-1
__device__ __forceinline__ void diagonal_body(const HamView& hv, const uint64_t* __restrict__ xs, Count n_x_,
                                              double* __restrict__ hdiag, uint64_t bid, uint64_t nb) {
  const int n = hv.n;
  const uint64_t n_x = n_x_.get();
  const int lane = threadIdx.x & 31;
  const uint64_t warps = nb * (blockDim.x >> 5);
  for (uint64_t l = bid * (blockDim.x >> 5) + (threadIdx.x >> 5); l < n_x; l += warps) {
    const uint64_t x = __ldg(xs + l);
    const uint32_t oa = spin_occ(x, 0, n), ob = spin_occ(x, 1, n);
    const bool ok = (__popc(oa) == hv.na) && (__popc(ob) == hv.nb) && (n == 32 || (x >> (2 * n)) == 0);
    // occupied spin-orbitals as (spatial index, spin)
    const int ne = hv.na + hv.nb;
    double e = 0.0;
    if (ok) {
      for (int t = lane; t < ne * ne + ne; t += 32) {
        if (t < ne * ne) {
          const int I = t / ne, J = t % ne;
          const int si = I < hv.na ? 0 : 1, sj = J < hv.na ? 0 : 1;
          const int i = nth_bit(si ? ob : oa, si ? I - hv.na : I);
          const int j = nth_bit(sj ? ob : oa, sj ? J - hv.na : J);
          e += 0.5 * G(hv, i, i, j, j);
          if (si == sj) e -= 0.5 * G(hv, i, j, j, i);
        } else {
          const int I = t - ne * ne;
          const int si = I < hv.na ? 0 : 1;
          const int i = nth_bit(si ? ob : oa, si ? I - hv.na : I);
          e += __ldg(hv.h + i * n + i);
        }
      }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
    if (lane == 0) hdiag[l] = ok ? hv.e_nuc + e : __longlong_as_double(0x7ff8000000000000ll);
  }
}

__global__ void diagonal_kernel(HamView hv, const uint64_t* __restrict__ xs, Count n_x, double* __restrict__ hdiag,
                                uint32_t* __restrict__ ctl) {
  ANQS_PDL_ENTRY();
  zero_ctl(ctl);
  diagonal_body(hv, xs, n_x, hdiag, blockIdx.x, gridDim.x);
}

// the connected set on blocks [0, nb_c) and the diagonal on the rest, in one
// launch
__global__ void connected_diag_kernel(HamView hv, const uint64_t* __restrict__ xs, Count n_x,
                                      uint64_t* __restrict__ xp_out, double* __restrict__ h_out,
                                      uint8_t* __restrict__ j_out, double* __restrict__ hdiag, unsigned nb_c,
                                      uint32_t* __restrict__ ctl) {
  ANQS_PDL_ENTRY();
  zero_ctl(ctl);
  if (blockIdx.x < nb_c) connected_body(hv, xs, n_x, xp_out, h_out, j_out, blockIdx.x, nb_c);
  else diagonal_body(hv, xs, n_x, hdiag, blockIdx.x - nb_c, gridDim.x - nb_c);
}

}  // namespace

int launch_connected(const HamView& hv, const uint64_t* x, Count n_x, uint64_t* xp, double* hval,
                     uint8_t* first_slot, double* hdiag, cudaStream_t s, uint32_t* ctl) {
  const int threads = 256;
  uint64_t total = n_x.n * hv.K;
  if (total && hdiag) {
    uint64_t bc = (total + threads - 1) / threads, bd = (n_x.n + 7) / 8;
    if (bc > 152ull * 64) bc = 152ull * 64;
    if (bd > 152ull * 16) bd = 152ull * 16;
    ProfScope ps(PROF_CONNECT, s);
    ANQS_CUDA_LAUNCH("connected_diag_kernel", launch_k(connected_diag_kernel, dim3(unsigned(bc + bd)), dim3(threads), 0, s, hv, x, n_x, xp, hval, first_slot, hdiag, unsigned(bc), ctl));
    return ANQS_OK;
  }
  if (total) {
    uint64_t blocks = (total + threads - 1) / threads;
    if (blocks > 152ull * 64) blocks = 152ull * 64;
    ProfScope ps(PROF_CONNECT, s);
    ANQS_CUDA_LAUNCH("connected_kernel", launch_k(connected_kernel, dim3(unsigned(blocks)), dim3(threads), 0, s, hv, x, n_x, xp, hval, first_slot, ctl));
    ctl = nullptr;
  }
  if (hdiag) {
    uint64_t blocks = (n_x.n + 7) / 8;  // 8 warps per CTA
    if (blocks > 152ull * 16) blocks = 152ull * 16;
    if (blocks == 0) blocks = 1;
    ProfScope ps(PROF_DIAGONAL, s);
    ANQS_CUDA_LAUNCH("diagonal_kernel", launch_k(diagonal_kernel, dim3(unsigned(blocks)), dim3(threads), 0, s, hv, x, n_x, hdiag, ctl));
  }
  return ANQS_OK;
}

}  // namespace anqs
