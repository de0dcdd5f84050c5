// Internal declarations shared by the libanqs translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstddef>
#include <utility>
#include <vector>

#include "anqs.h"

#define ANQS_MAX_ORB 32

namespace anqs {

int set_error(int code, const char* fmt, ...);
int cuda_error(cudaError_t e, const char* what, const char* file, int line);
void note_launch();

// Kernel families timed by the optional event profiler (anqs_profile_*).
enum ProfId {
  PROF_CONNECT = 0,
  PROF_DIAGONAL,
  PROF_MLP_FP32_LOGPSI,
  PROF_MLP_FP32_SLOT,
  PROF_MLP_FP32_GRAD,
  PROF_TABLE,
  PROF_ELOC_SUM,
  PROF_STATS,
  PROF_COTANGENT,
  PROF_SAMPLER,
  PROF_TC_PARENT,
  PROF_TC_SUFFIX,
  PROF_TC_SORT,
  PROF_TC_ELOC,
  PROF_TC_SLOT,
  PROF_TF,
  PROF_TC_FINALIZE,
  PROF_GRAD_REDUCE,
  PROF_SAMPLER_NET_FP32,
  PROF_TF_GRAD,
  PROF_TF_TC_PARENT,
  PROF_TF_TC_SUFFIX,
  PROF_TF_TC_SLOT,
  PROF_NADE,
  PROF_NADE_GRAD,
  PROF_NADE_SLOT,
  PROF_NADE_PARENT,
  PROF_NADE_SUFFIX,
  PROF_MLP_TC_GRAD,
  PROF_COUNT
};

// Records a pair of CUDA events around the launches in its scope when the
// profiler is on (no-op otherwise).
struct ProfScope {
  ProfScope(int id, cudaStream_t s);
  ~ProfScope();
  int id;
  cudaStream_t stream;
  cudaEvent_t start;
};

}  // namespace anqs

#define ANQS_CUDA(call)                                                  \
  do {                                                                   \
    cudaError_t e_ = (call);                                             \
    if (e_ != cudaSuccess) return anqs::cuda_error(e_, #call, __FILE__, __LINE__); \
  } while (0)

#define ANQS_CUDA_LAUNCH(what, call)                                     \
  do {                                                                   \
    cudaError_t e_ = (call);                                             \
    if (e_ != cudaSuccess) return anqs::cuda_error(e_, what, __FILE__, __LINE__); \
  } while (0)

#define ANQS_LAUNCHED(what)                                              \
  do {                                                                   \
    anqs::note_launch();                                                 \
    cudaError_t e_ = cudaGetLastError();                                 \
    if (e_ != cudaSuccess) return anqs::cuda_error(e_, what, __FILE__, __LINE__); \
  } while (0)

// Programmatic dependent launch: every library kernel waits for the
// previous kernel in the stream to complete (and its writes to be visible)
// before it reads anything, and only then lets the next kernel be scheduled.
// So the part of a kernel placed before ANQS_PDL_WAIT() (its prologue) runs
// while the previous kernel may still execute, but after the kernel before
// that has completed: a prologue may read data written two or more kernels
// earlier and set up TMEM and shared memory.  The weight-packing kernels do
// not trigger at all (their dependents start when they have completed), so a
// prologue may always read packed weight images.
#define ANQS_PDL_TRIGGER() asm volatile("griddepcontrol.launch_dependents;" ::: "memory")
#define ANQS_PDL_WAIT() asm volatile("griddepcontrol.wait;" ::: "memory")
#define ANQS_PDL_ENTRY() \
  do {                   \
    ANQS_PDL_WAIT();     \
    ANQS_PDL_TRIGGER();  \
  } while (0)

#define ANQS_TRY(expr)            \
  do {                            \
    int r_ = (expr);              \
    if (r_ != ANQS_OK) return r_; \
  } while (0)

// Number of rows of a call: a host value, or (when dev is set) a value that
// lives on the device (times mult), so that calls can be captured in a CUDA
// graph without knowing e.g. the number of unique samples on the host.  n
// always bounds the device value and sizes grids and workspaces.
struct Count {
  uint64_t n;
  const uint64_t* dev;
  uint64_t mult;
#ifdef __CUDACC__
  __device__ __forceinline__ uint64_t get() const { return dev ? *dev * mult : n; }
#endif
};
inline Count host_count(uint64_t n) { return Count{n, nullptr, 1}; }
inline Count scaled(const Count& c, uint64_t k) { return Count{c.n * k, c.dev, c.mult * k}; }

#ifdef __CUDACC__
// Count-weighted statistics of a sample set (Eq. energy_est): S = sum_l n_l,
// E = sum_l n_l E_loc(l) / S (complex) and Var = sum_l n_l |E_loc(l) - E|^2 / S
// over the rows l < n_x, written as stats = {Re E, Im E, Var, S}.  One CTA of
// NT threads, one pass over the rows with the shift K = E_loc(0):
//   A = sum_l n_l (E_loc(l) - K),  Q = sum_l n_l |E_loc(l) - K|^2,
//   E = K + A / S,  Var = Q / S - |A / S|^2  (clamped at 0),
// which equals the two-pass form up to rounding (the shift keeps |A / S| of
// the order of the spread, so the difference loses no significant digits).
// The reduction order is fixed (strided per-thread sums with RPT rows' loads
// issued together, a shuffle tree per warp, the warps' partials in warp order):
// the result is deterministic.  The loads go through L2, so a caller may
// reduce rows that other CTAs of its own grid wrote (after a fence).
template <int NT>
__device__ void cta_energy_stats(const double* ere, const double* eim, const uint64_t* counts, uint64_t n_x,
                                 double* stats) {
  constexpr int RPT = 4;
  __shared__ double red[4][NT / 32];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned long long* cnt = reinterpret_cast<const unsigned long long*>(counts);
  const double kr = n_x ? __ldcg(ere) : 0.0, ki = n_x ? __ldcg(eim) : 0.0;
  double cs = 0.0, ar = 0.0, ai = 0.0, q = 0.0;  // counts below 2^53 add exactly in FP64
  for (uint64_t l0 = 0; l0 < n_x; l0 += uint64_t(NT) * RPT) {
    double c[RPT], er[RPT], ei[RPT];
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      const uint64_t l = l0 + uint64_t(r) * NT + threadIdx.x;
      const bool in = l < n_x;
      c[r] = in ? double(__ldcg(cnt + l)) : 0.0;
      er[r] = in ? __ldcg(ere + l) : kr;
      ei[r] = in ? __ldcg(eim + l) : ki;
    }
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      const double dr = er[r] - kr, di = ei[r] - ki;
      cs += c[r];
      ar = fma(c[r], dr, ar);
      ai = fma(c[r], di, ai);
      q = fma(c[r], fma(dr, dr, di * di), q);
    }
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    cs += __shfl_xor_sync(0xffffffffu, cs, o);
    ar += __shfl_xor_sync(0xffffffffu, ar, o);
    ai += __shfl_xor_sync(0xffffffffu, ai, o);
    q += __shfl_xor_sync(0xffffffffu, q, o);
  }
  if (lane == 0) {
    red[0][w] = cs;
    red[1][w] = ar;
    red[2][w] = ai;
    red[3][w] = q;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double S = 0.0, tr = 0.0, ti = 0.0, tq = 0.0;
    for (int k = 0; k < NT / 32; ++k) {
      S += red[0][k];
      tr += red[1][k];
      ti += red[2][k];
      tq += red[3][k];
    }
    const double mr = tr / S, mi = ti / S;
    stats[0] = kr + mr;
    stats[1] = ki + mi;
    stats[2] = fmax(0.0, tq / S - fma(mr, mr, mi * mi));
    stats[3] = S;
  }
}
#endif

// Control words of one tensor-core local-energy call, in its workspace: the
// histogram of the connected rows' first differing slots (the sort), the
// sort's ticket and the assembly's statistics ticket.  The call's connected-set
// kernel zeroes them, so the later kernels of the call need no memset.
constexpr int TC_CTL_WORDS = ANQS_MAX_ORB + 2;
constexpr int TC_CTL_SORT_TICKET = ANQS_MAX_ORB;
constexpr int TC_CTL_STATS_TICKET = ANQS_MAX_ORB + 1;

// Where the local-energy assembly writes the statistics of the sample set
// (counts null: none).  ticket is a zeroed word (TC_CTL_STATS_TICKET); the
// assembly's CTAs take a ticket each when their rows are written and the last
// one reduces.
struct StatsOut {
  const uint64_t* counts;
  double* stats;
  uint32_t* ticket;
};

// Hamiltonian as seen by the kernels (passed by value).
struct HamView {
  int n, na, nb;
  uint32_t nsa, nsb, ndaa, ndbb, ndab;  // sizes of the five excitation blocks
  uint32_t K;                           // off-diagonal connected per determinant
  double e_nuc;
  const double* h;     // [n][n]
  const double* g;     // [n][n][n][n] chemist notation
  const uint8_t* mask; // [n][na+1][nb+1] allowed-outcome bits per slot and prefix counts
  int mu_lv;           // slots p < mu_lv are masked (MU), slots p >= mu_lv discard (DU): MU-d, d = n - mu_lv
  int nz;              // Z2 symmetries (Pauli-Z strings commuting with H), 0..ANQS_MAX_Z2
  uint64_t zmask[4];   // their qubit supports (bit q = qubit q)
  unsigned* status;    // sampler events (ANQS_HAM_* bits of anqs.h), set with atomicOr
};

// slot mask table entry of (slot p, a alpha and b beta electrons, Z2 parity
// bits z of the prefix)
__host__ __device__ inline int mask_index(const HamView& hv, int p, int a, int b, int z = 0) {
  return ((p * (hv.na + 1) + a) * (hv.nb + 1) + b) * (1 << hv.nz) + z;
}

#ifdef __CUDACC__
// Allowed-outcome bits of slot p after the prefix (slots < p) of x holding a
// alpha and b beta electrons (0 if the counts already leave the sector); the
// Z2 parities of the prefix select the entry when Z2 symmetries are set.
__device__ __forceinline__ unsigned slot_mask(const HamView& hv, int p, int a, int b, uint64_t x) {
  if (a > hv.na || b > hv.nb) return 0u;
  int z = 0;
  if (hv.nz) {
    const uint64_t pm = p >= 32 ? ~0ull : ((1ull << (2 * p)) - 1ull);
    for (int j = 0; j < hv.nz; ++j) z |= (__popcll(x & pm & hv.zmask[j]) & 1) << j;
  }
  return hv.mask[mask_index(hv, p, a, b, z)];
}

// Outcomes over which slot p's conditional is normalised (Sec. III.C): the
// allowed ones on MU levels (p < mu_lv), all four on DU levels, where samples
// that go to an unphysical child are discarded.
__device__ __forceinline__ unsigned norm_mask(const HamView& hv, int p, unsigned phys) {
  return p < hv.mu_lv ? phys : 0xFu;
}
#endif

// Cotangents of an adjoint: the given arrays cl, cp (log|psi|, arg psi per
// row), or, when stats is set, those of the VMC gradient computed per row:
// 2 (n_l / S) Re(E_loc,l - E) and 2 (n_l / S) Im(E_loc,l - E).
struct CotSrc {
  const float *cl, *cp;
  const double *ere, *eim, *stats;
  const uint64_t* counts;
};
#ifdef __CUDACC__
__device__ __forceinline__ void cot_of(const CotSrc& c, uint64_t l, float& a, float& b) {
  if (c.stats) {
    const double w = double(c.counts[l]) / c.stats[3];
    a = float(2.0 * w * (c.ere[l] - c.stats[0]));
    b = float(2.0 * w * (c.eim[l] - c.stats[1]));
  } else {
    a = c.cl[l];
    b = c.cp[l];
  }
}
#endif

// MLP parameters as seen by the kernels.
struct MlpView {
  int n, width, n_hidden;
  const float* params;
  uint32_t slot_off[ANQS_MAX_ORB + 1];
};

// Transformer parameters as seen by the kernels.
struct TfView {
  int n, d, H, L;
  const float* params;
};

// Per-qubit NADE parameters as seen by the kernels: qubit i's block
// (W1, b1, W2, b2, W3, b3, complex interleaved) starts at params + qoff[i].
struct NadeView {
  int n, w;
  const float* params;
  uint32_t qoff[2 * ANQS_MAX_ORB];
};

// Bump allocator over a caller-provided workspace; with base == nullptr it
// only measures.
struct Arena {
  char* base;
  size_t off, cap;
  explicit Arena(void* b, size_t c) : base(static_cast<char*>(b)), off(0), cap(c) {}
  template <class T>
  T* take(size_t count) {
    off = (off + 255) & ~size_t(255);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
  bool fits() const { return off <= cap; }
};

struct anqs_ham {
  int device;
  HamView v;
  uint64_t sector_dim;
  std::vector<uint8_t> mask_host;
  std::vector<uint64_t> phys_prefix;  // [p] physical prefixes holding slots < p (saturated)
  // Every physical prefix of the levels 0..n-1 when there are few (the
  // sampler's prefix table): prefixes of level p at [pt_off[p], pt_off[p+1])
  // in the order the sampler emits them, and per (prefix, outcome) the index
  // of the child prefix in the next level (-1: unphysical, or the last level).
  // Empty when the sector has too many prefixes.
  std::vector<uint64_t> pt_x;
  std::vector<uint32_t> pt_off;
  std::vector<int32_t> pt_child;
  uint64_t* d_pt_x;
  int32_t* d_pt_child;
  unsigned* d_status;  // HamView::status
  double* d_h;
  double* d_g;
  uint8_t* d_mask;
};

struct anqs_model {
  anqs_model_desc d;
  int device;
  const float* params;
  uint64_t n_params;
  MlpView mlp;
  TfView tf;
  NadeView nade;
  // BF16 form: packed weight images (see mlp_tc.cu)
  void* packed;
  size_t packed_bytes;
  std::vector<uint64_t> pack_off;  // per slot byte offset of its image
  float* tc_raw;                   // BF16 form: raw slot outputs of one chunk of anqs_logpsi rows
  uint64_t tc_raw_rows;
  // BF16 MLP: a second stream and its fork and join events, so that one local
  // energy call runs the parents' slots beside the connected set and its sort
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
};

// ---- launchers implemented in the kernel translation units ----
namespace anqs {

// Launch with the programmatic-stream-serialization attribute (see
// ANQS_PDL_ENTRY); counts the launch and reports launch errors.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t stream,
                            Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  note_launch();
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}


// connect.cu
// ctl (optional): a tensor-core local energy's control words, set to zero
int launch_connected(const HamView& hv, const uint64_t* x, Count n_x, uint64_t* xp, double* hval,
                     uint8_t* first_slot, double* hdiag, cudaStream_t s, uint32_t* ctl = nullptr);

// mlp_fp32.cu
int launch_mlp_fp32_logpsi(const MlpView& m, const HamView& hv, const uint64_t* x, Count n_x,
                           float* la, float* ph, cudaStream_t s);
int launch_mlp_fp32_slot_logits(const MlpView& m, int p, const uint64_t* prefixes,
                                const uint64_t* n_rows_dev, uint64_t max_rows, float* out8,
                                cudaStream_t s);
// part: per-tile partial gradients (mlp_fp32_grad_partial_floats floats) or
// null for atomic accumulation into grad (which must then be zeroed)
int launch_grad_partial_sum(const float* part, Count n_x, uint64_t n_params, int rows_per_tile, float* g,
                            cudaStream_t s);
bool mlp_tc_grad_supported(const anqs_model* M);
int launch_mlp_tc_grad(const anqs_model* M, const HamView& hv, const uint64_t* x, Count n_x, const CotSrc& cot,
                       float* grad, float* part, cudaStream_t s);
int launch_mlp_fp32_grad(const MlpView& m, const HamView& hv, const uint64_t* x, Count n_x, const CotSrc& cot,
                         float* grad, float* part, cudaStream_t s);
size_t mlp_fp32_grad_partial_floats(const MlpView& m, uint64_t n_x);

// table.cu
int launch_tf_fp32_logpsi(const TfView& m, const HamView& hv, const uint64_t* x, Count n_x, float* la, float* ph,
                          cudaStream_t s);
int launch_tf_fp32_slot_logits(const TfView& m, int p, const uint64_t* pre, const uint64_t* nr, uint64_t max_rows,
                               float* out, cudaStream_t s);
size_t tf_grad_workspace(const TfView& m, uint64_t n_x, bool recompute);  // recompute: block inputs only
int launch_tf_fp32_grad(const TfView& m, const HamView& hv, const uint64_t* x, Count n_x, const float* cl,
                        const float* cp, float* grad, void* ws, size_t ws_bytes, cudaStream_t s);
int launch_table_logpsi(const anqs_model* md, const HamView& hv, const uint64_t* x, Count n_x,
                        float* la, float* ph, cudaStream_t s);
int launch_table_slot_logits(const anqs_model* md, int p, const uint64_t* prefixes,
                             const uint64_t* n_rows_dev, uint64_t max_rows, float* out8,
                             cudaStream_t s);

// eloc.cu
int launch_eloc_sum(const HamView& hv, Count n_x, const double* hval, const double* hdiag,
                    const float* la_x, const float* ph_x, const float* la_p, const float* ph_p,
                    double* ere, double* eim, cudaStream_t s);
int launch_stats_combine(const double* in, int world, double* out, cudaStream_t s);
int launch_stats(const double* ere, const double* eim, const uint64_t* counts, Count n_x,
                 double* stats, cudaStream_t s);
int launch_grad_cotangents(const double* ere, const double* eim, const uint64_t* counts,
                           const double* stats, Count n_x, float* cot_la, float* cot_ph,
                           cudaStream_t s);

// mlp_tc.cu (BF16 tensor-core form)
int mlp_tc_pack_alloc(anqs_model* m);
int mlp_tc_pack(anqs_model* m, cudaStream_t s);
size_t eloc_tc_workspace(const anqs_model* M, const anqs_ham* H, uint64_t n_x);
// 16-bit MLP local energy in stages (pre: connected set, parents, sort; post:
// assembly) and the suffix stage of many problems in one persistent launch
struct MultiEloc {
  const anqs_model* model;
  const anqs_ham* ham;
  uint64_t n_x;  // the host bound of the problem's rows (workspace layout)
  void* ws;
  size_t ws_bytes;
};
// fork: run the parents' slots and finalize on the model's second stream,
// beside the connected set and the sort (joined back into s before returning)
int eloc_tc_pre(const anqs_model* M, const anqs_ham* H, const uint64_t* x, Count n_x, void* ws, size_t ws_bytes,
                cudaStream_t s, bool fork = false);
int eloc_tc_post(const anqs_ham* H, Count n_x, double* ere, double* eim, const uint64_t* counts, double* stats,
                 void* ws, size_t ws_bytes, cudaStream_t s);
int mlp_tc_multi_max();
size_t mlp_tc_multi_groups_bytes();
int launch_mlp_tc_multi(const MultiEloc* q, int n, int chunk, int dynamic, void* groups, uint32_t* ctl,
                        cudaStream_t s);
int run_eloc_tc(const anqs_model* M, const anqs_ham* H, const uint64_t* x, Count n_x, double* ere,
                double* eim, const uint64_t* counts, double* stats, void* ws, size_t ws_bytes, cudaStream_t s);
int launch_mlp_tc_logpsi(const anqs_model* M, const HamView& hv, const uint64_t* x, uint64_t n_x, float* la,
                         float* ph, cudaStream_t s);
int launch_mlp_tc_slot_logits(const anqs_model* M, const HamView& hv, int p, const uint64_t* pre,
                              const uint64_t* n_dev, uint64_t max_rows, float* out8, cudaStream_t s);
// slot-p outputs of every prefix of the prefix table (level p's rows use slot p), one launch
// Words that a launch sets to zero (block 0, after its dependency wait), for
// the kernel after it: up to two ranges of 32-bit words.
struct ZeroWords {
  uint32_t* p[2];
  int n[2];
};
int launch_mlp_tc_prefix_logits(const anqs_model* M, const anqs_ham* H, float* out8, cudaStream_t s,
                                ZeroWords zero = ZeroWords{});
int mlp_tc_status(const anqs_model* M, int* status);
// pieces of the tensor-core local-energy pipeline shared by the MLP and transformer forms
constexpr int TC_CACHE_F = 10;  // floats per (parent, slot): prefix la, ph, 4 masked terms, 4 phases
int launch_tc_finalize(const HamView& hv, const uint64_t* x, Count n_x, const float* raw, float* la, float* ph,
                       float* cache, cudaStream_t s);
// ctl: the call's control words, zeroed by the connected-set kernel before it
int launch_js_sort(const uint8_t* js, Count mc, int n, uint32_t* ctl, uint32_t* cursor, uint32_t* offsets,
                   uint32_t* perm, cudaStream_t s);
int launch_eloc_assemble(int n, uint32_t K, Count n_x, const uint64_t* xp, const uint8_t* js, const float* cache,
                         const float2* T, const double* hval, const double* hdiag, const float* la_x,
                         const float* ph_x, double* ere, double* eim, const StatsOut& so, cudaStream_t s,
                         bool tsum = false);
// BF16 transformer form
int tf_tc_pack_alloc(anqs_model* m);
int tf_tc_pack(anqs_model* m, cudaStream_t s);
int tf_tc_status(const anqs_model* M, int* status);
size_t tf_tc_eloc_workspace(const anqs_model* M, const anqs_ham* H, uint64_t n_x);
int run_eloc_tf_tc(const anqs_model* M, const anqs_ham* H, const uint64_t* x, Count n_x, double* ere, double* eim,
                   const uint64_t* counts, double* stats, void* ws, size_t ws_bytes, cudaStream_t s);
int launch_tf_tc_logpsi(const anqs_model* M, const HamView& hv, const uint64_t* x, uint64_t n_x, float* la,
                        float* ph, cudaStream_t s);
int launch_tf_tc_slot_logits(const anqs_model* M, int p, const uint64_t* pre, const uint64_t* n_dev,
                             uint64_t max_rows, float* out8, cudaStream_t s);

// nade.cu (per-qubit NADE, FP32)
int launch_nade_logpsi(const NadeView& m, const HamView& hv, const uint64_t* x, Count n_x, float* la, float* ph,
                       cudaStream_t s);
int launch_nade_slot_logits(const NadeView& m, const HamView& hv, int p, const uint64_t* pre, const uint64_t* n_dev,
                            uint64_t max_rows, float* out8, cudaStream_t s);
// part: nade_grad_partial_floats floats (null when that is 0); grad is overwritten
int launch_nade_grad(const NadeView& m, const HamView& hv, const uint64_t* x, Count n_x, const CotSrc& cot,
                     float* grad, uint64_t n_params, float* part, cudaStream_t s);
size_t nade_grad_partial_floats(const NadeView& m, uint64_t n_params, uint64_t n_x);
size_t nade_eloc_workspace(const anqs_ham* H, uint64_t n_x);
int run_eloc_nade(const anqs_model* M, const anqs_ham* H, const uint64_t* x, Count n_x, double* ere, double* eim,
                  const uint64_t* counts, double* stats, void* ws, size_t ws_bytes, cudaStream_t s);

// api.cu
int logpsi_dispatch(const anqs_model* M, const anqs_ham* H, const uint64_t* x, Count n_x, float* la,
                    float* ph, cudaStream_t s);

// sampler.cu
size_t sampler_workspace(const anqs_ham* ham, uint64_t n_samples);
// anqs_test_sampler_barrier: the persistent sampler's barrier target and limit
void sampler_test_barrier(unsigned extra_arrivals, uint64_t limit_ns);
int run_sampler(const anqs_model* md, const anqs_ham* ham, uint64_t n_samples, uint64_t seed,
                uint64_t counter, const uint64_t* counter_dev, uint64_t* x_out, uint64_t* n_out,
                uint64_t* n_unique, void* ws, size_t ws_bytes, cudaStream_t s, int rank = 0, int world = 1,
                int split_level = 0, bool binom = false);

}  // namespace anqs
