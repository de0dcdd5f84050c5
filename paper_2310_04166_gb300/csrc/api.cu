// C ABI entry points of libanqs: argument checks, handles, sector table,
// workspace planning and the order of kernel launches for each call.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <cstdlib>

#include "common.cuh"

namespace anqs {

static thread_local std::string g_msg;
static thread_local int g_code = ANQS_OK;

int set_error(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_msg = buf;
  g_code = code;
  return code;
}

int cuda_error(cudaError_t e, const char* what, const char* file, int line) {
  const char* base = strrchr(file, '/');
  return set_error(ANQS_ERR_CUDA, "%s failed: %s (%s:%d)", what, cudaGetErrorString(e),
                   base ? base + 1 : file, line);
}

// ---------------------------------------------------------------------------
// IsPhys (Algorithm 1) over the qubit tree, memoised in a dense lookup keyed
// by (i, n_e, 2 S_z, z) (Proposition 1).  Qubit i (1-based) adds n_e += x_i
// and 2 S_z += x_i for odd i (spin up), -x_i for even i (Appendix A, additive
// symmetries); each Z2 symmetry (a Pauli-Z string, Sec. IV.A, multiplicative)
// multiplies its eigenvalue by (-1)^x_i on the qubits of its support, kept
// here as parity bit j of z.  The target is the eigenvalue vector of the
// reference determinant.
// ---------------------------------------------------------------------------
struct IsPhysTable {
  int N, ne_ref, sz_ref, z_ref, nz;
  const uint64_t* zm;
  std::vector<int8_t> memo;  // -1 unknown, 0 false, 1 true
  IsPhysTable(int n_qubits, int ne, int sz, int nz_, const uint64_t* zmask, int zref)
      : N(n_qubits), ne_ref(ne), sz_ref(sz), z_ref(zref), nz(nz_), zm(zmask) {
    memo.assign(size_t(N + 2) * (N + 1) * (2 * N + 1) << nz, -1);
  }
  size_t key(int i, int ne, int sz, int z) const {
    return (((size_t(i) * (N + 1) + ne) * (2 * N + 1) + (sz + N)) << nz) + z;
  }
  int flip(int i) const {  // parity bits flipped by x_i = 1
    int f = 0;
    for (int j = 0; j < nz; ++j) f |= int((zm[j] >> (i - 1)) & 1ull) << j;
    return f;
  }
  bool operator()(int i, int ne, int sz, int z) {
    int8_t& m = memo[key(i, ne, sz, z)];
    if (m >= 0) return m != 0;
    bool r;
    if (i == N + 1) {
      r = (ne == ne_ref && sz == sz_ref && z == z_ref);
    } else {
      int dsz = (i % 2 == 1) ? 1 : -1;
      r = (*this)(i + 1, ne, sz, z) || (*this)(i + 1, ne + 1, sz + dsz, z ^ flip(i));
    }
    m = r ? 1 : 0;
    return r;
  }
};

static uint64_t sat_add(uint64_t a, uint64_t b) { return (a > UINT64_MAX - b) ? UINT64_MAX : a + b; }
static uint64_t binom(int n, int k) {
  if (k < 0 || k > n) return 0;
  uint64_t r = 1;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;  // exact for n <= 64 here
  return r;
}

static int check_stream_device(int device) {
  int cur = -1;
  ANQS_CUDA(cudaGetDevice(&cur));
  if (cur != device)
    return set_error(ANQS_ERR_ARG, "handle belongs to device %d but device %d is current", device, cur);
  return ANQS_OK;
}

}  // namespace anqs

namespace anqs {
int logpsi_dispatch(const anqs_model* M, const anqs_ham* H, const uint64_t* x, Count n_x, float* la,
                    float* ph, cudaStream_t s) {
  switch (M->d.kind) {
    case ANQS_MODEL_MLP:
      if (M->d.form == ANQS_FORM_BF16) {
        if (n_x.dev) return set_error(ANQS_ERR_UNSUPPORTED, "BF16 log psi takes host row counts");
        return launch_mlp_tc_logpsi(M, H->v, x, n_x.n, la, ph, s);
      }
      return launch_mlp_fp32_logpsi(M->mlp, H->v, x, n_x, la, ph, s);
    case ANQS_MODEL_TF:
      if (M->d.form == ANQS_FORM_BF16) {
        if (n_x.dev) return set_error(ANQS_ERR_UNSUPPORTED, "BF16 log psi takes host row counts");
        return launch_tf_tc_logpsi(M, H->v, x, n_x.n, la, ph, s);
      }
      return launch_tf_fp32_logpsi(M->tf, H->v, x, n_x, la, ph, s);
    case ANQS_MODEL_TABLE:
      return launch_table_logpsi(M, H->v, x, n_x, la, ph, s);
    case ANQS_MODEL_NADE:
      return launch_nade_logpsi(M->nade, H->v, x, n_x, la, ph, s);
    default:
      return set_error(ANQS_ERR_UNSUPPORTED, "model kind %d not supported by this library", M->d.kind);
  }
}
}  // namespace anqs

namespace anqs {
// FP32 form: every connected determinant evaluated over all slots.
static size_t eloc_plain_ws(const anqs_ham* H, uint64_t n_x, Arena& A, uint64_t** xp, double** hv,
                            double** hd, float** la_x, float** ph_x, float** la_p, float** ph_p) {
  uint64_t m = n_x * H->v.K;
  *xp = A.take<uint64_t>(m);
  *hv = A.take<double>(m);
  *hd = A.take<double>(n_x);
  *la_x = A.take<float>(n_x);
  *ph_x = A.take<float>(n_x);
  *la_p = A.take<float>(m);
  *ph_p = A.take<float>(m);
  return A.off;
}
}  // namespace anqs

namespace anqs {
// model kinds with a hand-written adjoint
static int check_adjoint(const anqs_model* M) {
  if (M->d.kind == ANQS_MODEL_MLP || M->d.kind == ANQS_MODEL_TF || M->d.kind == ANQS_MODEL_NADE) return ANQS_OK;
  return set_error(ANQS_ERR_UNSUPPORTED, "adjoint for model kind %d not supported by this library", M->d.kind);
}

// model-specific adjoint workspace (bytes) beyond the two cotangent arrays;
// with `least`, the smallest the adjoint accepts (the transformer then
// recomputes each block's activations from the block's input)
static size_t vjp_ws_bytes(const anqs_model* M, uint64_t n_x, bool least = false) {
  if (M->d.kind == ANQS_MODEL_TF) return tf_grad_workspace(M->tf, n_x, least);
  if (M->d.kind == ANQS_MODEL_NADE) return nade_grad_partial_floats(M->nade, M->n_params, n_x) * sizeof(float);
  return 0;
}

static int vjp_dispatch(const anqs_model* M, const anqs_ham* H, const uint64_t* x, Count n_x, const float* cl,
                        const float* cp, float* grad, float* part, void* ws, size_t ws_bytes, cudaStream_t s) {
  if (M->d.kind == ANQS_MODEL_MLP) {
    const CotSrc c{cl, cp, nullptr, nullptr, nullptr, nullptr};
    // the tensor-core adjoint writes per-tile partial gradients (anqs_grad's
    // workspace); anqs_logpsi_vjp, which has none for the MLP, stays in FP32
    if (part && M->d.form == ANQS_FORM_BF16 && mlp_tc_grad_supported(M))
      return launch_mlp_tc_grad(M, H->v, x, n_x, c, grad, part, s);
    return launch_mlp_fp32_grad(M->mlp, H->v, x, n_x, c, grad, part, s);
  }
  if (M->d.kind == ANQS_MODEL_TF) return launch_tf_fp32_grad(M->tf, H->v, x, n_x, cl, cp, grad, ws, ws_bytes, s);
  if (M->d.kind == ANQS_MODEL_NADE)
    return launch_nade_grad(M->nade, H->v, x, n_x, CotSrc{cl, cp, nullptr, nullptr, nullptr, nullptr}, grad,
                            M->n_params, static_cast<float*>(ws), s);
  return set_error(ANQS_ERR_UNSUPPORTED, "adjoint for model kind %d not supported by this library", M->d.kind);
}
}  // namespace anqs

using namespace anqs;

// Slot masks, physical-prefix counts per level and the sector dimension from
// IsPhys; the prefix counts come from a forward count of the qubit strings
// reaching each state (saturating).
static int build_sector(anqs_ham* H) {
  HamView& v = H->v;
  const int n = v.n, na = v.na, nb = v.nb, N = 2 * n, nz = v.nz, Z = 1 << nz;
  int zref = 0;  // reference determinant: the lowest N_a alpha and N_b beta orbitals
  for (int j = 0; j < nz; ++j) {
    uint64_t ref = 0;
    for (int p = 0; p < na; ++p) ref |= 1ull << (2 * p);
    for (int p = 0; p < nb; ++p) ref |= 1ull << (2 * p + 1);
    zref |= (__builtin_popcountll(ref & v.zmask[j]) & 1) << j;
  }
  IsPhysTable ip(N, na + nb, na - nb, nz, v.zmask, zref);
  H->mask_host.assign(size_t(n) * (na + 1) * (nb + 1) * Z, 0);
  for (int p = 0; p < n; ++p)
    for (int a = 0; a <= na; ++a)
      for (int b = 0; b <= nb; ++b)
        for (int z = 0; z < Z; ++z) {
          if (a > p || b > p) continue;
          if (!ip(2 * p + 1, a + b, a - b, z)) continue;
          uint8_t m = 0;
          for (int u = 0; u < 4; ++u) {
            const int da = u & 1, db = u >> 1;
            const int z2 = z ^ (da ? ip.flip(2 * p + 1) : 0) ^ (db ? ip.flip(2 * p + 2) : 0);
            if (ip(2 * p + 3, a + b + da + db, a - b + da - db, z2)) m |= uint8_t(1u << u);
          }
          H->mask_host[mask_index(v, p, a, b, z)] = m;
        }
  // forward counts of the (a, b, z) states over slot levels
  std::vector<uint64_t> cur(size_t(na + 1) * (nb + 1) * Z, 0), nxt;
  auto at = [&](int a, int b, int z) { return (size_t(a) * (nb + 1) + b) * Z + z; };
  cur[at(0, 0, 0)] = 1;
  H->phys_prefix.assign(n + 1, 0);
  for (int p = 0; p <= n; ++p) {
    uint64_t c = 0;
    for (int a = 0; a <= na; ++a)
      for (int b = 0; b <= nb; ++b)
        for (int z = 0; z < Z; ++z)
          if (cur[at(a, b, z)] && ip(2 * p + 1, a + b, a - b, z)) c = sat_add(c, cur[at(a, b, z)]);
    H->phys_prefix[p] = c;
    if (p == n) break;
    nxt.assign(cur.size(), 0);
    for (int a = 0; a <= na; ++a)
      for (int b = 0; b <= nb; ++b)
        for (int z = 0; z < Z; ++z) {
          const uint64_t w = cur[at(a, b, z)];
          if (!w) continue;
          for (int u = 0; u < 4; ++u) {
            const int a2 = a + (u & 1), b2 = b + (u >> 1);
            if (a2 > na || b2 > nb) continue;
            const int z2 = z ^ ((u & 1) ? ip.flip(2 * p + 1) : 0) ^ ((u >> 1) ? ip.flip(2 * p + 2) : 0);
            nxt[at(a2, b2, z2)] = sat_add(nxt[at(a2, b2, z2)], w);
          }
        }
    cur.swap(nxt);
  }
  H->sector_dim = H->phys_prefix[n];
  if (H->sector_dim == 0) return set_error(ANQS_ERR_SECTOR, "empty sector");
  return ANQS_OK;
}

// The sampler's prefix table: all physical prefixes of levels 0..n-1 by a
// breadth-first walk of the slot masks (children in ascending outcome, as the
// sampler emits them), when there are at most kPrefixTable of them and no
// level holds more than kPrefixLevel.  Uploads it to the device.
constexpr size_t kPrefixTable = 16384, kPrefixLevel = 2048;

static int build_prefix_table(anqs_ham* H) {
  const HamView& v = H->v;
  const int n = v.n;
  cudaFree(H->d_pt_x);
  cudaFree(H->d_pt_child);
  H->d_pt_x = nullptr;
  H->d_pt_child = nullptr;
  H->pt_x.clear();
  H->pt_off.clear();
  H->pt_child.clear();
  uint64_t total = 0;
  for (int p = 0; p < n; ++p) {
    if (H->phys_prefix[p] > kPrefixLevel) return ANQS_OK;
    total += H->phys_prefix[p];
  }
  if (total > kPrefixTable) return ANQS_OK;
  std::vector<uint64_t> x{0ull};
  std::vector<uint32_t> off{0u, 1u};
  std::vector<int32_t> child;
  for (int p = 0; p < n; ++p) {
    const uint64_t below = (1ull << (2 * p)) - 1ull;
    for (uint32_t i = off[p]; i < off[p + 1]; ++i) {
      const uint64_t xi = x[i];
      const int a = __builtin_popcountll(xi & below & 0x5555555555555555ull);
      const int b = __builtin_popcountll(xi & below & 0xAAAAAAAAAAAAAAAAull);
      int z = 0;
      for (int j = 0; j < v.nz; ++j) z |= (__builtin_popcountll(xi & below & v.zmask[j]) & 1) << j;
      const unsigned m = (a <= v.na && b <= v.nb) ? H->mask_host[mask_index(v, p, a, b, z)] : 0u;
      for (int u = 0; u < 4; ++u) {
        if (((m >> u) & 1u) && p + 1 < n) {
          child.push_back(int32_t(x.size()));
          x.push_back(xi | (uint64_t(u) << (2 * p)));
        } else {
          child.push_back(-1);
        }
      }
    }
    if (p + 1 < n) off.push_back(uint32_t(x.size()));
  }
  if (off.size() != size_t(n) + 1 || x.size() != total) return ANQS_OK;  // counts disagree: no table
  if (cudaMalloc(&H->d_pt_x, x.size() * sizeof(uint64_t)) != cudaSuccess ||
      cudaMalloc(&H->d_pt_child, child.size() * sizeof(int32_t)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(H->d_pt_x);
    H->d_pt_x = nullptr;
    return set_error(ANQS_ERR_CUDA, "cudaMalloc failed for the prefix table");
  }
  ANQS_CUDA(cudaMemcpy(H->d_pt_x, x.data(), x.size() * sizeof(uint64_t), cudaMemcpyHostToDevice));
  ANQS_CUDA(cudaMemcpy(H->d_pt_child, child.data(), child.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  H->pt_x.swap(x);
  H->pt_off.swap(off);
  H->pt_child.swap(child);
  return ANQS_OK;
}

extern "C" {

const char* anqs_version(void) { return "anqs 0.1 (sm_103a)"; }

int anqs_last_error(char* buf, size_t len) {
  if (buf && len) {
    size_t k = g_msg.size() < len - 1 ? g_msg.size() : len - 1;
    memcpy(buf, g_msg.data(), k);
    buf[k] = 0;
  }
  return g_code;
}

int anqs_hamiltonian_create(anqs_ham** out, int n, int na, int nb, const double* h_host,
                            const double* g_host, double e_nuc) {
  if (!out || !h_host || !g_host) return set_error(ANQS_ERR_ARG, "null argument");
  *out = nullptr;
  if (n < 1 || n > ANQS_MAX_ORB) return set_error(ANQS_ERR_ARG, "n_orb=%d outside 1..32", n);
  if (na < 0 || na > n || nb < 0 || nb > n)
    return set_error(ANQS_ERR_SECTOR, "N_alpha=%d, N_beta=%d outside 0..%d", na, nb, n);
  anqs_ham* H = new anqs_ham();
  ANQS_CUDA(cudaGetDevice(&H->device));
  HamView& v = H->v;
  v.n = n;
  v.na = na;
  v.nb = nb;
  uint64_t nsa = uint64_t(na) * (n - na), nsb = uint64_t(nb) * (n - nb);
  uint64_t ndaa = binom(na, 2) * binom(n - na, 2), ndbb = binom(nb, 2) * binom(n - nb, 2);
  uint64_t ndab = nsa * nsb;
  uint64_t K = nsa + nsb + ndaa + ndbb + ndab;
  if (K > 0x7fffffffull) {
    delete H;
    return set_error(ANQS_ERR_UNSUPPORTED, "connected set of %llu exceeds 2^31", (unsigned long long)K);
  }
  v.nsa = uint32_t(nsa);
  v.nsb = uint32_t(nsb);
  v.ndaa = uint32_t(ndaa);
  v.ndbb = uint32_t(ndbb);
  v.ndab = uint32_t(ndab);
  v.K = uint32_t(K);
  v.e_nuc = e_nuc;
  v.mu_lv = n;
  v.nz = 0;
  if (build_sector(H) != ANQS_OK) {
    delete H;
    return ANQS_ERR_SECTOR;
  }

  size_t hn = size_t(n) * n, gn = hn * hn;
  if (cudaMalloc(&H->d_h, hn * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&H->d_g, gn * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&H->d_mask, H->mask_host.size()) != cudaSuccess ||
      cudaMalloc(&H->d_status, sizeof(unsigned)) != cudaSuccess) {
    cudaGetLastError();
    anqs_hamiltonian_destroy(H);
    return set_error(ANQS_ERR_CUDA, "cudaMalloc failed for Hamiltonian tables");
  }
  ANQS_CUDA(cudaMemcpy(H->d_h, h_host, hn * sizeof(double), cudaMemcpyHostToDevice));
  ANQS_CUDA(cudaMemcpy(H->d_g, g_host, gn * sizeof(double), cudaMemcpyHostToDevice));
  ANQS_CUDA(cudaMemcpy(H->d_mask, H->mask_host.data(), H->mask_host.size(), cudaMemcpyHostToDevice));
  ANQS_CUDA(cudaMemset(H->d_status, 0, sizeof(unsigned)));
  v.status = H->d_status;
  v.h = H->d_h;
  v.g = H->d_g;
  v.mask = H->d_mask;
  v.mu_lv = n;
  if (build_prefix_table(H) != ANQS_OK) {
    anqs_hamiltonian_destroy(H);
    return ANQS_ERR_CUDA;
  }
  *out = H;
  return ANQS_OK;
}

int anqs_hamiltonian_set_z2(anqs_ham* H, int nz, const uint64_t* qubit_masks) {
  if (!H) return set_error(ANQS_ERR_ARG, "null Hamiltonian");
  if (nz < 0 || nz > 4) return set_error(ANQS_ERR_ARG, "nz %d outside 0..4", nz);
  if (nz && !qubit_masks) return set_error(ANQS_ERR_ARG, "null qubit masks");
  const int n = H->v.n;
  const uint64_t all = n >= 32 ? ~0ull : ((1ull << (2 * n)) - 1ull);
  for (int j = 0; j < nz; ++j)
    if (qubit_masks[j] & ~all) return set_error(ANQS_ERR_ARG, "Z2 mask %d reaches beyond qubit %d", j, 2 * n - 1);
  ANQS_TRY(check_stream_device(H->device));
  anqs_ham saved = *H;
  H->v.nz = nz;
  for (int j = 0; j < 4; ++j) H->v.zmask[j] = j < nz ? qubit_masks[j] : 0ull;
  if (build_sector(H) != ANQS_OK) {
    const int code = g_code;
    std::string msg = g_msg;
    H->v = saved.v;
    H->mask_host = saved.mask_host;
    H->phys_prefix = saved.phys_prefix;
    H->sector_dim = saved.sector_dim;
    set_error(code, "%s", msg.c_str());
    return code;
  }
  uint8_t* d = nullptr;
  ANQS_CUDA(cudaDeviceSynchronize());  // earlier work may still read the old table
  ANQS_CUDA(cudaMalloc(&d, H->mask_host.size()));
  ANQS_CUDA(cudaMemcpy(d, H->mask_host.data(), H->mask_host.size(), cudaMemcpyHostToDevice));
  cudaFree(H->d_mask);
  H->d_mask = d;
  H->v.mask = d;
  return build_prefix_table(H);
}

int anqs_hamiltonian_set_pruning(anqs_ham* H, int du_levels) {
  if (!H) return set_error(ANQS_ERR_ARG, "null Hamiltonian");
  if (du_levels < 0 || du_levels > H->v.n)
    return set_error(ANQS_ERR_ARG, "du_levels %d outside 0..%d", du_levels, H->v.n);
  H->v.mu_lv = H->v.n - du_levels;
  return ANQS_OK;
}

int anqs_hamiltonian_destroy(anqs_ham* H) {
  if (!H) return ANQS_OK;
  cudaFree(H->d_h);
  cudaFree(H->d_g);
  cudaFree(H->d_mask);
  cudaFree(H->d_pt_x);
  cudaFree(H->d_pt_child);
  cudaFree(H->d_status);
  delete H;
  return ANQS_OK;
}

int anqs_hamiltonian_status(const anqs_ham* H, int* status, int clear) {
  if (!H || !status) return set_error(ANQS_ERR_ARG, "null argument");
  ANQS_TRY(check_stream_device(H->device));
  unsigned v = 0;
  ANQS_CUDA(cudaMemcpy(&v, H->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost));
  if (clear) ANQS_CUDA(cudaMemset(H->d_status, 0, sizeof(unsigned)));
  *status = int(v);
  return ANQS_OK;
}

int anqs_hamiltonian_info(const anqs_ham* H, uint64_t* n_connected, uint64_t* sector_dim) {
  if (!H) return set_error(ANQS_ERR_ARG, "null Hamiltonian");
  if (n_connected) *n_connected = H->v.K;
  if (sector_dim) *sector_dim = H->sector_dim;
  return ANQS_OK;
}

int anqs_hamiltonian_slot_masks(const anqs_ham* H, uint8_t* out, size_t len) {
  if (!H || !out) return set_error(ANQS_ERR_ARG, "null argument");
  if (len < H->mask_host.size())
    return set_error(ANQS_ERR_CAPACITY, "need %zu bytes", H->mask_host.size());
  memcpy(out, H->mask_host.data(), H->mask_host.size());
  return ANQS_OK;
}

int anqs_connected(const anqs_ham* H, const uint64_t* x, uint64_t n_x, uint64_t* xp, double* hval,
                   uint8_t* first_slot, double* hdiag, void* stream) {
  if (!H) return set_error(ANQS_ERR_ARG, "null Hamiltonian");
  if (n_x == 0) return ANQS_OK;
  if (!x || !xp || !hval) return set_error(ANQS_ERR_ARG, "null array argument");
  ANQS_TRY(check_stream_device(H->device));
  return launch_connected(H->v, x, host_count(n_x), xp, hval, first_slot, hdiag, (cudaStream_t)stream);
}

// ---------------------------------------------------------------------------
// models
// ---------------------------------------------------------------------------
static int validate_desc(const anqs_model_desc* d) {
  if (!d) return set_error(ANQS_ERR_ARG, "null model description");
  if (d->n_orb < 1 || d->n_orb > ANQS_MAX_ORB) return set_error(ANQS_ERR_ARG, "n_orb=%d outside 1..32", d->n_orb);
  if (d->form != ANQS_FORM_FP32 && d->form != ANQS_FORM_BF16)
    return set_error(ANQS_ERR_ARG, "unknown form %d", d->form);
  switch (d->kind) {
    case ANQS_MODEL_MLP:
      if (d->width != 64 && d->width != 128 && d->width != 256)
        return set_error(ANQS_ERR_UNSUPPORTED, "MLP width %d not in {64,128,256}", d->width);
      if (d->n_hidden < 1 || d->n_hidden > 8)
        return set_error(ANQS_ERR_UNSUPPORTED, "MLP hidden layers %d outside 1..8", d->n_hidden);
      return ANQS_OK;
    case ANQS_MODEL_TF:
      if (d->d_model != 32 && d->d_model != 64 && d->d_model != 128 && d->d_model != 256)
        return set_error(ANQS_ERR_UNSUPPORTED, "d_model %d not in {32,64,128,256}", d->d_model);
      if (d->n_heads < 1 || d->d_model % d->n_heads)
        return set_error(ANQS_ERR_UNSUPPORTED, "n_heads %d does not divide d_model", d->n_heads);
      if (d->n_layers < 1 || d->n_layers > 16)
        return set_error(ANQS_ERR_UNSUPPORTED, "n_layers %d outside 1..16", d->n_layers);
      return ANQS_OK;
    case ANQS_MODEL_TABLE:
      if (d->n_orb > 11) return set_error(ANQS_ERR_UNSUPPORTED, "table model needs n_orb <= 11");
      if (d->form != ANQS_FORM_FP32) return set_error(ANQS_ERR_UNSUPPORTED, "table model is FP32 only");
      return ANQS_OK;
    case ANQS_MODEL_NADE:
      if (d->width != 32 && d->width != 64 && d->width != 128)
        return set_error(ANQS_ERR_UNSUPPORTED, "NADE width %d not in {32,64,128}", d->width);
      if (d->form != ANQS_FORM_FP32) return set_error(ANQS_ERR_UNSUPPORTED, "NADE model is FP32 only");
      return ANQS_OK;
  }
  return set_error(ANQS_ERR_ARG, "unknown model kind %d", d->kind);
}

// floats of qubit i's block: complex W1 [w][i], b1 [w], W2 [w][w], b2 [w], W3 [2][w], b3 [2]
static uint64_t nade_qubit_floats(uint64_t w, uint64_t i) { return 2 * (w * i + w + w * w + w + 2 * w + 2); }

static uint64_t count_params(const anqs_model_desc* d) {
  uint64_t n = d->n_orb;
  if (d->kind == ANQS_MODEL_MLP) {
    uint64_t w = d->width, t = 0;
    for (uint64_t p = 0; p < n; ++p) t += 4 * p * w + w + (d->n_hidden - 1) * (w * w + w) + 8 * w + 8;
    return t;
  }
  if (d->kind == ANQS_MODEL_TF) {
    uint64_t D = d->d_model;
    uint64_t per = 4 * D + 4 * (D * D + D) + 2 * (4 * D * D) + 4 * D + D;
    return 5 * D + n * D + d->n_layers * per + 2 * D + 8 * D + 8;
  }
  if (d->kind == ANQS_MODEL_NADE) {
    uint64_t t = 0;
    for (uint64_t i = 0; i < 2 * n; ++i) t += nade_qubit_floats(d->width, i);
    return t;
  }
  uint64_t t = 0, r = 1;
  for (uint64_t p = 0; p < n; ++p, r *= 4) t += 8 * r;
  return t;
}

int anqs_model_param_count(const anqs_model_desc* d, uint64_t* n) {
  ANQS_TRY(validate_desc(d));
  if (!n) return set_error(ANQS_ERR_ARG, "null output");
  *n = count_params(d);
  return ANQS_OK;
}

int anqs_model_create(anqs_model** out, const anqs_model_desc* d, const float* params) {
  if (!out) return set_error(ANQS_ERR_ARG, "null output");
  *out = nullptr;
  ANQS_TRY(validate_desc(d));
  if (!params) return set_error(ANQS_ERR_ARG, "null parameters");
  anqs_model* M = new anqs_model();
  M->d = *d;
  ANQS_CUDA(cudaGetDevice(&M->device));
  M->params = params;
  M->n_params = count_params(d);
  M->packed = nullptr;
  M->packed_bytes = 0;
  M->tc_raw = nullptr;
  M->tc_raw_rows = 0;
  if (d->kind == ANQS_MODEL_MLP) {
    MlpView& v = M->mlp;
    v.n = d->n_orb;
    v.width = d->width;
    v.n_hidden = d->n_hidden;
    v.params = params;
    uint64_t off = 0, w = d->width;
    for (int p = 0; p <= d->n_orb; ++p) {
      v.slot_off[p] = uint32_t(off);
      off += 4 * uint64_t(p) * w + w + (d->n_hidden - 1) * (w * w + w) + 8 * w + 8;
    }
    if (M->n_params > 0xffffffffull) {
      delete M;
      return set_error(ANQS_ERR_UNSUPPORTED, "too many parameters");
    }
    if (d->form == ANQS_FORM_BF16) {
      int r = mlp_tc_pack_alloc(M);
      if (r != ANQS_OK) {
        anqs_model_destroy(M);
        return r;
      }
      r = mlp_tc_pack(M, 0);
      if (r == ANQS_OK && cudaDeviceSynchronize() != cudaSuccess) r = set_error(ANQS_ERR_CUDA, "pack failed");
      if (r != ANQS_OK) {
        anqs_model_destroy(M);
        return r;
      }
    }
  } else if (d->kind == ANQS_MODEL_NADE) {
    NadeView& v = M->nade;
    v.n = d->n_orb;
    v.w = d->width;
    v.params = params;
    uint64_t off = 0;
    for (int i = 0; i < 2 * d->n_orb; ++i) {
      v.qoff[i] = uint32_t(off);
      off += nade_qubit_floats(d->width, i);
    }
  } else if (d->kind == ANQS_MODEL_TF) {
    M->tf.n = d->n_orb;
    M->tf.d = d->d_model;
    M->tf.H = d->n_heads;
    M->tf.L = d->n_layers;
    M->tf.params = params;
    if (d->form == ANQS_FORM_BF16) {
      int r = tf_tc_pack_alloc(M);
      if (r == ANQS_OK) r = tf_tc_pack(M, 0);
      if (r == ANQS_OK && cudaDeviceSynchronize() != cudaSuccess) r = set_error(ANQS_ERR_CUDA, "pack failed");
      if (r != ANQS_OK) {
        anqs_model_destroy(M);
        return r;
      }
    }
  }
  *out = M;
  return ANQS_OK;
}

int anqs_model_destroy(anqs_model* M) {
  if (!M) return ANQS_OK;
  if (M->packed) cudaFree(M->packed);
  if (M->tc_raw) cudaFree(M->tc_raw);
  if (M->ev_fork) cudaEventDestroy(M->ev_fork);
  if (M->ev_join) cudaEventDestroy(M->ev_join);
  if (M->side) cudaStreamDestroy(M->side);
  delete M;
  return ANQS_OK;
}

int anqs_model_sync(anqs_model* M, void* stream) {
  if (!M) return set_error(ANQS_ERR_ARG, "null model");
  ANQS_TRY(check_stream_device(M->device));
  if (M->d.kind == ANQS_MODEL_MLP && M->d.form == ANQS_FORM_BF16) return mlp_tc_pack(M, (cudaStream_t)stream);
  if (M->d.kind == ANQS_MODEL_TF && M->d.form == ANQS_FORM_BF16) return tf_tc_pack(M, (cudaStream_t)stream);
  return ANQS_OK;
}

int anqs_test_sampler_barrier(unsigned extra_arrivals, uint64_t limit_ns) {
  sampler_test_barrier(extra_arrivals, limit_ns);
  return ANQS_OK;
}

int anqs_model_status(const anqs_model* M, int* status) {
  if (!M || !status) return set_error(ANQS_ERR_ARG, "null argument");
  *status = 0;
  if (M->d.form != ANQS_FORM_BF16) return ANQS_OK;
  ANQS_TRY(check_stream_device(M->device));
  return M->d.kind == ANQS_MODEL_TF ? tf_tc_status(M, status) : mlp_tc_status(M, status);
}

static int check_pair(const anqs_model* M, const anqs_ham* H) {
  if (!M || !H) return set_error(ANQS_ERR_ARG, "null model or Hamiltonian");
  if (M->d.n_orb != H->v.n)
    return set_error(ANQS_ERR_ARG, "model has %d slots, Hamiltonian %d orbitals", M->d.n_orb, H->v.n);
  if (M->device != H->device) return set_error(ANQS_ERR_ARG, "model and Hamiltonian on different devices");
  return check_stream_device(M->device);
}


int anqs_logpsi(const anqs_model* M, const anqs_ham* H, const uint64_t* x, uint64_t n_x, float* la,
                float* ph, void* stream) {
  ANQS_TRY(check_pair(M, H));
  if (n_x == 0) return ANQS_OK;
  if (!x || !la || !ph) return set_error(ANQS_ERR_ARG, "null array argument");
  return logpsi_dispatch(M, H, x, host_count(n_x), la, ph, (cudaStream_t)stream);
}

// ---------------------------------------------------------------------------
// sampling
// ---------------------------------------------------------------------------
int anqs_sample_workspace_size(const anqs_model* M, const anqs_ham* H, uint64_t n_samples, size_t* bytes) {
  ANQS_TRY(check_pair(M, H));
  if (!bytes) return set_error(ANQS_ERR_ARG, "null output");
  if (n_samples == 0) return set_error(ANQS_ERR_ARG, "n_samples must be >= 1");
  *bytes = sampler_workspace(H, n_samples);
  return ANQS_OK;
}

int anqs_sample(const anqs_model* M, const anqs_ham* H, uint64_t n_samples, uint64_t seed,
                uint64_t counter, const uint64_t* counter_dev, uint64_t* x_out, uint64_t* n_out, uint64_t cap,
                uint64_t* n_unique, void* ws, size_t ws_bytes, void* stream) {
  ANQS_TRY(check_pair(M, H));
  if (n_samples == 0) return set_error(ANQS_ERR_ARG, "n_samples must be >= 1");
  if (!x_out || !n_out || !n_unique) return set_error(ANQS_ERR_ARG, "null output");
  uint64_t need = n_samples < H->sector_dim ? n_samples : H->sector_dim;
  if (cap < need)
    return set_error(ANQS_ERR_CAPACITY, "cap %llu < min(n_samples, sector_dim) = %llu",
                     (unsigned long long)cap, (unsigned long long)need);
  size_t wsn = sampler_workspace(H, n_samples);
  if (ws_bytes < wsn || (wsn && !ws))
    return set_error(ANQS_ERR_CAPACITY, "sampler workspace needs %zu bytes", wsn);
  return run_sampler(M, H, n_samples, seed, counter, counter_dev, x_out, n_out, n_unique, ws, ws_bytes,
                     (cudaStream_t)stream);
}

int anqs_sample_binomial(const anqs_model* M, const anqs_ham* H, uint64_t n_samples, uint64_t seed, uint64_t counter,
                         const uint64_t* counter_dev, uint64_t* x_out, uint64_t* n_out, uint64_t cap,
                         uint64_t* n_unique, void* ws, size_t ws_bytes, void* stream) {
  ANQS_TRY(check_pair(M, H));
  if (n_samples == 0) return set_error(ANQS_ERR_ARG, "n_samples must be >= 1");
  if (!x_out || !n_out || !n_unique) return set_error(ANQS_ERR_ARG, "null output");
  uint64_t need = n_samples < H->sector_dim ? n_samples : H->sector_dim;
  if (cap < need)
    return set_error(ANQS_ERR_CAPACITY, "cap %llu < min(n_samples, sector_dim) = %llu",
                     (unsigned long long)cap, (unsigned long long)need);
  size_t wsn = sampler_workspace(H, n_samples);
  if (ws_bytes < wsn || (wsn && !ws))
    return set_error(ANQS_ERR_CAPACITY, "sampler workspace needs %zu bytes", wsn);
  return run_sampler(M, H, n_samples, seed, counter, counter_dev, x_out, n_out, n_unique, ws, ws_bytes,
                     (cudaStream_t)stream, 0, 1, 0, true);
}

int anqs_sample_shard(const anqs_model* M, const anqs_ham* H, uint64_t n_samples, uint64_t seed, uint64_t counter,
                      const uint64_t* counter_dev, int rank, int world, int split_level, uint64_t* x_out,
                      uint64_t* n_out, uint64_t cap, uint64_t* n_unique, void* ws, size_t ws_bytes, void* stream) {
  ANQS_TRY(check_pair(M, H));
  if (world < 1 || rank < 0 || rank >= world) return set_error(ANQS_ERR_ARG, "rank %d of world %d", rank, world);
  if (split_level < 0 || split_level > H->v.n)
    return set_error(ANQS_ERR_ARG, "split level %d outside 0..%d", split_level, H->v.n);
  if (n_samples == 0) return set_error(ANQS_ERR_ARG, "n_samples must be >= 1");
  if (!x_out || !n_out || !n_unique) return set_error(ANQS_ERR_ARG, "null output");
  uint64_t need = n_samples < H->sector_dim ? n_samples : H->sector_dim;
  if (cap < need)
    return set_error(ANQS_ERR_CAPACITY, "cap %llu < min(n_samples, sector_dim) = %llu",
                     (unsigned long long)cap, (unsigned long long)need);
  size_t wsn = sampler_workspace(H, n_samples);
  if (ws_bytes < wsn || (wsn && !ws))
    return set_error(ANQS_ERR_CAPACITY, "sampler workspace needs %zu bytes", wsn);
  return run_sampler(M, H, n_samples, seed, counter, counter_dev, x_out, n_out, n_unique, ws, ws_bytes,
                     (cudaStream_t)stream, rank, world, split_level);
}

int anqs_stats_combine(const double* stats_in, int world, double* stats_out, void* stream) {
  if (world < 1) return set_error(ANQS_ERR_ARG, "world %d < 1", world);
  if (!stats_in || !stats_out) return set_error(ANQS_ERR_ARG, "null stats");
  return launch_stats_combine(stats_in, world, stats_out, (cudaStream_t)stream);
}

// ---------------------------------------------------------------------------
// local energy
// ---------------------------------------------------------------------------

// prefix-reuse local energy: the BF16 forms and the NADE
static bool uses_tc_eloc(const anqs_model* M) { return M->d.form == ANQS_FORM_BF16 || M->d.kind == ANQS_MODEL_NADE; }

static size_t tc_eloc_workspace(const anqs_model* M, const anqs_ham* H, uint64_t n_x) {
  if (M->d.kind == ANQS_MODEL_NADE) return nade_eloc_workspace(H, n_x);
  return M->d.kind == ANQS_MODEL_TF ? tf_tc_eloc_workspace(M, H, n_x) : eloc_tc_workspace(M, H, n_x);
}

int anqs_local_energy_workspace_size(const anqs_model* M, const anqs_ham* H, uint64_t n_x, size_t* bytes) {
  ANQS_TRY(check_pair(M, H));
  if (!bytes) return set_error(ANQS_ERR_ARG, "null output");
  if (uses_tc_eloc(M)) {
    *bytes = tc_eloc_workspace(M, H, n_x);
    return ANQS_OK;
  }
  Arena A(nullptr, 0);
  uint64_t* a;
  double *b, *c;
  float *d, *e, *f, *g;
  *bytes = eloc_plain_ws(H, n_x, A, &a, &b, &c, &d, &e, &f, &g);
  return ANQS_OK;
}

int anqs_local_energy(const anqs_model* M, const anqs_ham* H, const uint64_t* x, const uint64_t* counts,
                      uint64_t n_x, const uint64_t* n_x_dev, double* ere, double* eim, double* stats, void* ws,
                      size_t ws_bytes, void* stream) {
  ANQS_TRY(check_pair(M, H));
  if (n_x == 0) return set_error(ANQS_ERR_ARG, "n_x must be >= 1");
  if (!x || !ere || !eim) return set_error(ANQS_ERR_ARG, "null array argument");
  if (counts && !stats) return set_error(ANQS_ERR_ARG, "counts given without stats output");
  cudaStream_t s = (cudaStream_t)stream;
  const Count nc{n_x, n_x_dev, 1};
  if (uses_tc_eloc(M)) {
    size_t need = tc_eloc_workspace(M, H, n_x);
    if (ws_bytes < need || !ws) return set_error(ANQS_ERR_CAPACITY, "workspace needs %zu bytes", need);
    // the assembly kernel also writes the statistics (counts set)
    if (M->d.kind == ANQS_MODEL_NADE) ANQS_TRY(run_eloc_nade(M, H, x, nc, ere, eim, counts, stats, ws, ws_bytes, s));
    else if (M->d.kind == ANQS_MODEL_TF)
      ANQS_TRY(run_eloc_tf_tc(M, H, x, nc, ere, eim, counts, stats, ws, ws_bytes, s));
    else ANQS_TRY(run_eloc_tc(M, H, x, nc, ere, eim, counts, stats, ws, ws_bytes, s));
    return ANQS_OK;
  } else {
    Arena A(ws, ws_bytes);
    uint64_t* xp;
    double *hv, *hd;
    float *la_x, *ph_x, *la_p, *ph_p;
    size_t need = eloc_plain_ws(H, n_x, A, &xp, &hv, &hd, &la_x, &ph_x, &la_p, &ph_p);
    if (ws_bytes < need || !ws) return set_error(ANQS_ERR_CAPACITY, "workspace needs %zu bytes", need);
    ANQS_TRY(launch_connected(H->v, x, nc, xp, hv, nullptr, hd, s));
    ANQS_TRY(logpsi_dispatch(M, H, x, nc, la_x, ph_x, s));
    ANQS_TRY(logpsi_dispatch(M, H, xp, scaled(nc, H->v.K), la_p, ph_p, s));
    ANQS_TRY(launch_eloc_sum(H->v, nc, hv, hd, la_x, ph_x, la_p, ph_p, ere, eim, s));
  }
  if (counts) ANQS_TRY(launch_stats(ere, eim, counts, nc, stats, s));
  return ANQS_OK;
}

// ---------------------------------------------------------------------------
// gradient
// ---------------------------------------------------------------------------

// ---------------------------------------------------------------------------
// batched local energy: one stream per problem, forked from and joined back
// into the caller's stream with events
// ---------------------------------------------------------------------------
}  // extern "C"

struct anqs_batch {
  int device;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> done;  // problem k's work is queued
  std::vector<cudaEvent_t> pre;   // problem k's stages before the persistent launch are queued
  cudaEvent_t fork = nullptr, mid = nullptr;
  cudaEvent_t t0 = nullptr, t1 = nullptr;  // around the persistent launch (autotuner)
  bool timing = false;
  void* groups = nullptr;  // work groups of the persistent launch (device)
  uint32_t* ctl = nullptr;  // its counters (device)
  int mode = ANQS_BATCH_DYNAMIC, chunk = 8;
};

static void batch_release(anqs_batch* b) {
  for (cudaStream_t st : b->streams) cudaStreamDestroy(st);
  for (cudaEvent_t e : b->done) cudaEventDestroy(e);
  for (cudaEvent_t e : b->pre) cudaEventDestroy(e);
  for (cudaEvent_t e : {b->fork, b->mid, b->t0, b->t1})
    if (e) cudaEventDestroy(e);
  if (b->groups) cudaFree(b->groups);
  if (b->ctl) cudaFree(b->ctl);
  delete b;
}

// problems whose suffix stage can join the persistent multi-problem launch:
// 16-bit MLPs of one width (the width of the first such problem), at most
// mlp_tc_multi_max() of them
static std::vector<char> fusable(const anqs_batch* b, const anqs_eloc_problem* q, int n) {
  std::vector<char> f(size_t(n), 0);
  if (b->mode == ANQS_BATCH_STREAMS) return f;
  int width = 0, taken = 0;
  for (int k = 0; k < n && taken < mlp_tc_multi_max(); ++k) {
    const anqs_model* M = q[k].model;
    if (M->d.kind != ANQS_MODEL_MLP || M->d.form != ANQS_FORM_BF16) continue;
    if (!width) width = M->d.width;
    if (M->d.width != width) continue;
    f[size_t(k)] = 1;
    ++taken;
  }
  return f;
}

// checks of one problem, before anything of the call is queued
static int check_problem(const anqs_eloc_problem& q, int device) {
  ANQS_TRY(check_pair(q.model, q.ham));
  if (q.model->device != device) return set_error(ANQS_ERR_ARG, "problem on another device than the batch handle");
  if (q.n_x == 0) return set_error(ANQS_ERR_ARG, "n_x must be >= 1");
  if (!q.x_dev || !q.eloc_re_dev || !q.eloc_im_dev) return set_error(ANQS_ERR_ARG, "null array argument");
  if (q.counts_dev && !q.stats_dev) return set_error(ANQS_ERR_ARG, "counts given without stats output");
  size_t need = 0;
  ANQS_TRY(anqs_local_energy_workspace_size(q.model, q.ham, q.n_x, &need));
  if (q.workspace_bytes < need || !q.workspace_dev) return set_error(ANQS_ERR_CAPACITY, "workspace needs %zu bytes", need);
  if (uses_tc_eloc(q.model) && q.n_x * uint64_t(q.ham->v.K) > 0xffffffffull)
    return set_error(ANQS_ERR_UNSUPPORTED, "more than 2^32 connected determinants per call");
  return ANQS_OK;
}

extern "C" {

int anqs_batch_create(anqs_batch** out, int max_problems) {
  if (!out) return set_error(ANQS_ERR_ARG, "null output");
  *out = nullptr;
  if (max_problems < 1 || max_problems > 4096) return set_error(ANQS_ERR_ARG, "max_problems %d outside 1..4096", max_problems);
  anqs_batch* b = new anqs_batch();
  cudaError_t e = cudaGetDevice(&b->device);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->mid, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreate(&b->t0);
  if (e == cudaSuccess) e = cudaEventCreate(&b->t1);
  if (e == cudaSuccess) e = cudaMalloc(&b->groups, mlp_tc_multi_groups_bytes());
  if (e == cudaSuccess) e = cudaMalloc(&b->ctl, 4 * sizeof(uint32_t));
  for (int k = 0; e == cudaSuccess && k < max_problems; ++k) {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr, ep = nullptr;
    e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) b->streams.push_back(st);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) b->done.push_back(ev);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ep, cudaEventDisableTiming);
    if (e == cudaSuccess) b->pre.push_back(ep);
  }
  if (e != cudaSuccess) {
    batch_release(b);
    return set_error(ANQS_ERR_CUDA, "batch handle: %s", cudaGetErrorString(e));
  }
  *out = b;
  return ANQS_OK;
}

int anqs_batch_destroy(anqs_batch* b) {
  if (!b) return ANQS_OK;
  batch_release(b);
  return ANQS_OK;
}

int anqs_batched_local_energy(anqs_batch* b, const anqs_eloc_problem* q, int n, void* stream) {
  if (!b) return set_error(ANQS_ERR_ARG, "null batch handle");
  if (n < 0 || (n > 0 && !q)) return set_error(ANQS_ERR_ARG, "invalid problem list");
  if (n > int(b->streams.size()))
    return set_error(ANQS_ERR_CAPACITY, "%d problems for a handle of %zu streams", n, b->streams.size());
  ANQS_TRY(check_stream_device(b->device));
  for (int k = 0; k < n; ++k) {
    const int r = check_problem(q[k], b->device);
    if (r != ANQS_OK) return r;
  }
  if (n == 0) return ANQS_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const std::vector<char> fused = fusable(b, q, n);
  std::vector<MultiEloc> multi;
  for (int k = 0; k < n; ++k)
    if (fused[size_t(k)])
      multi.push_back(MultiEloc{q[k].model, q[k].ham, q[k].n_x, q[k].workspace_dev, q[k].workspace_bytes});
  // Host-side fault injection for tests of this error path: ANQS_BATCH_FAIL_AT=k
  // makes problem k fail as a queueing error would, after its stream was forked.
  int fail_at = -1;
  if (const char* e = getenv("ANQS_BATCH_FAIL_AT")) fail_at = atoi(e);
  ANQS_CUDA(cudaEventRecord(b->fork, s));
  // join[k]: the last event recorded on problem k's stream (0 none, 1 pre, 2 done)
  std::vector<int> join(size_t(n), 0);
  int r = ANQS_OK;
  auto fail = [&](const char* what) {
    if (r == ANQS_OK) r = set_error(ANQS_ERR_CUDA, "batched local energy: %s failed", what);
  };
  for (int k = 0; k < n && r == ANQS_OK; ++k) {
    cudaStream_t sk = b->streams[k];
    if (cudaStreamWaitEvent(sk, b->fork, 0) != cudaSuccess) {
      fail("stream fork");
      break;
    }
    const Count nc{q[k].n_x, q[k].n_x_dev, 1};
    if (k == fail_at) {
      r = set_error(ANQS_ERR_CUDA, "batched local energy: injected failure at problem %d", k);
      if (cudaEventRecord(b->done[k], sk) == cudaSuccess) join[k] = 2;
    } else if (fused[size_t(k)]) {
      r = eloc_tc_pre(q[k].model, q[k].ham, q[k].x_dev, nc, q[k].workspace_dev, q[k].workspace_bytes, sk);
      if (cudaEventRecord(b->pre[k], sk) == cudaSuccess) join[k] = 1;
      else fail("event record");
    } else {
      r = anqs_local_energy(q[k].model, q[k].ham, q[k].x_dev, q[k].counts_dev, q[k].n_x, q[k].n_x_dev,
                            q[k].eloc_re_dev, q[k].eloc_im_dev, q[k].stats_dev, q[k].workspace_dev,
                            q[k].workspace_bytes, sk);
      // joined even on an error, so that the caller's stream stays ordered after it
      if (cudaEventRecord(b->done[k], sk) == cudaSuccess) join[k] = 2;
      else fail("event record");
    }
  }
  if (!multi.empty()) {
    // the persistent launch waits for every fused problem's first stages
    bool all_pre = true;
    for (int k = 0; k < n; ++k)
      if (fused[size_t(k)]) {
        if (join[k] != 1) all_pre = false;
        else if (cudaStreamWaitEvent(s, b->pre[k], 0) != cudaSuccess) fail("stream join");
      }
    if (r == ANQS_OK && all_pre) {
      if (b->timing && cudaEventRecord(b->t0, s) != cudaSuccess) fail("timing event");
      if (r == ANQS_OK)
        r = launch_mlp_tc_multi(multi.data(), int(multi.size()), b->chunk, b->mode == ANQS_BATCH_DYNAMIC, b->groups,
                                b->ctl, s);
      if (b->timing && r == ANQS_OK && cudaEventRecord(b->t1, s) != cudaSuccess) fail("timing event");
      if (cudaEventRecord(b->mid, s) != cudaSuccess) fail("event record");
      // the last stages of every fused problem, back on its own stream
      for (int k = 0; k < n && r == ANQS_OK; ++k) {
        if (!fused[size_t(k)]) continue;
        cudaStream_t sk = b->streams[k];
        if (cudaStreamWaitEvent(sk, b->mid, 0) != cudaSuccess) {
          fail("stream fork");
          break;
        }
        const Count nc{q[k].n_x, q[k].n_x_dev, 1};
        r = eloc_tc_post(q[k].ham, nc, q[k].eloc_re_dev, q[k].eloc_im_dev, q[k].counts_dev, q[k].stats_dev,
                         q[k].workspace_dev, q[k].workspace_bytes, sk);
        if (cudaEventRecord(b->done[k], sk) == cudaSuccess) join[k] = 2;
        else fail("event record");
      }
    }
  }
  for (int k = 0; k < n; ++k) {
    if (!join[k]) continue;
    if (cudaStreamWaitEvent(s, join[k] == 2 ? b->done[k] : b->pre[k], 0) != cudaSuccess) fail("stream join");
  }
  return r;
}

int anqs_batch_set_schedule(anqs_batch* b, int mode, int chunk) {
  if (!b) return set_error(ANQS_ERR_ARG, "null batch handle");
  if (mode != ANQS_BATCH_STREAMS && mode != ANQS_BATCH_STATIC && mode != ANQS_BATCH_DYNAMIC)
    return set_error(ANQS_ERR_ARG, "unknown schedule mode %d", mode);
  if (chunk < 1 || chunk > 1024) return set_error(ANQS_ERR_ARG, "chunk %d outside 1..1024", chunk);
  b->mode = mode;
  b->chunk = chunk;
  return ANQS_OK;
}

int anqs_batch_get_schedule(const anqs_batch* b, int* mode, int* chunk) {
  if (!b || !mode || !chunk) return set_error(ANQS_ERR_ARG, "null argument");
  *mode = b->mode;
  *chunk = b->chunk;
  return ANQS_OK;
}

int anqs_batch_autotune(anqs_batch* b, const anqs_eloc_problem* q, int n, void* stream, float* times_ms) {
  if (!b) return set_error(ANQS_ERR_ARG, "null batch handle");
  cudaStream_t s = (cudaStream_t)stream;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  ANQS_CUDA(cudaStreamIsCapturing(s, &cs));
  if (cs != cudaStreamCaptureStatusNone) return set_error(ANQS_ERR_ARG, "autotuning cannot run inside a capture");
  const int mode0 = b->mode, chunk0 = b->chunk;
  if (b->mode == ANQS_BATCH_STREAMS) b->mode = ANQS_BATCH_DYNAMIC;
  bool any = false;
  for (char f : fusable(b, q, n)) any = any || f;
  if (!any) {
    b->mode = mode0;
    return set_error(ANQS_ERR_UNSUPPORTED, "no problem of the batch runs in the persistent launch");
  }
  // candidates: STATIC (contiguous tile ranges; chunk unused), then DYNAMIC
  // with 8 .. 512 tiles per work item
  static const int kChunks[8] = {1, 8, 16, 32, 64, 128, 256, 512};
  float best = -1.f;
  int best_mode = b->mode, best_chunk = b->chunk, r = ANQS_OK;
  b->timing = true;
  r = anqs_batched_local_energy(b, q, n, stream);  // warm-up (module loading, caches)
  for (int c = 0; c < 8 && r == ANQS_OK; ++c) {
    b->mode = c == 0 ? ANQS_BATCH_STATIC : ANQS_BATCH_DYNAMIC;
    b->chunk = kChunks[c];
    r = anqs_batched_local_energy(b, q, n, stream);
    float ms = 0.f;
    if (r == ANQS_OK && (cudaEventSynchronize(b->t1) != cudaSuccess ||
                         cudaEventElapsedTime(&ms, b->t0, b->t1) != cudaSuccess))
      r = set_error(ANQS_ERR_CUDA, "autotuner timing failed");
    if (times_ms) times_ms[c] = ms;
    if (r == ANQS_OK && (best < 0.f || ms < best)) {
      best = ms;
      best_mode = b->mode;
      best_chunk = b->chunk;
    }
  }
  b->timing = false;
  if (r != ANQS_OK) {
    b->mode = mode0;
    b->chunk = chunk0;
    return r;
  }
  b->mode = best_mode;
  b->chunk = best_chunk;
  ANQS_CUDA(cudaStreamSynchronize(s));
  return ANQS_OK;
}

static size_t grad_ws_bytes(const anqs_model* M, uint64_t n_x, bool least) {
  Arena A(nullptr, 0);
  A.take<float>(n_x);
  A.take<float>(n_x);
  if (M->d.kind == ANQS_MODEL_MLP) A.take<float>(mlp_fp32_grad_partial_floats(M->mlp, n_x));
  A.take<char>(vjp_ws_bytes(M, n_x, least));
  return A.off;
}

int anqs_grad_workspace_size(const anqs_model* M, const anqs_ham* H, uint64_t n_x, size_t* bytes) {
  ANQS_TRY(check_pair(M, H));
  if (!bytes) return set_error(ANQS_ERR_ARG, "null output");
  *bytes = grad_ws_bytes(M, n_x, false);
  return ANQS_OK;
}

int anqs_grad_workspace_size_min(const anqs_model* M, const anqs_ham* H, uint64_t n_x, size_t* bytes) {
  ANQS_TRY(check_pair(M, H));
  if (!bytes) return set_error(ANQS_ERR_ARG, "null output");
  *bytes = grad_ws_bytes(M, n_x, true);
  return ANQS_OK;
}

int anqs_grad(const anqs_model* M, const anqs_ham* H, const uint64_t* x, const uint64_t* counts, uint64_t n_x,
              const uint64_t* n_x_dev, const double* ere, const double* eim, const double* stats, float* grad,
              void* ws, size_t ws_bytes, void* stream) {
  ANQS_TRY(check_pair(M, H));
  if (n_x == 0) return set_error(ANQS_ERR_ARG, "n_x must be >= 1");
  if (!x || !counts || !ere || !eim || !stats || !grad) return set_error(ANQS_ERR_ARG, "null array argument");
  ANQS_TRY(check_adjoint(M));
  Arena A(ws, ws_bytes);
  float* cl = A.take<float>(n_x);
  float* cp = A.take<float>(n_x);
  float* part = (M->d.kind == ANQS_MODEL_MLP) ? A.take<float>(mlp_fp32_grad_partial_floats(M->mlp, n_x)) : nullptr;
  size_t tfb = vjp_ws_bytes(M, n_x);
  const size_t off0 = A.off;
  void* tfws = tfb ? A.take<char>(tfb) : nullptr;
  if (!A.fits() && tfb) {  // too small for every activation: the recomputing adjoint
    A.off = off0;
    tfb = vjp_ws_bytes(M, n_x, true);
    tfws = A.take<char>(tfb);
  }
  if (!A.fits() || !ws) return set_error(ANQS_ERR_CAPACITY, "workspace needs %zu bytes", A.off);
  cudaStream_t s = (cudaStream_t)stream;
  if (!part) ANQS_CUDA(cudaMemsetAsync(grad, 0, M->n_params * sizeof(float), s));
  const Count nc{n_x, n_x_dev, 1};
  // the MLP and NADE adjoints compute each row's cotangents themselves
  const CotSrc vmc{nullptr, nullptr, ere, eim, stats, counts};
  if (M->d.kind == ANQS_MODEL_MLP) {
    if (M->d.form == ANQS_FORM_BF16 && mlp_tc_grad_supported(M))  // 16-bit forward and adjoint on the tensor cores
      return launch_mlp_tc_grad(M, H->v, x, nc, vmc, grad, part, s);
    return launch_mlp_fp32_grad(M->mlp, H->v, x, nc, vmc, grad, part, s);
  }
  if (M->d.kind == ANQS_MODEL_NADE)
    return launch_nade_grad(M->nade, H->v, x, nc, vmc, grad, M->n_params, static_cast<float*>(tfws), s);
  ANQS_TRY(launch_grad_cotangents(ere, eim, counts, stats, nc, cl, cp, s));
  return vjp_dispatch(M, H, x, nc, cl, cp, grad, part, tfws, tfb, s);
}

int anqs_logpsi_vjp_workspace_size(const anqs_model* M, const anqs_ham* H, uint64_t n_x, size_t* bytes) {
  ANQS_TRY(check_pair(M, H));
  if (!bytes) return set_error(ANQS_ERR_ARG, "null output");
  *bytes = vjp_ws_bytes(M, n_x);
  return ANQS_OK;
}

int anqs_logpsi_vjp(const anqs_model* M, const anqs_ham* H, const uint64_t* x, uint64_t n_x, const float* cl,
                    const float* cp, float* grad, void* ws, size_t ws_bytes, void* stream) {
  ANQS_TRY(check_pair(M, H));
  if (!grad) return set_error(ANQS_ERR_ARG, "null gradient output");
  if (n_x && (!x || !cl || !cp)) return set_error(ANQS_ERR_ARG, "null array argument");
  ANQS_TRY(check_adjoint(M));
  const size_t need = vjp_ws_bytes(M, n_x, true);  // with less than vjp_ws_bytes(M, n_x) the transformer recomputes
  if (ws_bytes < need || (need && !ws)) return set_error(ANQS_ERR_CAPACITY, "workspace needs %zu bytes", need);
  cudaStream_t s = (cudaStream_t)stream;
  ANQS_CUDA(cudaMemsetAsync(grad, 0, M->n_params * sizeof(float), s));
  if (n_x == 0) return ANQS_OK;
  return vjp_dispatch(M, H, x, host_count(n_x), cl, cp, grad, nullptr, ws, ws_bytes, s);
}

}  // extern "C"
