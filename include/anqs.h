/*
 * anqs.h - C ABI of libanqs: the data-parallel hot path of symmetry-masked
 * autoregressive variational Monte Carlo for second-quantised molecular
 * Hamiltonians (Malyshev, Arrazola, Lvovsky, arXiv:2310.04166), on one
 * NVIDIA GB300 (sm_103a).
 *
 * Conventions shared by every call
 * --------------------------------
 * - Determinants are uint64 occupation strings.  Bit q is the occupation of
 *   spin-orbital q = 2 p + s (spatial orbital p, s = 0 alpha, 1 beta): the
 *   interleaved ordering of Appendix A (odd 1-based qubits carry spin up)
 *   under the Jordan-Wigner encoding of Sec. IV.A.  The autoregressive unit
 *   is the spatial orbital ("slot"): v_p = x_{2p} + 2 x_{2p+1} in {0..3}.
 *   At most 32 spatial orbitals.
 * - Every function returns ANQS_OK (0) or a negative ANQS_ERR_* code; the
 *   message of the last error on the calling thread is available from
 *   anqs_last_error().  Argument errors are detected on the host before any
 *   work is queued.  Nothing in the library traps or asserts on the device.
 * - Array arguments named *_dev are DEVICE pointers owned by the caller; the
 *   library never frees or reallocates them.  Arguments named *_host are
 *   host pointers, read before the call returns.
 * - Calls that take a stream are asynchronous with respect to the host and
 *   ordered on that stream (a cudaStream_t passed as void*, NULL = the
 *   legacy default stream).  They allocate nothing: scratch memory comes
 *   from the caller as (workspace_dev, workspace_bytes), sized by the
 *   matching *_workspace_size() query, 256-byte aligned.
 * - Handles (anqs_ham, anqs_model) are created on the current CUDA device,
 *   own their device memory and are released by *_destroy.
 *
 * Network parameters (flat float32 arrays, device memory, caller-owned):
 *   ANQS_MODEL_MLP  for each slot p = 0..n-1, for each layer k = 1..L+1:
 *                   W_k [out][in] row-major (absent for k = 1, p = 0), b_k [out].
 *                   Layer 1 maps the one-hot of v_<p (in = 4p, index 4q+v_q)
 *                   to `width`, layers 2..L map width -> width (tanh after
 *                   each hidden layer), the head maps width -> 8 outputs:
 *                   modulus logits l_0..l_3, then phases phi_0..phi_3.
 *   ANQS_MODEL_TF   tok[5][d] (rows 0..3 slot values, row 4 start token),
 *                   pos[n][d], per layer: ln1_g[d] ln1_b[d] wq[d][d] bq[d]
 *                   wk[d][d] bk[d] wv[d][d] bv[d] wo[d][d] bo[d] ln2_g[d]
 *                   ln2_b[d] w1[4d][d] b1[4d] w2[d][4d] b2[d], then lnf_g[d]
 *                   lnf_b[d] head_w[8][d] head_b[8].  Pre-LayerNorm (eps
 *                   1e-5) causal blocks, ReLU FFN; position t reads the start
 *                   token (t = 0) or v_{t-1} and outputs slot t's 8 values.
 *   ANQS_MODEL_TABLE for each slot p: table_p[4^p][8], row = the prefix bits
 *                   x & (4^p - 1).  n <= 11.
 *   ANQS_MODEL_NADE the per-qubit complex NADE of Appendix B.1 (FP32 form
 *                   only, width in {32, 64, 128}, n_orb <= 32).  For each
 *                   qubit i = 0..2n-1 (q = 2p + sigma, alpha first): W1
 *                   [w][i], b1 [w], W2 [w][w], b2 [w], W3 [2][w], b3 [2],
 *                   complex, row-major, each entry (re, im) interleaved.
 *                   z1 = W1 x_<i + b1, h1 = tanh(z1) (complex), z2 = W2 h1 +
 *                   b2, h2 = LeReLU(Re z2) + i LeReLU(Im z2) (slope 0.01
 *                   below zero), z3 = W3 h2 + b3, f3(z3) = z3 - LSE(2 Re
 *                   z3) / 2 = (log psi_i(0), log psi_i(1)).  Slot p's values
 *                   are l_v = 2 Re, phi_v = Im of log psi_2p(a) + log
 *                   psi_2p+1(b | a), v = a + 2b; on MU slots each qubit's
 *                   modulus is first renormalised over the values with an
 *                   allowed slot outcome (b given a for qubit 2p+1).
 * Slot conditional (Appendix B.1, activation f3, with MU masking of
 * Sec. III.C): |psi_p(v)|^2 = exp(l_v) / sum_{u allowed} exp(l_u) over the
 * outcomes u that can still reach the (N_alpha, N_beta) sector, 0 for the
 * others; arg psi_p(v) = phi_v.  log psi(x) = sum_p log psi_p(v_p | v_<p)
 * (Eq. anqs_def).
 */
#ifndef ANQS_H
#define ANQS_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define ANQS_API __attribute__((visibility("default")))
#else
#define ANQS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

enum {
  ANQS_OK = 0,
  ANQS_ERR_ARG = -1,         /* invalid argument (null pointer, size, mismatch) */
  ANQS_ERR_CAPACITY = -2,    /* an output or workspace is too small */
  ANQS_ERR_SECTOR = -3,      /* the requested sector is empty or invalid */
  ANQS_ERR_CUDA = -4,        /* a CUDA runtime call failed (message has the name) */
  ANQS_ERR_UNSUPPORTED = -5  /* configuration outside the supported range */
};

enum { ANQS_MODEL_MLP = 0, ANQS_MODEL_TF = 1, ANQS_MODEL_TABLE = 2, ANQS_MODEL_NADE = 3 };

/* Arithmetic form of a model's network evaluation.
 * FP32: plain SIMT float32 kernels, every configuration evaluated over all
 *       slots (no prefix reuse), except the NADE, whose local energy reuses
 *       the parent's slots for its connected determinants.
 * BF16: the 16-bit form: tensor-core (tcgen05, TMEM accumulators) 16-bit
 *       GEMMs with float32 accumulation, float32 activations/softmax/phase
 *       heads, and reuse of the parent determinant's slots for its connected
 *       determinants.  GEMM operands are fp16, the same MMA instruction and
 *       rate as bfloat16 with three more significand bits (the bf16 rounding
 *       of activations put the gradient's error above 1e-3 relative L2):
 *       the MLP's weights (layer 1 as two fp16 parts) and tanh activations,
 *       the transformer's activations and stored keys/values (its weights are
 *       bf16-representable, hence exact in fp16).  Conversions saturate at
 *       +-65504.  MLP width 64 or 128, transformer d_model 64 (at most 4
 *       blocks) or 128 with head width 16 or 32. */
enum { ANQS_FORM_FP32 = 0, ANQS_FORM_BF16 = 1 };

typedef struct anqs_ham anqs_ham;
typedef struct anqs_model anqs_model;

typedef struct {
  int32_t kind;      /* ANQS_MODEL_* */
  int32_t form;      /* ANQS_FORM_* (TABLE: FP32 only) */
  int32_t n_orb;     /* spatial orbitals n (slots), 1..32 */
  int32_t width;     /* MLP: hidden width in {64, 128, 256}; NADE: in {32, 64, 128} */
  int32_t n_hidden;  /* MLP: hidden layers L (1..8) */
  int32_t d_model;   /* TF: model width d in {32, 64, 128, 256} */
  int32_t n_heads;   /* TF: heads (d_model % n_heads == 0) */
  int32_t n_layers;  /* TF: blocks */
} anqs_model_desc;

/* Library version string (static storage). */
ANQS_API const char* anqs_version(void);

/* Copy the last error message of the calling thread into buf (always
 * NUL-terminated when len > 0).  Returns the code of that error. */
ANQS_API int anqs_last_error(char* buf, size_t len);

/* ---------------------------------------------------------------------------
 * Hamiltonian and sector (Eq. sq_hamiltonian, Sec. IV.A; Alg. 1)
 *
 * H = E_nuc + sum_{pq,s} h_pq a+_{ps} a_{qs}
 *           + 1/2 sum_{pqrs,s,t} g_pqrs a+_{ps} a+_{rt} a_{st} a_{qs}
 * with real chemist-notation integrals g_pqrs = (pq|rs) (8-fold symmetric)
 * and symmetric h.  The sector is fixed by N_alpha and N_beta, i.e. by the
 * particle number and S_z of the reference determinant (Sec. IV.A,
 * Appendix A).  At creation the library evaluates IsPhys (Algorithm 1) over
 * the qubit tree with the additive n_e and S_z symmetries and stores, for
 * every slot p and partial counts (a, b), the 4-bit mask of outcomes that
 * still reach the sector.
 *
 * h_host: n*n doubles, row-major.  g_host: n^4 doubles, index
 * ((p*n+q)*n+r)*n+s.  Copied to the current device; synchronous.
 * Errors: ANQS_ERR_ARG (null, n outside 1..32), ANQS_ERR_SECTOR (N_alpha or
 * N_beta outside 0..n), ANQS_ERR_CUDA.
 * ------------------------------------------------------------------------- */
ANQS_API int anqs_hamiltonian_create(anqs_ham** out, int n_orb, int n_alpha, int n_beta,
                            const double* h_host, const double* g_host, double e_nuc);
ANQS_API int anqs_hamiltonian_destroy(anqs_ham* ham);

/* Pruning strategy of unphysical subtrees (Sec. III.C, Fig. 1C): MU-d with
 * d = du_levels, i.e. MU on the first n_orb - d slots and DU on the last d
 * (slot levels of the library's 4-way tree).  d = 0 (the default) is MU:
 * conditionals are renormalised over the allowed outcomes and no sample is
 * lost.  d = n_orb is DU: on a DU level the conditional is the network's
 * softmax over all four outcomes, and samples drawn into an unphysical child
 * are discarded, so the counts may add up to less than n_samples; amplitudes
 * of sector determinants use the same unmasked conditionals on those levels
 * (log psi of a determinant outside the sector stays -inf).  Applies to
 * every later call with this Hamiltonian (sampling, log psi, local energy,
 * gradient).  ANQS_ERR_ARG unless 0 <= du_levels <= n_orb. */
ANQS_API int anqs_hamiltonian_set_pruning(anqs_ham* ham, int du_levels);

/* Sampler events recorded on the device for this Hamiltonian since its
 * creation or the last clear, as a bit set:
 *   ANQS_HAM_BINOMIAL_REJECT  a binomial draw of anqs_sample_binomial left
 *                             the BTRS rejection loop (Hormann 1993) after 256
 *                             rejections and took the mode;
 *   ANQS_HAM_BINOMIAL_CAP     a pmf-inversion walk (n q < 10) stopped at
 *                             k = 4096.
 * Both have negligible probability; either makes that one draw biased.
 * Synchronous (reads one word); clear != 0 resets the word.  ANQS_ERR_ARG
 * for a null pointer. */
#define ANQS_HAM_BINOMIAL_REJECT 1
#define ANQS_HAM_BINOMIAL_CAP 2
ANQS_API int anqs_hamiltonian_status(const anqs_ham* ham, int* status, int clear);

/* Z2 symmetries of H (Sec. IV.A: Pauli-Z strings that commute with H, such
 * as the images of the abelian point-group operations under the
 * Jordan-Wigner transform).  qubit_masks[j] (host) has bit q set when
 * symmetry j acts with Z on qubit q = 2p + sigma.  The target eigenvalues
 * are those of the reference determinant (the lowest N_alpha alpha and
 * N_beta beta orbitals occupied); IsPhys (Algorithm 1) then masks every
 * outcome that cannot reach them, on top of the electron counts, so the
 * sampler, the amplitudes and the sector dimension all refer to the smaller
 * sector.  The caller guarantees that the strings commute with H (the
 * connected set is not filtered: an excitation that changes a parity has
 * H_xx' = 0 and psi(x') = 0).  0 <= nz <= 4 (nz = 0 removes them); each mask
 * within the 2 n_orb qubits.  ANQS_ERR_SECTOR (and no change) when the
 * resulting sector is empty. */
ANQS_API int anqs_hamiltonian_set_z2(anqs_ham* ham, int nz, const uint64_t* qubit_masks);

/* n_connected: off-diagonal determinants connected to every sector
 * determinant by H (same for all of them):
 *   Na(n-Na) + Nb(n-Nb) + C(Na,2)C(n-Na,2) + C(Nb,2)C(n-Nb,2) + Na(n-Na)Nb(n-Nb).
 * sector_dim: the number of determinants in the sector (C(n,Na) C(n,Nb)
 * without Z2 symmetries; saturated at UINT64_MAX).  Either may be NULL. */
ANQS_API int anqs_hamiltonian_info(const anqs_ham* ham, uint64_t* n_connected, uint64_t* sector_dim);

/* Slot mask table computed by IsPhys: out_host receives
 * n*(Na+1)*(Nb+1)*2^nz bytes (nz = number of Z2 symmetries set), entry
 * [((p*(Na+1)+a)*(Nb+1)+b)*2^nz+z] = bit v set when outcome v of slot p is
 * allowed after a prefix holding a alpha and b beta electrons whose Z2
 * parities are the bits of z (0 when the prefix itself is unphysical).  len
 * must be at least that size. */
ANQS_API int anqs_hamiltonian_slot_masks(const anqs_ham* ham, uint8_t* out_host, size_t len);

/* ---------------------------------------------------------------------------
 * Connected set (Eq. local_energy_def: the x' with H_xx' != 0 by symmetry)
 *
 * For each of the n_x sector determinants x_dev[l], writes its K =
 * n_connected off-diagonal connected determinants to xp_dev[l*K + k], the
 * matrix elements <x'|H|x> (FP64, Slater-Condon rules, Jordan-Wigner signs)
 * to hval_dev[l*K + k], and optionally the first slot in which x' differs
 * from x to first_slot_dev[l*K + k] and the diagonal element <x|H|x> to
 * hdiag_dev[l].  Order within a row, fixed and documented so that lists can
 * be compared element by element: alpha singles, beta singles (each (I, A)
 * ascending, spatial indices), alpha-alpha doubles, beta-beta doubles (each
 * (I, J, A, B) lexicographic with I < J, A < B), alpha-beta doubles
 * (I_a, A_a, I_b, A_b) lexicographic.  Zero elements are kept.
 * A determinant outside the sector gets xp = x, hval = NaN, first_slot = 255
 * and hdiag = NaN on its row (no error code: the check runs on the device).
 * first_slot_dev and hdiag_dev may be NULL.  n_x may be 0.
 * ------------------------------------------------------------------------- */
ANQS_API int anqs_connected(const anqs_ham* ham, const uint64_t* x_dev, uint64_t n_x,
                   uint64_t* xp_dev, double* hval_dev, uint8_t* first_slot_dev,
                   double* hdiag_dev, void* stream);

/* ---------------------------------------------------------------------------
 * Model (Eq. anqs_def; Appendix B.1; MU masking Sec. III.C)
 * ------------------------------------------------------------------------- */
/* Number of float32 parameters of a model description. */
ANQS_API int anqs_model_param_count(const anqs_model_desc* desc, uint64_t* n_params);

/* Creates a model over params_dev (n_params floats, caller-owned device
 * memory that must outlive the model; the library keeps the pointer).  The
 * BF16 form keeps packed 16-bit copies of the weights: call
 * anqs_model_sync() after changing params_dev.  Synchronous.
 * Errors: ANQS_ERR_ARG, ANQS_ERR_UNSUPPORTED (sizes outside the ranges of
 * anqs_model_desc), ANQS_ERR_CUDA. */
ANQS_API int anqs_model_create(anqs_model** out, const anqs_model_desc* desc, const float* params_dev);
ANQS_API int anqs_model_destroy(anqs_model* model);

/* Re-derive the model's internal copies from params_dev, ordered on stream. */
ANQS_API int anqs_model_sync(anqs_model* model, void* stream);

/* log psi(x) for n_x determinants: log_abs_dev[l] = log|psi(x_l)|,
 * phase_dev[l] = arg psi(x_l) (unwrapped sum of slot phases), float32.
 * A determinant outside the sector has log_abs = -inf.  The model's n_orb
 * must equal the Hamiltonian's.  The BF16 form stages raw slot outputs in a
 * scratch buffer owned by the model: calls on the same BF16 model must not
 * run concurrently on different streams. */
ANQS_API int anqs_logpsi(const anqs_model* model, const anqs_ham* ham, const uint64_t* x_dev,
                uint64_t n_x, float* log_abs_dev, float* phase_dev, void* stream);

/* ---------------------------------------------------------------------------
 * Masked autoregressive statistics sampling (Sec. II.C with MU, Sec. III.C)
 *
 * Walks the slot tree breadth first.  A node with n_in samples splits them
 * among its allowed outcomes by n_in uniform draws u_i: sample i takes the
 * first allowed v with u_i < C_v, C_v the running sum of the masked
 * conditional over allowed outcomes in ascending v (the last allowed v if
 * rounding leaves u_i >= C_last).  The masked conditional is evaluated from
 * the network's float32 logits in float32 by a fixed sequence of IEEE
 * operations without fused multiply-adds: e_v = exp(l_v - max) by Cody-Waite
 * reduction and a degree-7 Taylor polynomial, the sum over allowed v in
 * ascending order, p_v = e_v / sum, C_v the running sum.  u_i comes
 * from Philox4x64-10 (Salmon et al., SC'11) with counter (prefix, i >> 2,
 * slot, counter) and key (seed, 0), word i & 3, top 53 bits times 2^-53.
 * Children with zero samples are dropped; no sample is lost (MU), so the
 * counts add up to n_samples.
 *
 * Output: *n_unique_dev (device uint64) = N_unq; x_out_dev[0..N_unq) the
 * unique determinants in lexicographic order of (v_0, v_1, ..., v_{n-1}),
 * n_out_dev their occurrence numbers.  cap must be at least
 * min(n_samples, sector_dim) (checked on the host: ANQS_ERR_CAPACITY).
 * n_samples >= 1.  The Philox counter word is counter + *counter_dev when
 * counter_dev (a device uint64) is not NULL, so that a captured CUDA graph
 * can draw fresh samples on every replay by advancing *counter_dev.
 * ------------------------------------------------------------------------- */
ANQS_API int anqs_sample_workspace_size(const anqs_model* model, const anqs_ham* ham,
                               uint64_t n_samples, size_t* bytes);
ANQS_API int anqs_sample(const anqs_model* model, const anqs_ham* ham, uint64_t n_samples,
                uint64_t seed, uint64_t counter, const uint64_t* counter_dev, uint64_t* x_out_dev,
                uint64_t* n_out_dev, uint64_t cap, uint64_t* n_unique_dev, void* workspace_dev,
                size_t workspace_bytes, void* stream);

/* Binomial statistics sampling (Sec. II.C, the trick of Barrett et al.):
 * the same tree walk, but a node splits its n_in samples by chained
 * binomials instead of n_in draws, so the cost per node does not depend on
 * n_in and n_samples can reach 1e8 and beyond.  For the allowed outcomes in
 * ascending v: k_v ~ B(rest, p_v / (p_v + ... + p_last)), rest -= k_v; the
 * last allowed outcome takes the rest (MU: nothing is lost).  p is the same
 * float32 masked conditional as above.  B(n, q) is drawn with q' = min(q,
 * 1 - q) by inversion of the pmf when n q' < 10, else by BTRS (Hormann 1993,
 * transformed rejection with squeeze; log Gamma by the Stirling series), in
 * FP64.  Uniforms: Philox4x64-10 with counter (prefix, (v << 32) | block,
 * slot, counter) and key (seed, 1), four per block.  The counts are an exact
 * multinomial split in distribution; they are not the counts of
 * anqs_sample.  Arguments and outputs as anqs_sample (same workspace). */
ANQS_API int anqs_sample_binomial(const anqs_model* model, const anqs_ham* ham, uint64_t n_samples, uint64_t seed,
                                  uint64_t counter, const uint64_t* counter_dev, uint64_t* x_out_dev,
                                  uint64_t* n_out_dev, uint64_t cap, uint64_t* n_unique_dev, void* workspace_dev,
                                  size_t workspace_bytes, void* stream);

/* One rank's share of the same sampling pass on `world` GPUs (the data-
 * parallel split of the tree: subtrees are independent).  Every rank walks
 * levels 0..split_level-1 exactly as anqs_sample does; the level-split_level
 * frontier (the output when split_level = n_orb) is then reduced to its
 * nodes i with i % world == rank, and the walk continues from those.  The
 * draws of a node depend only on its prefix, so the union over the ranks of
 * their outputs is exactly the output of anqs_sample with the same seed and
 * counter, and the counts add up to n_samples.  Energy statistics and
 * gradients of the shards combine by sums over the ranks (the host-side
 * exchange: S, S E, S (Var + |E|^2) and the gradient; anqs_grad takes the
 * combined stats).  Arguments otherwise as anqs_sample. */
ANQS_API int anqs_sample_shard(const anqs_model* model, const anqs_ham* ham, uint64_t n_samples, uint64_t seed,
                               uint64_t counter, const uint64_t* counter_dev, int rank, int world, int split_level,
                               uint64_t* x_out_dev, uint64_t* n_out_dev, uint64_t cap, uint64_t* n_unique_dev,
                               void* workspace_dev, size_t workspace_bytes, void* stream);

/* Energy statistics of the union of `world` disjoint sample sets (the
 * estimator of Eq. energy_est over all ranks' samples) from each set's
 * statistics: stats_in_dev [world][4] (layout of anqs_local_energy's stats),
 * stats_out_dev [4]:  S = sum S_r,  E = sum S_r E_r / S,
 * Var = sum S_r (Var_r + |E_r - E|^2) / S; sets with S_r = 0 (an empty
 * shard, whose E_r is 0/0) are skipped.  FP64, one thread; stats_in_dev
 * and stats_out_dev may not overlap.  ANQS_ERR_ARG for world < 1 or null
 * pointers. */
ANQS_API int anqs_stats_combine(const double* stats_in_dev, int world, double* stats_out_dev, void* stream);

/* Device-side status of the model's BF16 tensor-core kernels (synchronous):
 * 0, or 1 when a bounded wait inside a kernel (weight copy or MMA completion,
 * 2 s each) or the persistent sampler's grid barrier (2 s per level) gave up
 * since the model was created; the kernel then stopped and the outputs of
 * that call are invalid (a sampling pass that gave up returns n_unique = 0).
 * Always 0 for the FP32 forms. */
ANQS_API int anqs_model_status(const anqs_model* model, int* status);

/* Test hook for failure detection without a GPU fault (process-wide, not
 * thread-safe; set it only while no sampling call is being queued).  With
 * extra_arrivals > 0 every grid barrier of the persistent sampler waits for
 * that many CTAs more than its grid has, an arrival that never comes, and
 * gives up after limit_ns (0: the default 2 s): every CTA leaves, the model's
 * status word is set and the pass returns no samples.  extra_arrivals = 0 and
 * limit_ns = 0 restore the defaults.  Always ANQS_OK. */
ANQS_API int anqs_test_sampler_barrier(unsigned extra_arrivals, uint64_t limit_ns);

/* ---------------------------------------------------------------------------
 * Local energy and energy statistics (Eq. local_energy_def, Eq. energy_est)
 *
 * eloc[l] = H_xx + sum_k H_{x x'_k} exp(log psi(x'_k) - log psi(x)), complex,
 * accumulated in FP64 over the K connected determinants of x = x_dev[l].
 * If counts_dev is not NULL, stats_dev receives 4 doubles
 *   (Re E, Im E, Var, S) with S = sum_l n_l, E = sum_l n_l eloc_l / S,
 *   Var = sum_l n_l |eloc_l - E|^2 / S.
 * n_x >= 1.  Workspace from anqs_local_energy_workspace_size(n_x).
 * Row count on the device: when n_x_dev is not NULL, only the first *n_x_dev
 * rows (read on the device, at most n_x) are processed and n_x is the
 * capacity that sizes launches and the workspace; e.g. pass the sampler's
 * n_unique_dev so that sampling, local energy and gradient can be captured
 * in one CUDA graph.  Outputs beyond *n_x_dev are left untouched.
 * The statistics are reduced in a fixed order (deterministic), in one pass
 * shifted by eloc_0 (equal to the two-pass form up to rounding).
 * The 16-bit MLP form runs part of the call on a second stream owned by the
 * model, forked from `stream` and joined back into it with events: the call
 * still orders with the work queued on `stream` and can be captured in a
 * CUDA graph, but one model must not be used by several host threads at once.
 * ------------------------------------------------------------------------- */
ANQS_API int anqs_local_energy_workspace_size(const anqs_model* model, const anqs_ham* ham,
                                     uint64_t n_x, size_t* bytes);
ANQS_API int anqs_local_energy(const anqs_model* model, const anqs_ham* ham, const uint64_t* x_dev,
                      const uint64_t* counts_dev, uint64_t n_x, const uint64_t* n_x_dev,
                      double* eloc_re_dev, double* eloc_im_dev, double* stats_dev, void* workspace_dev,
                      size_t workspace_bytes, void* stream);

/* ---------------------------------------------------------------------------
 * Batched local energy (no counterpart in the paper, which treats one
 * molecule at a time: many independent problems in one call)
 *
 * anqs_eloc_problem holds the arguments of one anqs_local_energy call.
 * anqs_batched_local_energy computes every problem's local energies and
 * statistics exactly as anqs_local_energy would, each problem on its own
 * stream of the batch handle, forked from `stream` with an event and joined
 * back into it with one event per problem: the problems run side by side,
 * after the work queued on `stream` before the call and before the work
 * queued after it.  The fork and join are ordinary event dependencies, so
 * the call can be recorded into a CUDA graph by capturing `stream`.
 * - Every problem is checked (model/Hamiltonian pair, n_x >= 1, arrays,
 *   workspace size from anqs_local_energy_workspace_size) before anything is
 *   queued; errors: ANQS_ERR_ARG, ANQS_ERR_CAPACITY (a workspace too small or
 *   more problems than the handle's streams), ANQS_ERR_UNSUPPORTED, as for
 *   anqs_local_energy.  A CUDA error while queueing (ANQS_ERR_CUDA) still
 *   joins the work already queued into `stream`.
 * - Problems may share a model or a Hamiltonian (read only) but not their
 *   outputs or workspaces.
 * - Persistent launch: the 16-bit MLP problems of one width (the width of
 *   the first such problem, at most 32 of them) share one launch for their
 *   amplitude stage, the connected determinants' slots (the bulk of the
 *   work).  Their earlier stages (connected set, parents, sort by first
 *   slot) run on their streams; the caller's stream then waits for all of
 *   them and runs one plan kernel and one persistent kernel of one CTA per
 *   SM over every (problem, slot, tile); each problem's assembly and
 *   statistics then run on its stream again.  Results are bit-identical to
 *   anqs_local_energy's.  Other problems run whole on their streams.
 * - Schedule of the persistent launch (anqs_batch_set_schedule).  The
 *   128-row tiles of every (problem, slot) form one sequence in
 *   problem-major order.  ANQS_BATCH_STATIC: CTA i of G takes the tiles
 *   [i T / G, (i + 1) T / G) (chunk unused).  ANQS_BATCH_DYNAMIC (the
 *   default, chunk 8): work items of `chunk` tiles of one (problem, slot)
 *   taken from a global counter.  ANQS_BATCH_STREAMS: every problem whole on
 *   its own stream (no persistent launch).
 * - anqs_batch_autotune times the persistent launch on the given problems
 *   for each candidate schedule (STATIC, then DYNAMIC with chunk 8, 16, 32,
 *   64, 128, 256, 512; times_ms, if not NULL, receives the 8 times in ms,
 *   CUDA events on `stream`) and keeps the fastest in the handle.  It runs the
 *   batched call 9 times (outputs are overwritten, inputs unchanged) and
 *   synchronises `stream`; it must not be called while `stream` is being
 *   captured (ANQS_ERR_ARG), and returns ANQS_ERR_UNSUPPORTED when no
 *   problem would use the persistent launch.
 * - The handle owns max_problems non-blocking streams, 2 max_problems + 4
 *   events and 16 KB of device memory (the persistent launch's work groups)
 *   on the device current at creation; a handle serves one call at a time
 *   (calls on it are ordered by the caller).
 * ------------------------------------------------------------------------- */
typedef struct anqs_batch anqs_batch;

typedef struct {
  const anqs_model* model;
  const anqs_ham* ham;
  const uint64_t* x_dev;
  const uint64_t* counts_dev;   /* or NULL (then no statistics) */
  uint64_t n_x;
  const uint64_t* n_x_dev;      /* or NULL */
  double* eloc_re_dev;
  double* eloc_im_dev;
  double* stats_dev;            /* 4 doubles, required with counts_dev */
  void* workspace_dev;
  size_t workspace_bytes;
} anqs_eloc_problem;

ANQS_API int anqs_batch_create(anqs_batch** out, int max_problems);
ANQS_API int anqs_batch_destroy(anqs_batch* batch);
ANQS_API int anqs_batched_local_energy(anqs_batch* batch, const anqs_eloc_problem* problems_host, int n_problems,
                                       void* stream);

enum { ANQS_BATCH_STREAMS = 0, ANQS_BATCH_STATIC = 1, ANQS_BATCH_DYNAMIC = 2 };
ANQS_API int anqs_batch_set_schedule(anqs_batch* batch, int mode, int chunk);
ANQS_API int anqs_batch_get_schedule(const anqs_batch* batch, int* mode, int* chunk);
ANQS_API int anqs_batch_autotune(anqs_batch* batch, const anqs_eloc_problem* problems_host, int n_problems,
                                 void* stream, float* times_ms);

/* ---------------------------------------------------------------------------
 * VMC gradient (Eq. grad_def)
 *
 * grad = 2 Re{ E[eloc d ln psi*] - E[eloc] E[d ln psi*] } with expectations
 * weighted by n_l / S and eloc held fixed:
 *   grad = sum_l (n_l/S) 2 [ Re(eloc_l - E) d log|psi(x_l)| + Im(eloc_l - E) d arg psi(x_l) ]
 * with E = stats[0] + i stats[1] and S = stats[3] (as written by
 * anqs_local_energy).  grad_dev: n_params floats, overwritten.  n_x_dev as
 * for anqs_local_energy.
 * Hand-written adjoint of the masked log psi (MLP, transformer, NADE); the
 * table model returns ANQS_ERR_UNSUPPORTED before anything is queued.
 * ------------------------------------------------------------------------- */
ANQS_API int anqs_grad_workspace_size(const anqs_model* model, const anqs_ham* ham, uint64_t n_x,
                             size_t* bytes);
/* The smallest workspace anqs_grad accepts.  For the transformer it holds
 * only each block's input rows: given less than anqs_grad_workspace_size,
 * the adjoint recomputes a block's activations from its input just before
 * that block's backward (one more forward pass; about a third of the memory
 * at 4 blocks of width 128).  Equal to anqs_grad_workspace_size for the other
 * kinds. */
ANQS_API int anqs_grad_workspace_size_min(const anqs_model* model, const anqs_ham* ham, uint64_t n_x,
                                          size_t* bytes);
ANQS_API int anqs_grad(const anqs_model* model, const anqs_ham* ham, const uint64_t* x_dev,
              const uint64_t* counts_dev, uint64_t n_x, const uint64_t* n_x_dev,
              const double* eloc_re_dev, const double* eloc_im_dev, const double* stats_dev,
              float* grad_dev, void* workspace_dev, size_t workspace_bytes, void* stream);

/* Adjoint of the masked log psi (vector-Jacobian product): grad_dev
 * (n_params floats, overwritten) = d/dtheta sum_l [cot_abs_dev[l] log|psi(x_l)|
 * + cot_phase_dev[l] arg psi(x_l)].  anqs_grad is this product with the
 * cotangents 2 (n_l/S) Re(eloc_l - E) and 2 (n_l/S) Im(eloc_l - E).
 * The transformer's adjoint keeps every forward activation of the n_x
 * determinants in the workspace (anqs_logpsi_vjp_workspace_size), or, when
 * given less, only the block inputs, recomputing each block's activations
 * before its backward (the least it accepts is the size anqs_grad needs
 * beyond its cotangents, see anqs_grad_workspace_size_min); the NADE's
 * uses it for per-CTA partial gradients when its rows span several tile
 * groups; the MLP's needs none (workspace may be null).  The table model has
 * no adjoint: ANQS_ERR_UNSUPPORTED before anything is queued. */
ANQS_API int anqs_logpsi_vjp_workspace_size(const anqs_model* model, const anqs_ham* ham, uint64_t n_x,
                                            size_t* bytes);
ANQS_API int anqs_logpsi_vjp(const anqs_model* model, const anqs_ham* ham, const uint64_t* x_dev, uint64_t n_x,
                    const float* cot_abs_dev, const float* cot_phase_dev, float* grad_dev, void* workspace_dev,
                    size_t workspace_bytes, void* stream);

/* ---------------------------------------------------------------------------
 * Local energy without caller workspace (the paper has no counterpart: this
 * is an interface for callers that cannot allocate device memory)
 *
 * Same computation and outputs as anqs_local_energy for FP32-form models
 * (MLP, transformer, table, NADE), but the scratch memory lives in a fixed
 * 16 MiB array inside
 * the library (one per GPU that loads it, kept until the process exits)
 * instead of a caller-provided workspace, and nothing is allocated.  Meant
 * for callers that cannot hand out device memory at run time, e.g. plug-ins
 * whose host application owns all device allocations, or loops that must not
 * call cudaMalloc after start-up.
 * - Needs n_x * n_connected * 24 + n_x * 16 bytes (plus alignment) to fit in
 *   16 MiB; larger requests fail with ANQS_ERR_CAPACITY before any work is
 *   queued.  BF16 forms: ANQS_ERR_UNSUPPORTED.
 * - The first call on a device looks up the array's device address (with
 *   that device current); make that first call before any stream capture.
 *   A context made anew on the device (e.g. after cudaDeviceReset) makes the
 *   next call look the address up again, so make that call outside capture
 *   too.
 * - All calls on a device share the array: calls that may run concurrently
 *   on the GPU race and must be ordered by the caller.  Every scratch
 *   element is written before it is read, so no clearing is needed.
 * ------------------------------------------------------------------------- */
ANQS_API int anqs_local_energy_static(const anqs_model* model, const anqs_ham* ham, const uint64_t* x_dev,
                                      const uint64_t* counts_dev, uint64_t n_x, double* eloc_re_dev,
                                      double* eloc_im_dev, double* stats_dev, void* stream);

/* ---------------------------------------------------------------------------
 * Instrumentation (no counterpart in the paper: measurement support)
 *
 * anqs_launch_count: number of CUDA kernels the library has launched in this
 * process.  anqs_profile_enable(on): clears the totals and switches CUDA-event
 * timing of the library's kernel families on or off (off by default; events
 * are recorded on the launching stream; do not enable while capturing a
 * graph).  anqs_profile_read(id, ...): waits for the recorded events and
 * returns the family's name (static storage), launch count and summed
 * device time in milliseconds; ids run from 0 until it returns ANQS_ERR_ARG.
 * ------------------------------------------------------------------------- */
ANQS_API int anqs_launch_count(uint64_t* n);
ANQS_API int anqs_profile_enable(int on);
ANQS_API int anqs_profile_read(int id, const char** name, uint64_t* launches, double* total_ms);

#ifdef __cplusplus
}
#endif
#endif /* ANQS_H */
