/*
 * crv.h - C ABI of the GB300 spherical curvelet transform library (libcrv.so).
 *
 * Second-generation curvelets on the sphere (Chan, Leistedt, Kitching, McEwen,
 * arXiv:1511.05578). The library computes, on one GPU:
 *   - the spin spherical harmonic transform on the MW equiangular grid
 *     (f_lm = <f, sY_lm>, Sec. II-A, Eq. spin_sphericalHarmonics);
 *   - curvelet analysis: the directional convolution of Eq. (wav_analysis) in its
 *     harmonic form Eq. (wav_analysis_harmonic), evaluated as an inverse Wigner
 *     transform of the coefficients of Eq. (wav_harmonic_coeff) onto the SO(3)
 *     grid of Eqs. (nodes_alpha, nodes_beta, nodes_gamma), plus the scaling
 *     coefficients of Eq. (analysis_scaling_harmonic);
 *   - curvelet synthesis, Eq. (wav_synthesis_harmonic), through the forward Wigner
 *     quadrature of Sec. III-A-2 (Eqs. Fmn, TildaFmn, Fmnmp, gmnmp, flml),
 *     exact for band-limited signals by the admissibility of Eq. (admissibility).
 *
 * Conventions (all entry points):
 *   - Band limit L: f_lm = 0 for l >= L. Spin s, |s| < L; f_lm = 0 for l < |s|.
 *   - Harmonic coefficients f_lm: complex double (interleaved re, im), index
 *     l*l + l + m, length L*L per map.
 *   - Maps on the MW grid: [L][2L-1], theta_t = pi(2t+1)/(2L-1),
 *     phi_p = 2 pi p/(2L-1). Real doubles with CRV_F_REAL, otherwise complex double.
 *   - Scales j = J0..J, J the smallest integer with lambda^J >= L. Scale j has band
 *     limit L_j = min(L, ceil(lambda^(j+1))) (Sec. III-A-3) and coefficients
 *     W_j[b][a][g] on alpha_a = 2 pi a/(2L_j-1), beta_b = pi(2b+1)/(2L_j-1),
 *     gamma_g = 2 pi g/(2L_j-1): L_j * (2L_j-1) * (2L_j-1) samples per map. Real with
 *     CRV_F_REAL, else complex; double, or float with CRV_F_W_FP32.
 *   - Scaling coefficients W^Phi: spin-0 map on the MW grid of band limit
 *     L_phi = ceil(lambda^J0), [L_phi][2L_phi-1], real with CRV_F_REAL else complex,
 *     always double.
 *   - Batches: B maps stored back to back ([B][...]), B <= max_batch of the plan.
 *
 * Memory and streams: every data pointer is caller-owned DEVICE memory (cudaMalloc,
 * or a torch tensor's data_ptr) that must stay valid until the call's work on the
 * stream has finished. The plan owns its tables and workspace (allocated by
 * crv_plan_create, freed by crv_plan_destroy). Calls are asynchronous on the given
 * CUDA stream (NULL = legacy default stream); only crv_plan_create and
 * crv_plan_destroy synchronise. A plan may be used by one stream at a time. No C++
 * exception crosses this boundary; every call returns a crv_status code and records
 * a message for crv_last_error().
 */
#ifndef CRV_H
#define CRV_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct crv_plan_s* crv_plan_t;

typedef enum crv_status {
  CRV_OK = 0,
  CRV_EINVAL = 1,        /* invalid argument (sizes, lambda, spin, batch, null pointer) */
  CRV_ENOMEM = 2,        /* device allocation of tables or workspace failed */
  CRV_ECUDA = 3,         /* a CUDA runtime call or kernel launch failed */
  CRV_ETIMEOUT = 4,      /* a bounded device-side wait gave up */
  CRV_EUNSUPPORTED = 5,  /* valid but not supported by this build (e.g. no GPU) */
  CRV_EGUARD = 6         /* a write went past the end of a plan buffer (CRV_F_GUARD plans) */
} crv_status;

/* Azimuthal band-limit rule. The curvelet rule is the only one: N_j = L_j and the
 * directional component is supported on |m| = l before rotation (Sec. II-B). */
enum { CRV_NRULE_CURVELET = 0 };

/* Plan flags. */
enum {
  CRV_F_REAL = 1,   /* spin-0 real signal: real maps and real W (conjugate symmetry, Sec. III-A-3) */
  CRV_F_MIXED = 2,  /* split-FP32 contraction on tensor cores and FP32 FFTs; Delta recursion
                       and the synthesis accumulation of f_lm stay FP64 */
  CRV_F_W_FP32 = 4, /* store W_j as float instead of double */
  CRV_F_TUNE = 16,   /* autotune at creation: time a batch of zero maps for each number of
                       concurrent map workers (1, 2, 4, 8 up to max_batch) and ring-chunk size
                       (64 MB, 256 MB) and keep the fastest (crv_plan_tuning reports it) */
  CRV_F_FP64_TC = 32, /* plain FP64 plans only: the two Delta contractions (Eqs. inverse_Fmnmp and
                         flml) run on the TF32 tensor cores with FP64 accuracy, by error-free
                         splitting: each operand row is scaled by a power of two and cut into
                         seven integer slices of 7 bits (6 bits when a K range exceeds 1024:
                         complex signals above L = 512), slice products of one level accumulate
                         exactly in FP32, and the levels are added in FP64. Sliced Delta Psi tables per scale are built at creation
                         (about 7x the size of the FP32 ones); the per-map A operands are sliced
                         into a 4 GB buffer in passes over m' (CRV_FP64_TC_A_GB sets its size) */
  CRV_F_GUARD = 64,  /* debugging aid in place of a memory checker: every device buffer of the plan
                        (tables and workspace, workers included) is followed by a 4 KB guard
                        region of a known byte pattern, which crv_plan_check_guards compares;
                        costs one synchronisation per allocation at creation, nothing per call */
  CRV_F_UNROTATED = 8 /* W_j are the coefficients of the unrotated curvelets s-psi~^(j) (Sec. III-A-1),
                         i.e. W~(rho) with W(rho) = W~(rho rho*), rho* = (0, vartheta^j, 0) (Eq.
                         rotateWigner). Their Wigner coefficients vanish unless |n| = l (Eq.
                         curvelet_Wigner_property), so Eq. inverse_Fmnmp keeps the one term l = |n|
                         and the Delta contraction costs O(L^3) instead of O(L^4) per scale (the
                         paper's own fast algorithm); the synthesis keeps n = +-l of Eq. flml.
                         Same grids, sizes and layouts as the rotated W_j. */
};

/* Create a plan.
 *   L         band limit, 2 <= L <= 4096
 *   lambda    dilation parameter, lambda > 1 (Sec. II-B)
 *   J0        lowest curvelet scale, J0 >= 0, J0 <= J; lambda^J0 >= |spin| so that
 *             vartheta^j = arccos(-s/lambda^j) of Eq. (theta_peakj) exists
 *   spin      s; CRV_F_REAL requires s = 0
 *   nrule     CRV_NRULE_CURVELET
 *   flags     CRV_F_* bits
 *   max_batch largest B accepted by the transform calls. When max_batch > 1 and one map's
 *             workspace is small (<= 1 GB, L <= 256: the band limits whose kernels cannot fill
 *             the GPU one map at a time), the plan also holds up to 3 (CRV_F_TUNE: 7) worker instances
 *             sharing its tables, each with a workspace and a stream of its own: the B maps of
 *             a call run on up to 4 workers at once (map b on worker b mod K), forked from the
 *             call's stream and joined back into it by events, so calls stay stream-ordered.
 *             Above 1 GB the plan holds one worker (two maps at once) when the two workspaces
 *             fit in a quarter of the device memory. The environment variable
 *             CRV_WORKER_MAX_GB replaces both rules by one workspace limit for up to 4 workers
 *   stream    CUDA stream used for the table build (Delta recursion)
 * Builds the radial kernels kappa^(j) and scaling function (Sec. II-B), the rotated
 * directional components zeta^(j) (Eq. after directionality_normalisation; with
 * CRV_F_UNROTATED the unrotated zeta~ with zeta~_{l,l} = 1/sqrt2, zeta~_{l,-l} = (-1)^l/sqrt2), the
 * Delta^l = d^l(pi/2) tables (FP64, on the device), FFT tables and workspace.
 * Synchronises the stream. On error *out is NULL. */
int crv_plan_create(crv_plan_t* out, int L, double lambda, int J0, int spin, int nrule,
                    unsigned flags, int max_batch, void* stream);

/* Free a plan and its device memory (synchronises the device first). NULL is ok. The
 * read-only tables a plan shares with its clones are freed with the last of them. */
int crv_plan_destroy(crv_plan_t plan);

/* A second instance of a plan for concurrent use on another stream (a plan serves one stream
 * at a time). The clone shares the source's read-only tables (Delta^l(pi/2), the tensor-core
 * Delta Psi tables, FFT tables, kernels) by reference count and allocates only its own
 * workspace (f_lm buffers, the (m, n, m') volumes, ring buffer, per-map tensor-core A tables,
 * error flag), so concurrent requests of the same (L, lambda, J0, spin, flags) hold the tables
 * once. The two plans are independent otherwise: either may be destroyed first. Synchronises
 * the stream. CRV_ENOMEM if the workspace does not fit; on error *out is NULL. */
int crv_plan_clone(crv_plan_t* out, crv_plan_t src, void* stream);

/* Device bytes of a plan: table_bytes of its (shared) read-only tables, workspace_bytes of its
 * own workspace (its workers' included). Either pointer may be NULL. A clone adds
 * workspace_bytes to the device. */
int crv_plan_bytes(crv_plan_t plan, size_t* table_bytes, size_t* workspace_bytes);

/* Launch settings of a plan: the number of map workers a call uses, the ring-chunk size of the
 * SO(3) ring transforms, and whether the autotuner (CRV_F_TUNE) chose them. Any pointer may be
 * NULL. */
int crv_plan_tuning(crv_plan_t plan, int* workers, size_t* ring_bytes, int* tuned);

/* Sizes of a plan. Any output pointer may be NULL.
 *   J                 largest scale
 *   Lj[j], j=0..J     band limit of scale j (entries j < J0 are 0)
 *   w_elems[j]        samples per map of W_j (L_j (2L_j-1)^2; 0 for j < J0)
 *   L_phi             band limit of the scaling map
 *   workspace_bytes   device memory the plan uses (its shared tables + its own workspace)
 * Lj and w_elems must have room for J+1 entries (J <= 64). */
int crv_plan_info(crv_plan_t plan, int* J, int* Lj, size_t* w_elems, int* L_phi,
                  size_t* workspace_bytes);

/* Wait for the device and report whether any bounded device-side wait of this plan's
 * kernels gave up since the last check (CRV_ETIMEOUT; the affected results are
 * invalid). Clears the condition. */
int crv_plan_check(crv_plan_t plan);

/* As crv_plan_check, but ordered on one stream instead of the whole device: waits for the
 * work already queued on `stream` (the stream the plan's calls ran on), then reads and clears
 * the plan's error flag. Work of other streams and plans is not waited for, so a caller that
 * runs several plans concurrently (one stream each) can collect one without stalling the
 * others. CRV_ETIMEOUT as crv_plan_check; CRV_ECUDA if the stream reports an error. */
int crv_plan_check_stream(crv_plan_t plan, void* stream);

/* Self-test of that error path: launch, on the stream, one thread that waits on a device
 * barrier nothing arrives at, giving up after `polls` polls (1 <= polls <= 1e6) as every
 * bounded wait of the library does; the next crv_plan_check then returns CRV_ETIMEOUT.
 * Makes no other device work, leaves nothing in flight; CRV_EINVAL for a bad argument. */
int crv_debug_bounded_wait(crv_plan_t plan, long polls, void* stream);

/* Guard regions (plans created with CRV_F_GUARD; no counterpart in the paper: a check of this
 * library's own kernels). crv_plan_check_guards waits for the device and compares every guard
 * region of the plan (shared tables, workspace, workers' workspaces) with its fill pattern:
 * CRV_OK if all are intact, CRV_EGUARD if any byte past the end of a buffer was written (*nbad,
 * if not NULL, gets the number of changed regions; crv_last_error names the first), CRV_EINVAL
 * for a plan without guards. crv_plan_guard_count gives the number of regions (0 without
 * guards). crv_debug_poke_guard changes one byte inside region `which` from the host, inside
 * the allocation, to test the check itself. */
int crv_plan_check_guards(crv_plan_t plan, int* nbad);
int crv_plan_guard_count(crv_plan_t plan, int* n);
int crv_debug_poke_guard(crv_plan_t plan, int which);

/* Host check of the K runs of the tensor-core contractions (no counterpart in the paper; runs
 * on the host only, no device work). For one scale of band limit Lb (1 <= Lb <= 1024) and the
 * column set of a real spin-0 signal (real != 0) or a complex spin-`spin` one, rotated or
 * unrotated (unrot != 0), it builds the runs as a plan does: analysis B runs and synthesis
 * l-tiles from l = lmin_b, analysis A runs from l = lmin_a (a plan passes the first l of the
 * scale's kernel support as both; 0 <= lmin <= Lb). It counts the tiles that break the
 * engines' rules: an analysis tile whose K chunks leave its B or A run, or miss an l >= lmin_b
 * that its products need; a synthesis tile whose output the reduction over m' reads, with no
 * K chunks or with chunks missing an n it needs. *bad gets that count (0: consistent), *tiles
 * (if not NULL) the number of tiles checked. CRV_EINVAL for a bad argument. */
int crv_debug_check_tc_ranges(int Lb, int lmin_b, int lmin_a, int real, int spin, int unrot, long long* tiles,
                              long long* bad);

/* Host copy of plan tables, for inspection and tests.
 *   crv_plan_kernel:  psi[l][n + L_j - 1] = sPsi^(j)_ln (real, Eq. wav_factorized), l < L_j
 *   crv_plan_scaling: phi[l] = sqrt(4pi/(2l+1)) Phi_l0 = sqrt(k_lambda(l/lambda^J0)), l < L
 *   crv_plan_delta:   out[m'][n] = Delta^l_{m'n} for 0 <= m', n <= l (quarter table read
 *                     back from the device; the other quadrants follow by symmetry) */
int crv_plan_kernel(crv_plan_t plan, int j, double* psi_host);
int crv_plan_scaling(crv_plan_t plan, double* phi_host);
int crv_plan_delta(crv_plan_t plan, int l, double* out_host);

/* Forward spin SHT: map [B][L][2L-1] -> f_lm [B][L*L] (complex double). Exact for
 * band-limited maps (MW sampling theorem; same quadrature steps as Sec. III-A-2 with
 * n = -s). */
int crv_sht_fwd(crv_plan_t plan, const void* map, void* flm, int B, void* stream);

/* Inverse spin SHT: f_lm [B][L*L] -> map [B][L][2L-1] (Eq. spin_sphericalHarmonics
 * summed over l, m). With CRV_F_REAL the imaginary part is dropped. */
int crv_sht_inv(crv_plan_t plan, const void* flm, void* map, int B, void* stream);

/* Curvelet analysis from a map: forward SHT, then for each scale the inverse Wigner
 * transform of (8pi^2/(2l+1)) f_lm Psi^(j)*_ln onto the SO(3) grid (Eqs.
 * wav_harmonic_coeff, inverse_Fmnmp in general-n form, inverse_feul), and the scaling
 * map (Eq. analysis_scaling_harmonic).
 *   W     array of J+1 device pointers; W[j] for J0 <= j <= J receives [B][W_j] (see
 *         conventions); entries j < J0 are ignored and may be NULL
 *   Wphi  [B][L_phi][2L_phi-1]; may be NULL to skip the scaling map */
int crv_analysis(crv_plan_t plan, const void* map, void* const* W, void* Wphi, int B, void* stream);

/* Curvelet synthesis to a map: per scale the forward Wigner transform of W_j and the
 * sum over n with Psi^(j)_ln, plus the scaling term (Eq. wav_synthesis_harmonic), then
 * the inverse SHT. W[j] for J0 <= j <= J must be valid; Wphi may be NULL (treated as
 * zero). */
int crv_synthesis(crv_plan_t plan, const void* const* W, const void* Wphi, void* map, int B,
                  void* stream);

/* Harmonic-space forms: as crv_analysis / crv_synthesis but starting from / ending at
 * f_lm [B][L*L] (no SHT). For CRV_F_REAL plans f_lm must satisfy
 * f_{l,-m} = (-1)^m conj(f_lm); the synthesis output does. */
int crv_analysis_lm(crv_plan_t plan, const void* flm, void* const* W, void* Wphi, int B, void* stream);
int crv_synthesis_lm(crv_plan_t plan, const void* const* W, const void* Wphi, void* flm, int B,
                     void* stream);

/* Rotation of Wigner coefficients of scale j (Sec. III-A-1, Eqs. curvelet_Wigner,
 * curvelet_Wigner_inverse, rotateWigner): from the Wigner coefficients of the unrotated
 * curvelet coefficients W~_j (the paper's fast representation) to those of the rotated W_j.
 * With rho* = (0, vartheta^j, 0), vartheta^j = arccos(-s/lambda^j), W(rho) = W~(rho rho*)
 * gives (W)^l_mk = sum_n (W~)^l_mn d^l_kn(vartheta^j); (W~)^l_mn vanishes unless |n| = l
 * (Eq. curvelet_Wigner_property), so
 *     (W)^l_mk = (W~)^l_{m,l} d^l_{k,l}(vartheta^j) + (W~)^l_{m,-l} d^l_{k,-l}(vartheta^j),
 * O(L_j^3) per scale. Coefficients are those of W(rho) = sum (2l+1)/(8pi^2) (W)^l_mn D^l*_mn(rho)
 * with D^l_mn(a, b, g) = e^{-ima} d^l_mn(b) e^{-ing}; e.g. (W~)^l_mn = (8pi^2/(2l+1)) f_lm Psi~_ln.
 *   j   scale, J0 <= j <= J (any plan: vartheta^j depends only on lambda, j and the spin)
 *   wt  [B][2][L_j][2L_j-1] complex double: wt[b][0][l][m + L_j - 1] = (W~)^l_{m,l},
 *       wt[b][1][l][m + L_j - 1] = (W~)^l_{m,-l} (entries |m| > l and wt[b][1][0] are ignored)
 *   w   [B][L_j][2L_j-1][2L_j-1] complex double: w[b][l][m + L_j - 1][k + L_j - 1] = (W)^l_mk,
 *       zero where |m| > l or |k| > l
 * Device pointers, stream-ordered; CRV_EINVAL for j outside [J0, J], B outside [0, max_batch]
 * or a NULL pointer with B > 0. FP64. */
int crv_rotate_wigner(crv_plan_t plan, int j, const void* wt, void* w, int B, void* stream);

/* Adjoint of crv_rotate_wigner: (W~)^l_{m,+-l} = sum_k (W)^l_mk d^l_{k,+-l}(vartheta^j), which
 * inverts it on rotated coefficients (d^l is orthogonal); writes every entry of wt (zeros for
 * |m| > l and for wt[b][1][0]). Same layouts and errors as crv_rotate_wigner. */
int crv_rotate_wigner_adjoint(crv_plan_t plan, int j, const void* w, void* wt, int B, void* stream);

/* Message of the last failing call on this thread ("" if none). */
const char* crv_last_error(void);

/* Human-readable name of a status code. */
const char* crv_status_string(int status);

/* Number of kernel launches this library has issued since load (all plans, all
 * threads). Used to count device work inside timed regions. */
unsigned long long crv_launch_count(void);

/* Allocation-free build of the Delta^l = d^l(pi/2) quarter table. The paper has no
 * counterpart: this entry point exists for callers that must not allocate device
 * memory themselves, such as code that runs inside a host framework owning a fixed
 * device arena, code issued while a stream is being captured into a CUDA graph, or
 * latency-critical paths where the implicit synchronisation of cudaMalloc/cudaFree
 * is not acceptable. It calls no cudaMalloc, cudaFree or allocating library routine.
 *   L       1 <= L <= CRV_NOALLOC_MAX_L
 *   Q       caller-owned device buffer of L*L*L doubles; on return (stream order) it holds
 *           Q[m'][l][n] = Delta^l_{m'n} for 0 <= m', n <= l < L and 0 elsewhere, the same
 *           values crv_plan_delta reads back from a plan of band limit >= L
 *   stream  CUDA stream (NULL = legacy default stream)
 * Scratch: the recursion's per-l seed rows live in a library-wide device array sized for
 * CRV_NOALLOC_MAX_L (3 MB); every GPU that loads libcrv holds it until the process exits.
 * The first call on a device looks up that array's device address with the device
 * current; make that first call before any stream capture. All calls share the array,
 * so calls that overlap on the GPU (different streams, or devices sharing a context)
 * race; serialise them. Errors: CRV_EINVAL for L outside the range or Q == NULL,
 * CRV_ECUDA for a failed address lookup or launch (message in crv_last_error()). */
#define CRV_NOALLOC_MAX_L 512
int crv_delta_table_noalloc(int L, double* Q, void* stream);

/* Optional per-kernel timing for measurement tools. When bit k of kind_mask is set,
 * every launch of kernel kind k is bracketed by CUDA events recorded on the stream it
 * is launched on; crv_profile_read waits for the recorded events and returns the
 * launch count and summed device time (ms) of kind k since the last reset. Kinds are
 * numbered 0 .. crv_profile_num_kinds()-1 and named by crv_profile_kind_name.
 * Off by default; enabling it adds two event records per timed launch. */
int crv_profile_enable(unsigned kind_mask);
int crv_profile_num_kinds(void);
const char* crv_profile_kind_name(int k);
int crv_profile_read(int k, unsigned long long* launches, double* total_ms);
int crv_profile_reset(void);

#ifdef __cplusplus
}
#endif

#endif /* CRV_H */
