/*
 * fpeps.h - C ABI of the GB300 boundary-MPS row-absorption library.
 *
 * What it computes (Scheb, "Improved contraction of finite projected entangled
 * pair states", arXiv:2511.01039):
 *   Sec. II   <psi|O|psi> of an open Lx x Ly PEPS (bond D, physical dim p) with a
 *             PEPO O (bond w), contracted row by row into a boundary MPS whose
 *             bundles of D*w*D legs are compressed to a bond chi.
 *   Sec. III  every compression step is built from the contraction pattern of
 *             Fig. 2(a): environment, boundary, and the sandwich C of a PEPS, a
 *             PEPO and the adjoint PEPS tensor (PEPO indices kept separate).
 *   Sec. IV   the compression uses a randomized SVD (Gaussian sketch, repeated
 *             application of the matrix and its transpose, thin QR, SVD of the
 *             projected matrix), first in a left-to-right zip-up pass and then in
 *             a right-to-left variational fit with controlled bond expansion
 *             (CBE, Fig. 3-5).
 *
 * Conventions
 *   PEPS site  A[l,u,r,d,p]       PEPO site W[l,u,r,d,p,p']  (p meets the ket,
 *   p' the bra); open-boundary legs have dimension 1; the bra is A itself (real
 *   data). Sites are packed in row-major site order (r = 0..Lx-1 top to bottom,
 *   c = 0..Ly-1 left to right), each site C-contiguous.
 *   Boundary MPS tensors T_c[t_{c-1}, (u,u_w,u'), t_c], bundle index bra-fastest.
 *
 * Threading and streams: an env is not thread-safe; different envs are
 * independent. All GPU work is enqueued on the stream given at creation.
 * Calls that return scalars to host memory synchronise that stream; the
 * others only enqueue work (they may synchronise to read tiny status words).
 *
 * Errors: every call returns an fpeps_status; nothing throws, aborts or traps.
 * After FPEPS_ERR_CUDA the env is poisoned: every later call except
 * fpeps_last_error and fpeps_env_destroy returns FPEPS_ERR_STATE.
 */
#ifndef FPEPS_H
#define FPEPS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FPEPS_OK = 0,
  FPEPS_ERR_ARG = 1,         /* bad argument (NULL, size, dimension, enum) */
  FPEPS_ERR_STATE = 2,       /* call out of order, or env poisoned */
  FPEPS_ERR_OOM = 3,         /* allocator returned NULL */
  FPEPS_ERR_CUDA = 4,        /* a CUDA call failed; env poisoned */
  FPEPS_ERR_NUMERIC = 5,     /* non-finite value or failed factorisation */
  FPEPS_ERR_TIMEOUT = 6,     /* a bounded device wait gave up */
  FPEPS_ERR_UNSUPPORTED = 7  /* valid request this build does not implement */
} fpeps_status;

/* Arithmetic of the contraction GEMMs (the QR and the small SVD always run in
 * FP64-class precision). FP64: everything in double. F32: plain FP32 CUDA-core
 * products. TF32X3 / BF16X3: split-precision products on the tensor cores,
 * a_hi*b_hi + a_hi*b_lo + a_lo*b_hi with FP32 accumulation, the operands split
 * into TF32 (3 x 2^-22 relative error per product) or BF16 (3 x 2^-16) halves.
 * In BF16X3 every tensor-core GEMM (boundary and environment products, the
 * QR's tall products, the CBE projectors) takes the BF16 split; the site
 * sandwich stays 3xTF32, and the calibration columns and unbiased products
 * run on the FP32 CUDA cores as in TF32X3. */
typedef enum { FPEPS_F64 = 0, FPEPS_F32 = 1, FPEPS_TF32X3 = 2, FPEPS_BF16X3 = 3 } fpeps_precision;

/* Device-memory provider. alloc(ctx, bytes, stream) returns device memory usable
 * on `stream` (NULL on failure); free(ctx, ptr, stream) releases it. Pass NULL
 * for the allocator to use cudaMallocAsync/cudaFreeAsync on the env stream. */
typedef struct {
  void* ctx;
  void* (*alloc)(void* ctx, size_t bytes, void* stream);
  void (*free)(void* ctx, void* ptr, void* stream);
} fpeps_allocator;

typedef struct {
  int32_t Lx, Ly;        /* lattice, >= 1 */
  int32_t D;             /* PEPS bond dimension (interior legs), >= 1 */
  int32_t p;             /* physical dimension, >= 1 */
  int32_t w;             /* PEPO bond dimension (interior legs), >= 1 */
  int32_t chi;           /* boundary bond dimension, >= 1 */
  fpeps_precision prec;  /* contraction arithmetic */
  uint64_t seed;         /* key of the Gaussian sketches */
  int32_t symmetry;      /* 0 = dense, 1 = U(1) x U(1) charge sectors */
  int32_t n_envs;        /* independent environments in the handle, 1 .. FPEPS_MAX_ENVS
                            (see fpeps_env_select) */
} fpeps_config;

#define FPEPS_MAX_ENVS 1024
#define FPEPS_MAX_FIT_PASSES 8

/* rSVD / CBE settings (Sec. IV). Zero-initialised fields take the defaults in
 * brackets where stated. */
typedef struct {
  int32_t oversample;   /* sketch width = kept bond + oversample            */
  int32_t power_iters;  /* q: applications of A^T A after the first A       */
  int32_t chi_tilde;    /* CBE expansion width; 0 => ceil(chi / 10)         */
  int32_t n_fit;        /* CBE fit passes after the zip-up: 0 .. FPEPS_MAX_FIT_PASSES
                           (more than 1: dense mode only, symmetry = 0)      */
  int32_t exact_svd;    /* 1 => sketch width = full rank (exact factorisation) */
} fpeps_rsvd_params;

typedef struct {
  double seconds;        /* device time of the call (CUDA events)         */
  double alg_flops;      /* algorithmic flops of the contractions          */
  double log_scale;      /* ln of the scale moved out of the new boundary  */
  double trunc_err_est;  /* sum of squared discarded Ritz values / total (zip-up) */
} fpeps_stats;

typedef struct fpeps_env fpeps_env;

/* Create an environment for one PEPS and one operator PEPO.
 *   cfg        lattice and method configuration (copied).
 *   peps_dev   device buffer with all PEPS sites (row-major site order, each
 *              [Dl,Du,Dr,Dd,p] C-contiguous, edge legs 1), element type dtype_in.
 *   pepo_dev   device buffer with all operator PEPO sites [wl,wu,wr,wd,p,p'],
 *              or NULL for none (then only fpeps_contract_norm is available).
 *   charges_host  NULL when cfg->symmetry == 0; else host int32 charges
 *              (N_up, N_dn) of every leg index (Sec. V: U(1) x U(1) symmetric
 *              tensors): for each PEPS site in row-major order its legs
 *              l, u, r, d, each as dim pairs; then, if pepo_dev is given, the
 *              same for every PEPO site (dims w or 1 at the edges). The caller
 *              guarantees the tensors conserve them: PEPS q_l+q_u+q_p =
 *              q_r+q_d+f_site, PEPO q_l+q_u+q_p = q_r+q_d+q_p'. The buffer is read
 *              during the call. With symmetry 1 every factorisation of the
 *              compression (zip-up rSVD, CBE rSVD, SVD of the fitted tensor) runs
 *              sector by sector in the charge of the bond it cuts, with one global
 *              truncation; a boundary imported by fpeps_import_boundary carries
 *              the charges of its checkpoint's charge section (without one,
 *              compression returns FPEPS_ERR_STATE).
 *   dtype_in   0 = float64, 1 = float32.
 *   cuda_stream   cudaStream_t on which all work is enqueued (NULL = default).
 *   alloc      device allocator or NULL.
 * The inputs are copied (and converted to the compute precision) before the
 * call returns; the caller keeps ownership of its buffers.
 * Errors: FPEPS_ERR_ARG (bad sizes/pointers), FPEPS_ERR_OOM, FPEPS_ERR_CUDA,
 * FPEPS_ERR_ARG also when n_envs is outside 1 .. FPEPS_MAX_ENVS, when symmetry is not 0 or 1, or
 * when charges_host does not match it. */
fpeps_status fpeps_env_create(const fpeps_config* cfg, const void* peps_dev, const void* pepo_dev,
                              const int32_t* charges_host, int32_t dtype_in, void* cuda_stream,
                              const fpeps_allocator* alloc, fpeps_env** out);

/* Absorb row `row` (rows must come in order 0, 1, ..., Lx-1; row 0 starts a new
 * sweep of the given layer). layer 0 = identity PEPO (norm), 1 = operator PEPO.
 *   row 0        builds the exact boundary from the row-0 sandwiches (Sec. II).
 *   0<row<Lx-1   stages the row; fpeps_compress_rsvd must follow.
 *   row Lx-1     closes the network exactly (vector transfer); the sweep value
 *                becomes available to fpeps_sweep_value.
 * Errors: FPEPS_ERR_STATE (out of order / compress pending), FPEPS_ERR_ARG. */
fpeps_status fpeps_absorb_row(fpeps_env* env, int32_t row, int32_t layer);

/* Compress the staged row into a new boundary of bond chi: zip-up rSVD pass,
 * then n_fit CBE fit passes (Sec. IV, Fig. 3: the variational right-to-left fit
 * with controlled bond expansion). Every pass after the first starts from the
 * previous one re-canonicalised left to right (thin QR per site, the factor
 * carried right, left environments rebuilt by pattern 2(a)); pass p draws its
 * CBE sketch at generator stage 1 + 16 (p - 1). out_host (nullable) receives
 * stats. Errors: FPEPS_ERR_STATE if no interior row is staged,
 * FPEPS_ERR_NUMERIC if a factorisation broke down or a value became
 * non-finite, FPEPS_ERR_UNSUPPORTED for n_fit outside 0 .. FPEPS_MAX_FIT_PASSES
 * or n_fit > 1 with charge sectors. */
fpeps_status fpeps_compress_rsvd(fpeps_env* env, const fpeps_rsvd_params* params, fpeps_stats* out_host);

/* Value of the network closed by the last absorbed row (Sec. II: the energy
 * functional <psi|O|psi>, or <psi|psi> for layer 0, as the sandwich of PEPS,
 * PEPO and adjoint PEPS contracted through the boundary MPS).
 *   log_abs, sign  host pointers; value = sign * exp(log_abs) (the log form keeps
 *                  lattices whose value under- or overflows a double).
 * Errors: FPEPS_ERR_ARG (NULL pointers), FPEPS_ERR_STATE (no sweep has been
 * closed since the last row 0). Reads host state only; no GPU work. */
fpeps_status fpeps_sweep_value(fpeps_env* env, double* log_abs, int32_t* sign);

/* <psi|psi> of the PEPS (Sec. II: the norm network, PEPS and adjoint PEPS with
 * the identity in place of the PEPO, w = 1), by one top-to-bottom boundary sweep
 * of layer 0: row 0 exactly, every interior row compressed by fpeps_compress_rsvd
 * with `params` (Sec. IV), the last row closed exactly.
 *   params         rSVD / CBE settings (read during the call).
 *   log_abs, sign  host pointers: <psi|psi> = sign * exp(log_abs).
 * Any row state of the env is replaced (a new sweep starts at row 0). Synchronises
 * the env stream. Errors: FPEPS_ERR_ARG (NULL pointers), FPEPS_ERR_NUMERIC
 * (non-finite input or a factorisation breakdown), FPEPS_ERR_OOM, FPEPS_ERR_CUDA,
 * FPEPS_ERR_TIMEOUT (a bounded device wait gave up). */
fpeps_status fpeps_contract_norm(fpeps_env* env, const fpeps_rsvd_params* params, double* log_abs,
                                 int32_t* sign);

/* Expectation value <O> = <psi|O|psi> / <psi|psi> (Sec. II: the energy
 * functional E = <psi|H|psi> of Fig. 1, normalised by the norm network): one
 * boundary sweep with the operator PEPO (layer 1) and one with the identity
 * (layer 0), each as in fpeps_contract_norm, with the same sketch seed.
 *   params       rSVD / CBE settings (read during the call).
 *   value        host pointer: <O>.
 *   log_abs_num, sign_num  host pointers: <psi|O|psi> = sign_num * exp(log_abs_num).
 * Synchronises the env stream. Errors: FPEPS_ERR_STATE if the env has no operator
 * PEPO; otherwise as fpeps_contract_norm. */
fpeps_status fpeps_expect(fpeps_env* env, const fpeps_rsvd_params* params, double* value,
                          double* log_abs_num, int32_t* sign_num);

/* Checkpoint of the current boundary (after row 0 or a compressed row). The
 * paper has no counterpart: this is the library's restart format (the boundary
 * MPS of Sec. II after the rows absorbed so far, with its accumulated scale).
 * Layout: int64 header {magic, Ly, next_row, layer, elem_bytes, bond[Ly+1],
 * phys[Ly]}, double log_scale, then the tensors T_c in compute precision; in
 * the charge-sector mode (symmetry = 1) a charge section follows: int64 magic
 * 0x3151425350455046 ("FPEPSBQ1"), then for every bond c = 0..Ly its bond[c]
 * U(1) x U(1) charge pairs as int32, zero-padded to a multiple of 8 bytes.
 *   host_buf  host memory of *bytes bytes, or NULL: then *bytes receives the
 *             required size and nothing is copied.
 * A staged row that has not been compressed yet is not part of the checkpoint.
 * Synchronises the env stream. Errors: FPEPS_ERR_ARG (NULL bytes, or a buffer
 * smaller than the checkpoint), FPEPS_ERR_STATE (no boundary yet, or the sweep
 * has been closed by its last row), FPEPS_ERR_CUDA. */
fpeps_status fpeps_export_boundary(fpeps_env* env, void* host_buf, size_t* bytes);

/* Load a boundary (same layout as fpeps_export_boundary, from any source with
 * the right shapes) and make `next_row` the next row to absorb in `layer`. The
 * paper has no counterpart: this restarts a sweep from a stored boundary MPS
 * (Sec. II). A charge section, if present, gives the bond charges (only an env
 * with symmetry = 1 accepts one). Errors: FPEPS_ERR_ARG (bad magic, element
 * size, lattice width, end bonds or byte count; unknown or truncated data after
 * the tensors; charges for an env without charge sectors; next_row outside
 * 1..Lx-1), FPEPS_ERR_STATE (layer 1 without
 * an operator PEPO), FPEPS_ERR_OOM, FPEPS_ERR_CUDA. Bundles that do not match the
 * up legs of row `next_row` are reported by the next fpeps_compress_rsvd or
 * closing fpeps_absorb_row (FPEPS_ERR_ARG).
 * `host_buf` may point to host memory (copied host -> device, the call
 * synchronises) or to device memory (copied device -> device on the env
 * stream, only the header is read back). The buffer must stay valid until the
 * copies have executed. */
fpeps_status fpeps_import_boundary(fpeps_env* env, const void* host_buf, size_t bytes, int32_t next_row,
                                   int32_t layer);

/* Task table of a block-sparse site map applied to the vectors of one charge
 * sector q, the ops of fpeps_apply_theta_op: Y = Theta_c X (op 0), its
 * transpose (op 1), the right-environment map of the CBE fit (op 2) and its
 * transpose (op 3) (Sec. III: contractions cut into quantum-number slices
 * whose outputs do not overlap; Sec. IV: the application of the zip-up, pattern
 * 2(a)). Host code, no device work. With charge-conserving tensors each of the
 * three contractions (1: boundary x vectors, 2: the site sandwich, 3:
 * environment x vectors) splits into charge blocks; a task computes one output
 * block, summing the block products that feed it. Charge rules, pairs
 * (N_up, N_dn): T[t, U, t'] q_t = Q_U + q_t'; sandwich Q_L + Q_U = Q_R + Q_Dn;
 * left environment EL[a, t, L] q_a = q_t + Q_L; X[t', R] in sector q where
 * q_t' + Q_R = q, Y[a, Dn] where q_a - Q_Dn = q. Op 1 runs the mirror steps
 * (1: environment^T x vectors, 2: the sandwich transposed, 3: boundary^T x
 * vectors). For ops 2 and 3 the leg a is the right environment's bond,
 * ER[a, t', R] with q_a = q_t' + Q_R, vectors X[Dn, a] with Q_Dn + q_a = q and
 * Z[t, L] with q_t + Q_L = q.
 *   qa, qt, qu, qtp, ql, qr, qd  host int32 charge pairs of the legs a, t, U,
 *              t', L, R, Dn (n entries each, pairs interleaved); q the sector.
 *   tasks      host int32 [cap][8]: step (1..3), number of block products,
 *              then the output block's charges: op 0 step 1 (t, U, R), step 2
 *              (t, L, Dn), step 3 (a, Dn) and one zero pair; op 1 step 1
 *              (t, L, Dn), step 2 (t, U, R), step 3 (t', R); op 2 step 1
 *              (t', R, Dn), step 2 (t', L, U), step 3 (t, L); op 3 step 1
 *              (t', L, U), step 2 (t', R, Dn), step 3 (Dn, a);
 *              steps in order, within a step the legs' charges in order of
 *              first appearance.
 *   flops      host double [cap]: 2 x multiply-adds of the task per vector.
 *   n_inout    in: cap; out: number of tasks. With cap 0 (tasks, flops may be
 *              NULL) only the count is returned.
 * Errors: FPEPS_ERR_ARG (op outside 0..3, NULL pointer, empty leg, cap too
 * small). */
fpeps_status fpeps_theta_block_tasks(int32_t op, const int32_t* qa, int32_t na, const int32_t* qt, int32_t nt,
                                     const int32_t* qu, int32_t nu, const int32_t* qtp, int32_t ntp,
                                     const int32_t* ql, int32_t nl, const int32_t* qr, int32_t nr,
                                     const int32_t* qd, int32_t nd, const int32_t* q, int32_t* tasks,
                                     double* flops, int32_t* n_inout);

/* Select environment e (0 .. n_envs - 1) of the handle: every later call
 * (absorb, compress, sweep value, contract, expect, checkpoints, spectra, site
 * maps) acts on it until the next select. The environments of one handle are
 * independent sweeps over the same lattice (Sec. V computes sixteen such
 * environments): each has its own boundary, sweep state and value, and its own
 * Gaussian sketches, since its index enters the generator counter (word 3 =
 * row | e << 16); they share the lattice, the staged sandwich data, the
 * engine's scratch and the stream. Environment 0 is selected at creation.
 * Selecting costs no device work. Errors: FPEPS_ERR_ARG (e out of range). */
fpeps_status fpeps_env_select(fpeps_env* env, int32_t e);

/* Last error message of the env (never NULL; "" when none). */
const char* fpeps_last_error(const fpeps_env* env);

/* Release every resource of the env (safe on NULL). */
void fpeps_env_destroy(fpeps_env* env);

/* ---- diagnostics used by the tests (same arithmetic as the path) ---------- */

/* Number of elements of the boundary tensor of site c (after the last step). */
fpeps_status fpeps_boundary_shape(const fpeps_env* env, int32_t c, int32_t* t_left, int32_t* phys,
                                  int32_t* t_right);

/* Singular values kept at bond c by the last compress call (zip-up pass when
 * which = 0, fit pass when which = 1); n_inout in: capacity, out: count. */
fpeps_status fpeps_bond_spectrum(const fpeps_env* env, int32_t which, int32_t c, double* sv_host,
                                 int32_t* n_inout);

/* Apply one site's matrix Theta_c of the staged row to k host vectors:
 * op 0: Y = Theta_c X, X [k][t_c * |R_c|] (column index t_c * |R_c| + R flat,
 *       C order), Y [k][a * |Dn_c|] using the left environment `el_host`
 *       [a][t_{c-1}][|L_c|] given by the caller.
 * Element type = compute precision. Synchronises the stream. */
fpeps_status fpeps_apply_theta(fpeps_env* env, int32_t c, int32_t a, const void* el_host, int32_t k,
                               const void* x_host, void* y_host);

/* The four site maps of the staged row on k host vectors (Sec. IV: the rSVD
 * applies the site matrix and its transpose; the CBE fit of Sec. IV / Fig. 5
 * applies the same contraction pattern 2(a) of Sec. III with the environment
 * on the right). Notation: t = left bond of the boundary tensor T_c, t' = its
 * right bond, L, R, Dn = the (ket, PEPO, bra) bundles of the site's left,
 * right and down legs, a = the caller's environment bond. All host arrays are
 * C order, vector index outermost, bundles in (ket, PEPO, bra) order:
 *   op 0  Y = Theta_c X          env [a][t][L]   in X [k][t'][R]  out Y [k][a][Dn]
 *   op 1  Z = Theta_c^T Y        env [a][t][L]   in Y [k][a][Dn]  out Z [k][t'][R]
 *   op 2  Z = ThetaR_c X         env [a][t'][R]  in X [k][Dn][a]  out Z [k][t][L]
 *   op 3  X = ThetaR_c^T Z       env [a][t'][R]  in Z [k][t][L]   out X [k][Dn][a]
 * where ThetaR_c maps a vector on (Dn, a) through the right environment, the
 * site sandwich and T_c to (t, L). The buffers are the caller's and must hold
 * the sizes above (the library cannot check host sizes). Element type =
 * compute precision; the products run in the env's precision mode on the same
 * kernels as the compress step. Synchronises the stream.
 * Errors: FPEPS_ERR_ARG for op outside 0..3, c outside the row, a, k < 1 or a
 * NULL buffer; FPEPS_ERR_STATE when no row is staged. */
fpeps_status fpeps_apply_theta_op(fpeps_env* env, int32_t op, int32_t c, int32_t a, const void* env_host, int32_t k,
                                  const void* in_host, void* out_host);

/* One contraction GEMM of the path on caller device buffers (diagnostic):
 * C[M][N] (row-major) = sum_k A[m][k] B[n][k]; A [M][lda], B [N][ldb] fp32.
 * mode FPEPS_F32: CUDA-core FP32; FPEPS_TF32X3 / FPEPS_BF16X3: tensor-core
 * 3xTF32 / 3xBF16 (needs K >= 32, lda and ldb multiples of 4, 16-byte aligned
 * A and B, else FPEPS_ERR_UNSUPPORTED). Synchronises `cuda_stream` for the
 * tensor-core modes. */
fpeps_status fpeps_gemm_f32(int32_t mode, int64_t M, int64_t N, int64_t K, const float* A, int64_t lda,
                            const float* B, int64_t ldb, float* C, void* cuda_stream);

/* Small dense SVD of the path (diagnostic), FP64, one-sided Jacobi:
 * M (k x k, column-major, device, not modified) = U diag(sigma) V^T with sigma
 * descending and U, V column-major k x k (device). Columns whose singular value
 * is below 1e-15 of the Frobenius norm get a zero U column. 1 <= k <= 1024.
 * The path passes the transposed triangular factor of a QR, for which the
 * method converges in about ten sweeps; the sweep count is capped at 30, so a
 * badly conditioned general matrix may return before full convergence.
 * Allocates its scratch (2 k^2 doubles) with cudaMallocAsync on `cuda_stream`
 * and synchronises it. */
fpeps_status fpeps_svd_f64(const double* M, int32_t k, double* U, double* sigma, double* V, void* cuda_stream);

/* Largest k accepted by fpeps_svd_f64_noalloc. */
#define FPEPS_SVD_NOALLOC_MAX_K 256

/* Same SVD as fpeps_svd_f64, for callers that cannot allocate device memory
 * during the call (for instance when another allocator already owns the whole
 * device pool, or in a latency-critical loop where an allocation could stall or
 * fail). It allocates nothing: its working storage (2 k^2 doubles, k ints and a
 * few counters; about 1.05 MB) is a fixed device array inside the library, held
 * on every GPU that loads the library until the process exits. The paper has no
 * counterpart; this is an interface of this library only.
 *   M (k x k, column-major, device, unchanged), U, V (k x k, column-major,
 *   device), sigma (k, device): outputs as for fpeps_svd_f64.
 *   1 <= k <= FPEPS_SVD_NOALLOC_MAX_K; larger k returns FPEPS_ERR_ARG.
 * The first call on a device looks up the array's device address (once per
 * device, with that device current); make that first call before any stream
 * capture. The address is kept for the life of the process: after a
 * cudaDeviceReset of that device it is stale, and the entry point must not be
 * called on that device again. Calls share the array: calls that overlap on the GPU (other streams,
 * other host threads) race. Synchronises `cuda_stream`. */
fpeps_status fpeps_svd_f64_noalloc(const double* M, int32_t k, double* U, double* sigma, double* V,
                                   void* cuda_stream);

/* Self-test of the failure path (diagnostic): launches the tensor-core GEMM with
 * its loads withheld, on a 128 x 128 x 32 product (single CTA) and on a
 * 256 x 128 x 32 product (CTA pair), so that every bounded wait in the kernel
 * (about one second each) runs out; the kernel sets its error word, frees its
 * tensor memory and exits, and the context stays usable. Returns
 * FPEPS_ERR_TIMEOUT when both launches took that path as designed (FPEPS_OK
 * means a wait did not notice the missing data). Allocates its buffers with
 * cudaMallocAsync on `cuda_stream` and synchronises it. The paper has no
 * counterpart. */
fpeps_status fpeps_selftest_wait_timeout(void* cuda_stream);

/* Number of kernels this library has launched in the process so far. */
int64_t fpeps_launch_count(void);

/* Per-kernel-class timing with CUDA events recorded on the launching stream.
 * fpeps_profile(1) clears the records and starts recording, fpeps_profile(0)
 * clears and stops. fpeps_profile_read(kind) returns, for the recorded
 * launches of one class, their count, summed device time (ms), summed
 * algorithmic flops and summed algorithmic bytes; it synchronises on the
 * recorded events. kind: 0 tensor-core GEMM, 1 CUDA-core GEMM, 2 sandwich,
 * 3 Gram, 4 small factorisations (Cholesky, inverse, Jacobi), 5 Gaussian
 * sketch (flops 0, bytes = the sketch matrix written). */
fpeps_status fpeps_profile(int32_t enable);
fpeps_status fpeps_profile_read(int32_t kind, int64_t* launches, double* ms, double* flops, double* bytes);

/* Library version string. */
const char* fpeps_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FPEPS_H */
