/*
 * subapsnap.h — C ABI of the GB300 library for the online stage of SubApSnap
 * (Jones & Nakatsukasa, "SubApSnap", arXiv 2510.04825).
 *
 * For a parameter-dependent system A(p) x(p) = b(p), an orthonormal snapshot
 * basis S (n x r) and a row subsample J (|J| = s, r <= s <= n), every new
 * parameter p is solved by
 *     M(p) = A(p)_{J,:} S                       (Alg. 1 step 4; Sec. 3.1)
 *     y(p) = argmin_y || M(p) y - b_J ||_2      (Alg. 1 step 4; Eq. 3)
 *     x(p) ~ S y(p)   or   H(p) ~ (c^T S) y(p)  (Alg. 1 step 4; Sec. 5.2.2)
 *
 * Conventions for every entry point:
 *  - Pointers named "device" must be CUDA device (or managed) memory on the
 *    current device; "host" pointers are ordinary host memory.
 *  - Matrices are column-major unless stated: entry (i, k) of an n x r matrix
 *    with leading dimension ld sits at [i + k*ld].  Complex values are
 *    interleaved (re, im) pairs of double (C99 double _Complex layout).
 *  - The caller owns every buffer it passes; a context keeps the device
 *    pointers given at setup (S, CSR arrays, kernel points) and the caller
 *    must keep them alive and unchanged until subapsnap_destroy.  The
 *    context owns what it allocates (blocks, copies, scratch).
 *  - Work is enqueued on the caller's stream (a cudaStream_t passed as
 *    void*, NULL = legacy default stream) and is asynchronous unless stated.
 *    A returned status reports argument checks and launch errors only.
 *  - No call throws; on failure a call returns a non-zero sas_status and
 *    subapsnap_last_error() gives a message (per host thread).
 *  - A context is not thread-safe: one host thread at a time per context.
 */
#ifndef SUBAPSNAP_H
#define SUBAPSNAP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sas_ctx sas_ctx;

/* Return codes. */
typedef enum {
  SAS_OK = 0,
  SAS_EINVAL = 1,    /* bad argument (sizes, NULL pointer, J out of range or repeated, ...) */
  SAS_ENOMEM = 2,    /* device allocation failed */
  SAS_ECUDA = 3,     /* CUDA runtime error (launch or synchronisation) */
  SAS_ERANK = 4,     /* M(p_sel) is numerically rank deficient at setup */
  SAS_ETIMEOUT = 5,  /* a bounded device wait ran out (see subapsnap_device_status) */
  SAS_ENOTSUP = 6,   /* combination of options not supported */
  SAS_ENOCONV = 7    /* an iterative solve stopped (iteration limit or breakdown)
                        before its tolerance; the outputs hold the last iterates */
} sas_status;

/* Per-parameter flag bits written to the optional flags[m] array. */
enum {
  SAS_FLAG_ILLCOND = 1u,   /* min|R_ii| <= 1e-13 max|R_ii|: M(p) near rank deficient */
  SAS_FLAG_NONFINITE = 2u, /* a NaN or Inf reached y */
  SAS_FLAG_REFINE_STALL = 4u, /* mixed mode: refinement did not reach its tolerance */
  SAS_FLAG_SURROGATE = 8u,     /* gated solve: the network's prediction was accepted */
  SAS_FLAG_FALLBACK = 16u      /* gated solve: rejected, solved by least squares instead */
};

/* Element type of S, b and the outputs. */
enum { SAS_REAL64 = 0, SAS_COMPLEX128 = 1 };

/* How theta(p) is formed from a parameter vector p (dp doubles per parameter):
 *  SAS_THETA_LINEAR: theta = (1, p_1, ..., p_{K-1}), dp = K - 1, real.
 *                    A(p) = A_0 + sum_k p_k A_k.
 *  SAS_THETA_PENCIL: theta = (-1, i*omega), dp = 1 (p = omega), K = 2,
 *                    A = (i omega) E - A_0 with blocks (A_0, E): the
 *                    transfer-function resolvent of Sec. 5.2 (Eq. 9) on the
 *                    imaginary axis.  Requires SAS_COMPLEX128.
 *  SAS_THETA_DELAY:  theta = (i*omega, -1, -exp(i*omega*tau)), dp = 2
 *                    (p = (omega, tau)), K = 3: A = p I - A_0 - e^{tau p} A_1
 *                    with blocks (I, A_0, A_1) at p = i omega, the delay
 *                    system of Sec. 5.2.3.  Requires SAS_COMPLEX128.       */
enum { SAS_THETA_LINEAR = 0, SAS_THETA_PENCIL = 1, SAS_THETA_DELAY = 2 };

/* Quantity of interest computed from y without any n-vector (Sec. 5.2.2). */
enum { SAS_QOI_NONE = 0, SAS_QOI_TRANSPOSE = 1 /* c^T x, plain transpose */,
       SAS_QOI_MEAN = 2 /* (1/n) sum_i x_i */ };

/* Arithmetic of the online solve.
 *  SAS_MODE_PLAIN: float64 (complex128) assembly, Householder QR and
 *                  reconstruction.
 *  SAS_MODE_MIXED: float32 assembly and Householder QR, iterative refinement
 *                  of y with the subsampled residual b_J - M y formed in
 *                  float64, and a float64-accurate reconstruction on the
 *                  tensor cores: 9-bit fixed-point digits of S and y, their
 *                  products summed exactly in the f32 accumulators and
 *                  assembled as int64 (x_hat returned as float64, within
 *                  ~2^-43 of the scale max_k|S_ik| ||y||_1 of each entry;
 *                  r <= 64, otherwise the float64 CUDA-core product).  With
 *                  SAS_OPT_XHAT_F32 = 1, x_hat is float32 from three tf32
 *                  products instead.  Not in the paper.                     */
enum { SAS_MODE_PLAIN = 0, SAS_MODE_MIXED = 1 };

/* What subapsnap_solve_batch writes to `out` for each of its m parameters. */
enum {
  SAS_OUT_Y = 0,     /* y: m x r, row j at out + j*r (dtype of S) */
  SAS_OUT_XHAT = 1,  /* x_hat = S y: m x n, row j at out + j*n; double (real),
                        float when SAS_MODE_MIXED and SAS_OPT_XHAT_F32 = 1 */
  SAS_OUT_QOI = 3    /* H = (c^T S) y: m values (dtype of S) */
};

#define SAS_MAX_TERMS 8

/* Affine operator family A(p) = sum_k theta_k(p) A_k with constant b.
 * The A_k are real sparse n x n matrices in CSR form (device arrays). */
typedef struct {
  int64_t n;            /* order of A(p); rows of S */
  int32_t r;            /* columns of S (1 <= r <= 128) */
  int32_t s;            /* rows in the subsample (r <= s <= n, s <= 512) */
  int32_t K;            /* number of terms, 1..SAS_MAX_TERMS */
  int32_t dtype;        /* SAS_REAL64 or SAS_COMPLEX128 */
  int32_t theta_rule;   /* SAS_THETA_LINEAR, SAS_THETA_PENCIL or SAS_THETA_DELAY */
  int32_t mode;         /* SAS_MODE_PLAIN or SAS_MODE_MIXED */
  const void* S;        /* device, n x r, leading dimension ldS >= n */
  int64_t ldS;
  const int64_t* J;     /* host, s distinct row indices in [0, n); order kept */
  const void* b;        /* device, n entries of dtype */
  const int64_t* rowptr[SAS_MAX_TERMS]; /* device, n + 1 offsets per term */
  const int32_t* colind[SAS_MAX_TERMS]; /* device, column indices per term */
  const double* values[SAS_MAX_TERMS];  /* device, values per term */
  int32_t qoi_kind;     /* SAS_QOI_* */
  const double* c;      /* device, n real entries for SAS_QOI_TRANSPOSE, else NULL */
  const double* w;      /* host, s positive row weights (leverage-score sampling,
                           Sec. 4.3.2 footnote): row i of M(p) and of b_J is scaled
                           by w[i]; NULL = unweighted */
} sas_affine_desc;

/* Gaussian-kernel ridge regression A(sigma, lambda) = K_sigma + lambda I,
 * K_sigma(x, x') = exp(-|x - x'|^2 / (2 sigma^2)), b = targets (Sec. 5.3,
 * Eqs. 10-11).  Parameters are p = (sigma, lambda), dp = 2.  Real only. */
typedef struct {
  int64_t n;            /* number of points N */
  int32_t d;            /* point dimension (1..16) */
  int32_t r;            /* columns of S (<= 128) */
  int32_t s;            /* rows in the subsample (r <= s <= 512) */
  int32_t mode;         /* SAS_MODE_PLAIN or SAS_MODE_MIXED */
  const double* X;      /* device, N x d row-major (point i at X + i*d) */
  const double* S;      /* device, N x r, leading dimension ldS >= N */
  int64_t ldS;
  const int64_t* J;     /* host, s distinct indices in [0, N) */
  const double* b;      /* device, N targets */
} sas_kernel_desc;

/* One shard of the points of a Gaussian-kernel problem (the data-parallel
 * split of Sec. 5.3's rows over N for several GPUs): base.X and base.S hold
 * this shard's N_g points and rows of S (base.n = N_g; base.J and base.b are
 * ignored), and the subsample's rows come from the caller, so that every shard
 * uses the same J of the full problem. */
typedef struct {
  sas_kernel_desc base;
  const double* XJ;  /* device, s x d row-major: coordinates of the points at J */
  const double* SJ;  /* device, s x r column-major (ld s): S's rows at J on ONE shard, zeros on
                        the others, so that the lambda S_J term enters the sum once */
  const double* bJ;  /* device, s: b at J */
} sas_kernel_shard_desc;

/* Build a context for the affine family: gathers b_J, precomputes the blocks
 * G_k = (A_k)_{J,:} S (s x r each) so that M(p) = sum_k theta_k(p) G_k costs
 * O(K s r) per parameter (Sec. 3.1, "Computing S A(p*) X"; Sec. 5.2.2), and
 * the QoI vector c^T S.  Synchronous: returns after the device work is done.
 * Errors: SAS_EINVAL for inconsistent sizes, NULL pointers or a J that is
 * out of range or repeated; SAS_ENOMEM; SAS_ECUDA. */
sas_status subapsnap_setup_affine(const sas_affine_desc* desc, sas_ctx** out);

/* Build a context for the Gaussian-kernel family (Sec. 5.3): keeps X, S and
 * gathers X_J, S_J and b_J.  The rows K_sigma(X_J, X) are formed on the fly
 * in every solve.  Synchronous.  Errors as subapsnap_setup_affine. */
sas_status subapsnap_setup_kernel(const sas_kernel_desc* desc, sas_ctx** out);

/* Context over one point shard (see sas_kernel_shard_desc).  Its rows are
 * partial: subapsnap_kernel_rows gives M_g = K_sigma(X_J, X_g) S_g + lambda
 * S_J^(g); the caller sums them over the shards (one all-reduce of m x s x r
 * doubles) and solves with subapsnap_solve_batch_rows.  subapsnap_solve_batch
 * refuses a shard context (SAS_ENOTSUP).  Not in the paper.  Synchronous.
 * Errors as subapsnap_setup_kernel. */
sas_status subapsnap_setup_kernel_shard(const sas_kernel_shard_desc* desc, sas_ctx** out);

/* Kernel rows of a Gaussian-kernel context (Sec. 5.3, Sec. 3.1's rows at J):
 * M_q = K_sigma(X_J, X) S + lambda S_J for m parameters (sigma, lambda), by
 * the context's assembly (float64 in the plain form, the tensor-core rows in
 * the mixed form).  M: device, m x (s x r) doubles, each parameter's block
 * column-major with ld s.  Asynchronous on `stream`.  Errors: SAS_EINVAL,
 * SAS_ENOTSUP (not a kernel context), SAS_ECUDA. */
sas_status subapsnap_kernel_rows(sas_ctx* ctx, const double* params, int64_t m, double* M,
                                 void* stream);

/* Least squares min ||M_q y - b_J|| from given rows (Alg. 1 step 4), e.g. the
 * shard sums of subapsnap_kernel_rows: the context's solver (plain float64
 * Householder, or the mixed form with float64 refinement against M).  Y:
 * device m x r; flags, rho as in subapsnap_solve_batch.  Asynchronous.
 * Errors: SAS_EINVAL, SAS_ENOTSUP (not a kernel context), SAS_ECUDA. */
sas_status subapsnap_solve_batch_rows(sas_ctx* ctx, const double* params, int64_t m, const double* M,
                                      double* Y, uint32_t* flags, double* rho, void* stream);

/* Solve m new parameters (Alg. 1 step 4).
 *  params: device, m x dp row-major doubles (dp from the family).
 *  out:    device, layout per out_kind (see SAS_OUT_*).
 *  flags:  device, m uint32 (SAS_FLAG_* bits) or NULL.
 *  rho:    device, m doubles or NULL: the subsampled relative residual
 *          ||M(p) y - b_J|| / ||b_J|| (Sec. 4.3.1 residual estimate).
 * Asynchronous on `stream`.  m = 0 is a no-op.  Errors: SAS_EINVAL (bad
 * pointer, out_kind or family), SAS_ECUDA (launch failure). */
sas_status subapsnap_solve_batch(sas_ctx* ctx, const double* params, int64_t m,
                                 int32_t out_kind, void* out, uint32_t* flags,
                                 double* rho, void* stream);

/* subapsnap_solve_batch (Alg. 1 step 4) with HOST buffers: params (m x dp),
 * out (layout per out_kind), flags and rho (or NULL) are ordinary host
 * memory.  The call copies params to the device, solves, and returns after
 * the outputs are in the host buffers (synchronous on `stream`).  x_hat is
 * written straight into `out` by the reconstruction when `out` is page-locked
 * host memory mapped into the device's address space (cudaHostAlloc or
 * cudaHostRegister; every such allocation is mapped under unified
 * addressing), so the transfer overlaps the computation; pageable `out` goes
 * through a device buffer in chunks (SAS_OPT_HOST_CHUNK, default 1 GiB).
 * Device staging is owned by the context.  Errors: as subapsnap_solve_batch,
 * SAS_EINVAL for a device pointer. */
sas_status subapsnap_solve_batch_host(sas_ctx* ctx, const double* params, int64_t m,
                                      int32_t out_kind, void* out, uint32_t* flags,
                                      double* rho, void* stream);

/* Reconstruction x_hat = S y of given coefficient vectors (Alg. 1 step 4,
 * "output X c"), in the context's arithmetic: float64 DFMA in
 * SAS_MODE_PLAIN; in SAS_MODE_MIXED float32 from tf32 splits of S and y on
 * the tensor cores.  Lets a caller solve a large batch with SAS_OUT_Y once and
 * reconstruct it in chunks.
 *  Y:   device, m x r of the dtype of S (row j = y of parameter j).
 *  out: device, m x n: double (plain) or float (mixed); row j = x_hat_j.
 * Asynchronous.  Errors: SAS_EINVAL (NULL pointer), SAS_ENOTSUP (complex
 * context), SAS_ECUDA. */
sas_status subapsnap_reconstruct(sas_ctx* ctx, const void* Y, int64_t m, void* out, void* stream);

/* Subsampled relative residual ||M(p) y - b_J|| / ||b_J|| of given
 * coefficient vectors (Sec. 4.3.1), in float64.
 *  params: device m x dp; Y: device m x r (dtype of S); rho: device m. */
sas_status subapsnap_residual(sas_ctx* ctx, const double* params, int64_t m,
                              const void* Y, double* rho, void* stream);

/* True relative residual ||A(p) x - b|| / ||b|| of full-length vectors
 * (affine family only; the quantity Tables 3-4 report as (max, median)).
 *  params: device m x dp; X: device m x n (row j = x for parameter j, dtype
 *  of S); rho: device m.  Reads every CSR block once per parameter. */
sas_status subapsnap_true_residual(sas_ctx* ctx, const double* params, int64_t m,
                                   const void* X, double* rho, void* stream);

/* Row selection by column-pivoted QR on (A(p_sel) S)^T (Sec. 4.3; Alg. 1
 * step 3), in rounds for s > r: round 1 is CPQR; each later round repeats
 * CPQR on the same matrix with the earlier picks removed (the union of
 * pivot sets of Sec. 4.3.2), until s rows are held.  Pivot rule: largest
 * remaining residual norm in float64, exact ties to the lowest index.
 *  desc:   as for setup (J, b, qoi fields are ignored).
 *  p_sel:  host, dp doubles.
 *  J_out:  host, s indices in pick order.
 *  gap_out: host, s doubles or NULL: (best - runner-up) / best per step.
 * Synchronous.  Errors: SAS_EINVAL, SAS_ENOMEM, SAS_ECUDA, SAS_ERANK if a
 * round runs out of non-zero residuals. */
sas_status subapsnap_select_rows_affine(const sas_affine_desc* desc, const double* p_sel,
                                        int64_t* J_out, double* gap_out);

/* Capacity, in coefficients (m * r), of the fixed device array used by
 * subapsnap_solve_batch_xhat_noalloc: 65536 doubles = 512 KiB. */
#define SAS_NOALLOC_MAX_Y 65536

/* Same result as subapsnap_solve_batch(ctx, params, m, SAS_OUT_XHAT, out,
 * flags, rho, stream) on the plain float64 path (whatever the context's
 * mode), for callers that cannot allocate device memory when they solve:
 * the call calls no cudaMalloc, cudaFree or allocating library routine.  The
 * m x r coefficient vectors between the least-squares and reconstruction
 * kernels go to one fixed device array of SAS_NOALLOC_MAX_Y doubles that
 * every device loading the library holds until the process exits.  No
 * counterpart in the paper.
 *  params: device m x dp; out: device m x n doubles (row j = x_hat of
 *  parameter j); flags, rho: device m or NULL, as for solve_batch.
 * Context set-up looks the array's address up (and brings the array onto the
 * device); every call looks it up again, so the address stays right after a
 * device reset.  Make the first call before any stream capture.  All calls
 * share the array and calls that overlap on the GPU race on it.
 * Errors: SAS_EINVAL if m * r > SAS_NOALLOC_MAX_Y or a pointer is NULL;
 * SAS_ENOTSUP for a complex or kernel-family context; SAS_ECUDA. */
sas_status subapsnap_solve_batch_xhat_noalloc(sas_ctx* ctx, const double* params, int64_t m,
                                              double* out, uint32_t* flags, double* rho,
                                              void* stream);

/* Bytes that subapsnap_solve_batch / subapsnap_solve_batch_host write per
 * parameter for out_kind (and subapsnap_reconstruct for SAS_OUT_XHAT) under the
 * context's current mode and options: r elements for SAS_OUT_Y, n for
 * SAS_OUT_XHAT (8-byte double, or 4-byte float when SAS_OPT_XHAT_F32 = 1 in
 * SAS_MODE_MIXED), one for SAS_OUT_QOI.  A caller sizes `out` as m times this.
 * Not in the paper.  Errors: SAS_EINVAL (NULL argument or bad out_kind). */
sas_status subapsnap_output_row_bytes(const sas_ctx* ctx, int32_t out_kind, int64_t* bytes);

/* Per-context options (subapsnap_set_option).  Not in the paper.
 *  SAS_OPT_RECON_KERNEL: mixed-form reconstruction kernel.  float64 x_hat:
 *      1 = float64 CUDA-core product, any other value = the digit products on
 *      the tensor cores (when r <= 64).  float32 x_hat (SAS_OPT_XHAT_F32): 0 =
 *      automatic (tensor cores when r <= 64, as 3), 1 = CUDA cores, 2 = tensor cores
 *      (tcgen05, kind::tf32, three split products) with 64-parameter tiles,
 *      3 = as 2 with 128-parameter tiles, 4 = as 3 with the parameter tiles
 *      of each row tile visited in a rotated order, 5 = tensor cores
 *      (kind::f16) on power-of-two-scaled f16 splits of S and y, three
 *      products into two accumulators, 128-parameter tiles, 6 = as 3 with
 *      eight epilogue warps (direct stores).
 *  SAS_OPT_MAX_REFINE: most refinement steps of the mixed solve (0..16,
 *      default 4).
 *  SAS_OPT_REFINE_TOL: refinement stops when ||delta|| <= tol ||y||
 *      (default 1e-13) or when a step no longer halves the correction.
 *  SAS_OPT_LS_VARIANT: launch shape of the least-squares kernel of the
 *      context's mode (the index subapsnap_autotune reports; 0 = default).
 *  SAS_OPT_ASSEMBLY_KERNEL: kernel rows of the mixed kernel-ridge form:
 *      0 = automatic (tensor cores), 1 = CUDA cores (float32 entries, float64
 *      chunk sums), 2 = tensor cores (tcgen05, kind::tf32, entries and S in
 *      three split products, float32 TMEM sums folded into float64).
 *  SAS_OPT_ASSEMBLY_SEGMENT: tensor-core kernel rows: points summed in float32
 *      before each float64 fold (multiple of 32 in [32, 2^20], default 1024);
 *      shorter segments cost more folds and round less.
 *  SAS_OPT_RECON_STORE: epilogue of the tensor-core reconstruction: 0 = tiles
 *      staged in shared memory and written by TMA bulk-tensor stores (when n
 *      is a multiple of 4 and the output 16-byte aligned), 1 = coalesced
 *      streaming stores straight from registers (default).
 *  SAS_OPT_HOST_CHUNK: subapsnap_solve_batch_host with pageable x_hat: bytes
 *      of the device chunk x_hat goes through (at least one parameter's row;
 *      default 2^30).
 *  SAS_OPT_XHAT_F32: mixed form only: 1 = x_hat returned as float32 (three
 *      tf32 products, ~2^-21 relative; not residual-equivalent to float64
 *      for an operator with large ||A||), 0 = float64 (default). *  SAS_OPT_SURROGATE_F32_OUT: 1 = the surrogate's output layer uses its float32
 *      weights (each entered as two bfloat16 terms on the tensor cores) instead
 *      of the bfloat16 copy; training, prediction and gradients use the current
 *      setting (default 0).
 */
enum { SAS_OPT_RECON_KERNEL = 0, SAS_OPT_MAX_REFINE = 1, SAS_OPT_REFINE_TOL = 2,
       SAS_OPT_LS_VARIANT = 3, SAS_OPT_ASSEMBLY_KERNEL = 4, SAS_OPT_ASSEMBLY_SEGMENT = 5,
       SAS_OPT_RECON_STORE = 6, SAS_OPT_HOST_CHUNK = 7, SAS_OPT_XHAT_F32 = 8,
       SAS_OPT_SURROGATE_F32_OUT = 9 };

/* Set one option of a context.  Errors: SAS_EINVAL for an unknown key or a
 * value out of range. */
sas_status subapsnap_set_option(sas_ctx* ctx, int32_t key, double value);

/* ---------------------------------------------------------------- offline stage */

/* Flags of subapsnap_krylov_affine. */
enum { SAS_KRYLOV_WARM = 1,     /* X holds start vectors (else zero start) */
       SAS_KRYLOV_MIXED = 2,    /* float32 iterates, float64 residual replacements */
       SAS_KRYLOV_BICGSTAB = 4  /* BiCGStab for nonsymmetric A(p): float64 iterates, diagonal
                                   preconditioner; when its iterated residual reaches tol the
                                   true residual decides, and it restarts from that one */ };

/* Snapshot solves A(p_j) x_j = b, j = 0..B-1, all at once (Alg. 1 step 1,
 * "fully or approximately"): conjugate gradients in the bilinear form x^T y
 * (COCG; plain CG for real data) with the diagonal of A(p_j) as
 * preconditioner.  A(p) must be symmetric (A^T = A; complex symmetric for the
 * pencil and delay rules) with a non-zero diagonal; the method converges for
 * positive definite A(p) and in practice for the complex symmetric families
 * here.  Nonsymmetric A(p) take SAS_KRYLOV_BICGSTAB.  The same call refines given start vectors (SAS_KRYLOV_WARM), e.g.
 * the SubApSnap output x_hat as the initial guess of Sec. 3.2.  Convergence
 * is only ever declared on the true residual b - A x computed in float64:
 * when the iterated residual reaches tol it is replaced by the true one and
 * the iteration goes on if that is still above tol; a column stops (as not
 * converged) once four replacements in a row fail to halve the true
 * residual, i.e. when tol lies below the attainable accuracy.  With SAS_KRYLOV_MIXED
 * the iterates, directions and matrix values are float32 and the float64
 * solution takes their corrections, the residual being replaced by the true
 * float64 one whenever the float32 residual has fallen 10x since the last
 * replacement (not in the paper; needs kappa(A) well below 1e7).
 *  desc:    the family (n, K, dtype, theta_rule, CSR blocks, b); r, s, S, J,
 *           mode, qoi and w are ignored.
 *  params:  host, B x dp, 1 <= B <= 256.
 *  X:       device, n x B column-major (column j = x_j, ld n), float64 or
 *           complex128; on entry the start vectors with SAS_KRYLOV_WARM.
 *  flags:   SAS_KRYLOV_* bits.
 *  tol:     column j stops once ||b - A x_j|| / ||b|| <= tol; maxit bounds
 *           its iterations.
 *  iters_out:  host, B ints or NULL: iterations per column.
 *  relres_out: host, B doubles or NULL: the true ||b - A x_j|| / ||b|| of
 *           the returned x_j, recomputed at the end.
 * Synchronous (own stream).  Errors: SAS_EINVAL (sizes, pointers, rule, zero
 * diagonal, b = 0), SAS_ENOMEM, SAS_ECUDA, SAS_ENOCONV (a column stopped at
 * maxit or broke down; X holds the last iterates). */
sas_status subapsnap_krylov_affine(const sas_affine_desc* desc, const double* params, int32_t B,
                                   void* X, int32_t flags, double tol, int32_t maxit,
                                   int32_t* iters_out, double* relres_out);

/* Preconditioners of subapsnap_krylov_affine_ex. */
enum { SAS_PRECOND_JACOBI = 0, SAS_PRECOND_POISSON = 1 };

/* SAS_PRECOND_POISSON (not in the paper; a classical preconditioner for its
 * grid problems): M_j = alpha_j L + beta_j I with L the unit-spacing
 * Dirichlet Laplacian of an nx x ny x nz grid (the sum over the axes of
 * tridiag(-1, 2, -1)), point i = ix + nx (iy + ny iz).  M_j^-1 is applied
 * exactly by the discrete sine transform along each axis (dense float32
 * transforms on the tensor cores).  For the 2-D diffusion family A(p) =
 * A_0 + sum p_k A_k with A_0 = h^-2 L, alpha = h^-2 and beta = 0 make A_0 the
 * preconditioner; for the transfer function i omega E - A_0 with
 * A_0 = -h^-2 L, alpha = h^-2 and beta = i omega mean(E). */
typedef struct {
  int32_t kind;        /* SAS_PRECOND_* */
  int32_t ndim;        /* POISSON: 1, 2 or 3 axes */
  int64_t dims[3];     /* POISSON: grid size per axis (each <= 8192), product = n */
  const double* coef;  /* POISSON: host, B x 4 doubles per column:
                          alpha_re, alpha_im, beta_re, beta_im (imaginary parts 0 for real data) */
} sas_krylov_precond;

/* subapsnap_krylov_affine with a choice of preconditioner (NULL = Jacobi).
 * Errors: as subapsnap_krylov_affine; SAS_EINVAL for a grid that does not
 * have n points, an axis above 8192 or complex coefficients on real data. */
sas_status subapsnap_krylov_affine_ex(const sas_affine_desc* desc, const double* params, int32_t B,
                                      void* X, int32_t flags, double tol, int32_t maxit,
                                      const sas_krylov_precond* precond, int32_t* iters_out,
                                      double* relres_out);

/* Snapshots of the Gaussian-kernel family (Alg. 1 step 1 for Sec. 5.3): the
 * solutions x of (K_sigma + lambda I) x = b on the grid of nsigma sigma values
 * times nlambda lambda values, by multishift conjugate gradients: for each
 * sigma one CG on the smallest lambda, every other lambda from the shifted
 * recurrences of the same Krylov space (one kernel product per sigma and
 * iteration for all lambda).  All sigma advance together.  A system stops once
 * its recurrence residual is at most tol ||b||.  float64 throughout: distances
 * from direct coordinate differences, entries by exp.
 *  desc:   X (device N x d), n, d and b (device N) are used; S, J, r, s, mode
 *          are ignored.
 *  sigma:  host, nsigma values > 0 (1 <= nsigma <= 16).
 *  lambda: host, nlambda values > 0 (1 <= nlambda <= 32).
 *  X_out:  device, N x (nsigma nlambda) column-major (ld ldx >= N); column
 *          a nlambda + b solves (sigma_a, lambda_b).
 *  iters_out (host or NULL): iterations per system; relres_out (host or
 *  NULL): true float64 residuals ||(K + lambda I) x - b|| / ||b||.
 * Allocates device work space (about N (nsigma nlambda + 2 nsigma + 32)
 * doubles).  Synchronous on `stream`.  Errors: SAS_EINVAL, SAS_ENOMEM,
 * SAS_ECUDA, SAS_ENOCONV (a system did not reach tol within maxit iterations
 * or broke down; X_out holds the last iterates). */
sas_status subapsnap_krr_snapshots(const sas_kernel_desc* desc, const double* sigma, int32_t nsigma,
                                   const double* lambda, int32_t nlambda, double tol, int32_t maxit,
                                   double* X_out, int64_t ldx, int32_t* iters_out, double* relres_out,
                                   void* stream);

/* Thin QR X = Q R of a tall n x r matrix on the device by TSQR (Alg. 1 step
 * 2: an orthonormal basis Q of the snapshots' range): Householder QR of row
 * panels in shared memory and of stacks of their R factors up a reduction
 * tree, Q formed by applying the reflectors top-down.  Column signs are
 * chosen so that diag(R) >= 0 (R real on its diagonal), which makes Q unique
 * when X has full rank; a rank-deficient X still gets an orthonormal Q.
 *  X:  device n x r (ld ldx >= n), dtype SAS_REAL64 or SAS_COMPLEX128.
 *  Q:  device n x r (ld ldq >= n); may be X itself (ldq == ldx).
 *  R_out: host r x r column-major or NULL.
 * Limits: r <= 120 real, r <= 84 complex (a panel of 2r rows in shared
 * memory).  Synchronous.  Errors: SAS_EINVAL, SAS_ENOTSUP (r too large),
 * SAS_ENOMEM, SAS_ECUDA. */
sas_status subapsnap_tsqr(const void* X, int64_t n, int32_t r, int64_t ldx, int32_t dtype,
                          void* Q, int64_t ldq, void* R_out);

/* Union of pivot sets (Sec. 4.3.4): the CPQR selection of
 * subapsnap_select_rows_affine with s = s_each at each of t parameters
 * points[i * dp .. i * dp + dp), the picks merged in order of first
 * appearance.  J_out: host, room for t * s_each indices; *count_out: how many
 * distinct rows (between s_each and t * s_each).  Synchronous.  Errors: as for
 * subapsnap_select_rows_affine. */
sas_status subapsnap_select_rows_union_affine(const sas_affine_desc* desc, const double* points,
                                              int32_t t, int32_t s_each, int64_t* J_out,
                                              int32_t* count_out);

/* Nearest selection point of each parameter (Sec. 4.3.4: the rows chosen at
 * the snapshot point closest to p): idx_out[q] = argmin_i |params_q -
 * points_i| in the Euclidean norm of the parameter vector, ties to the lowest
 * i.  Host arrays: params m x dp, points t x dp, idx_out m.  Errors: SAS_EINVAL. */
sas_status subapsnap_nearest_points(const double* params, int64_t m, int32_t dp,
                                    const double* points, int32_t t, int32_t* idx_out);

/* Leverage scores of [A(p_sel) S, b] (Sec. 4.3.2-4.3.3): the squared row norms
 * of Q in the thin QR of the n x (r+1) matrix, computed on the device in
 * float64 by shifted CholeskyQR3.  Row selection by leverage-score sampling draws
 * rows with probability proportional to these scores.
 *  d: affine descriptor (J, w, mode and QoI fields unused); p_sel: host, dp
 *     doubles; scores: host, n doubles (sum r + 1 for full column rank).
 * Synchronous.  Errors: SAS_EINVAL, SAS_ERANK (the matrix is numerically rank
 * deficient), SAS_ENOMEM, SAS_ECUDA. */
sas_status subapsnap_leverage_scores_affine(const sas_affine_desc* d, const double* p_sel,
                                            double* scores);

/* Leverage-score sampling with weights (host only, Sec. 4.3.2 footnote).
 * s draws with replacement by inverse CDF of pi = scores / total on the
 * caller's uniforms u[0..s) in [0, 1): the running sums C_i of the scores in
 * row order give cdf_i = C_i / C_{n-1}, and draw t is the first i with
 * cdf_i > u[t].  Rows drawn k times are kept once, in increasing order, with
 * weight sqrt(k / (s pi_i)): pass J_out and w_out (room for s entries) to the
 * setup (sas_affine_desc.J, .w) with s = *count_out.  The weighted subsampled
 * residual then estimates the true residual within (1 -/+ eps), eps ~ r log(r)
 * / s, at p_sel (Sec. 4.3.3).  Errors: SAS_EINVAL. */
sas_status subapsnap_sample_rows_leverage(const double* scores, int64_t n, int32_t s,
                                          const double* u, int64_t* J_out, double* w_out,
                                          int32_t* count_out);

/* Autotuner (not in the paper): times every launch shape of the context's
 * least-squares kernel (threads per CTA, lanes per column group; for the mixed
 * form also where the float64 M lives: shared memory, a global slot per CTA,
 * or recomputed, and how the Householder panels run: column by column, blocked
 * with the panel on the CTA or on one warp, or, for s <= 128, blocked with the
 * panel and the refinement corrections in one warp's registers) on the caller's
 * parameters, `reps` timed
 * launches each after one warm-up, keeps the fastest in the context and
 * returns it.
 *  params: device, m x dp (a representative batch; its size matters).
 *  times_ms: host, room for SAS_MAX_VARIANTS doubles or NULL: mean time per variant
 *            (a variant that cannot run for this shape reports -1).
 *  chosen: host or NULL: index of the kept variant.
 * If the environment variable SAS_TUNE_CACHE names a file, the choice is
 * appended there under a key of (family, mode, dtype, s, r, K, m) and later
 * calls with the same key read it back instead of timing.  Synchronous on
 * `stream`.  Errors: SAS_EINVAL, SAS_ECUDA. */
#define SAS_MAX_VARIANTS 32
sas_status subapsnap_autotune(sas_ctx* ctx, const double* params, int64_t m, int32_t reps,
                              double* times_ms, int32_t* chosen, void* stream);

/* Kernel classes reported by the tracer. */
enum { SAS_KERNEL_LS = 0,           /* assembly + least squares (+ QoI epilogue) */
       SAS_KERNEL_RECONSTRUCT = 1,  /* x_hat = S y */
       SAS_KERNEL_RESIDUAL = 2,     /* subsampled / true residual */
       SAS_KERNEL_ASSEMBLE = 3,     /* Gaussian-kernel rows K_sigma(X_J, X) S */
       SAS_KERNEL_SURROGATE = 4,    /* network inference */
       SAS_KERNEL_CLASSES = 5 };

/* Tracing: when enabled (enable != 0) every kernel the context launches is
 * bracketed by a pair of CUDA events recorded on the launch stream.  Costs
 * two event records per launch; off by default.  Not part of the paper. */
sas_status subapsnap_set_tracing(sas_ctx* ctx, int32_t enable);

/* Sum of traced launch durations (milliseconds, host) and number of traced
 * launches (host) of one kernel class since the last read; resets that
 * class.  Synchronises on the recorded events.  Errors: SAS_EINVAL for a
 * bad class or NULL pointer. */
sas_status subapsnap_trace_read(sas_ctx* ctx, int32_t kernel_class, double* total_ms,
                                int64_t* launches);

/* Row selection for the Gaussian-kernel family: the same CPQR rounds on
 * V = (K_sigma + lambda I) S at p_sel = (sigma, lambda) (host, 2 doubles),
 * with V formed from float64 kernel rows of all N points (O(N^2 r) work,
 * done once).  desc: as for setup_kernel (J and b are ignored).  Synchronous.
 * Errors: SAS_EINVAL, SAS_ENOMEM, SAS_ECUDA, SAS_ERANK. */
sas_status subapsnap_select_rows_kernel(const sas_kernel_desc* desc, const double* p_sel,
                                        int64_t* J_out, double* gap_out);

/* ------------------------------------------------------------------------
 * Learned surrogate (not in the paper).  A network p -> y(p) (d_in -> 256 ->
 * 256 -> r, exact GELU, bfloat16 weights, tensor-core products with float32
 * accumulation, float32 master weights, Adam) attached to an affine context, trained by the library's own
 * kernels on coefficient vectors the online stage produced.  Its predictions
 * are accepted only when the subsampled relative residual
 * ||M(p) y_hat - b_J|| / ||b_J|| (the online residual estimate of Sec. 4.3.1,
 * evaluated in float64) is at most gate_tol; the others are solved exactly.
 * ---------------------------------------------------------------------- */

/* Train (creating the network with N(0, 1/fan_in) weights from `seed` on the
 * first call).  P: device ntrain x dp; Y: device ntrain x r (float64).
 * Inputs are scaled to [-1, 1] and outputs standardised per component from
 * this training set.  Mini-batches of `batch` rows in a seeded shuffle, Adam
 * with learning rate lr.  loss_out: host, `epochs` mean losses, or NULL.
 * Synchronous.  Errors: SAS_EINVAL, SAS_ENOMEM, SAS_ECUDA. */
sas_status subapsnap_surrogate_train(sas_ctx* ctx, const double* P, const double* Y, int64_t ntrain,
                                     int32_t epochs, int32_t batch, double lr, uint64_t seed,
                                     double* loss_out, void* stream);

/* Network predictions y_hat for m parameters (device m x dp -> device m x r). */
sas_status subapsnap_surrogate_predict(sas_ctx* ctx, const double* params, int64_t m,
                                       double* Yhat, void* stream);

/* Gated solve: predict, accept the predictions whose float64 subsampled
 * relative residual is <= gate_tol, solve the rest by the context's least
 * squares.  out_kind SAS_OUT_Y or SAS_OUT_QOI; flags (device m or NULL) gets
 * SAS_FLAG_SURROGATE or SAS_FLAG_FALLBACK (plus the solve's own flags); rho
 * (device m or NULL) the final subsampled residuals; accepted (host or NULL)
 * the number accepted.  Synchronises once (to size the fallback batch). */
sas_status subapsnap_solve_batch_surrogate(sas_ctx* ctx, const double* params, int64_t m,
                                           int32_t out_kind, void* out, uint32_t* flags,
                                           double* rho, double gate_tol, int64_t* accepted,
                                           void* stream);

/* Discard the network (weights, optimiser state and its copy of the anchors);
 * the next subapsnap_surrogate_train creates a fresh one from its seed.
 * Synchronises the device first.  Errors: SAS_EINVAL, SAS_ECUDA. */
sas_status subapsnap_surrogate_reset(sas_ctx* ctx);

/* Anchors for the next subapsnap_surrogate_train: n parameter points P
 * (device n x dp, float64) with their coefficient vectors Y (device n x r), for
 * instance the snapshot parameters with the online solution there.  A network
 * trained with anchors learns y(p) - Y[a(p)], a(p) the anchor nearest to p in
 * the network's input scaling (sum_k ((p_k - P[a]_k) / half-width_k)^2, lowest
 * index on ties), and predicts Y[a(p)] plus its output; it keeps its own copy
 * of the anchors.  The context copies P and Y (the caller keeps ownership);
 * n = 0 clears them.  Errors: SAS_EINVAL, SAS_ENOTSUP, SAS_ENOMEM, SAS_ECUDA. */
sas_status subapsnap_surrogate_set_anchors(sas_ctx* ctx, const double* P, const double* Y, int64_t n);

/* Read (get != 0) or write the network: theta (host float32, layout W1 b1 W2
 * b2 W3 b3, W_l row-major out x in) and norm (host float64: input centre[dp],
 * input half-width[dp], output mean[r], output sd[r]); either may be NULL.
 * *nparam (host, may be NULL) receives the parameter count.  Writing creates
 * the network if needed.  For checkpoints and gradient checks. */
sas_status subapsnap_surrogate_weights(sas_ctx* ctx, int32_t get, float* theta, double* norm,
                                       int64_t* nparam);

/* One forward and backward pass on a normalised batch (device float64
 * X: B x dp, Yn: B x r): loss (host) and gradients (host float32, theta
 * layout).  The bfloat16 weights of the matrix products are those the
 * network trains with.  For gradient checks. */
sas_status subapsnap_surrogate_grad(sas_ctx* ctx, const double* X, const double* Yn, int64_t B,
                                    double* loss, float* grads);

/* ------------------------------------------------------------------------
 * Persistent batched launch over several contexts (not in the paper).  One
 * kernel launch drains the parameters of nctx contexts whose s, r and K may
 * differ (operator families of the same dtype and mode): CTAs take tasks
 * from a global counter, and each task runs the same per-parameter solve as
 * subapsnap_solve_batch with the first context's launch shape.  A plan holds
 * the device descriptors; launching it is capture-safe (no allocation, no
 * synchronisation) and can replay a CUDA graph the plan captured once.
 * ---------------------------------------------------------------------- */
typedef struct sas_multi_plan sas_multi_plan;

/* Build a plan.  ctxs: host array of nctx affine contexts (same dtype and
 * mode).  params, outs, flags, rho: host arrays of nctx device pointers
 * (flags and rho may be NULL, or hold NULL entries); m: host array of batch
 * sizes.  out_kind: SAS_OUT_Y or SAS_OUT_QOI.  The pointed-to buffers must
 * outlive the plan.  Synchronous.  Errors: SAS_EINVAL, SAS_ENOMEM, SAS_ECUDA. */
sas_status subapsnap_multi_plan_create(sas_ctx* const* ctxs, int32_t nctx,
                                       const double* const* params, const int64_t* m,
                                       int32_t out_kind, void* const* outs,
                                       uint32_t* const* flags, double* const* rho,
                                       sas_multi_plan** plan);

/* Enqueue the plan on `stream`: a counter reset and one persistent launch.
 * use_graph != 0: the first call captures them into a CUDA graph (on a
 * stream of the plan's own) and every call launches that graph on `stream`. */
sas_status subapsnap_multi_plan_launch(sas_multi_plan* plan, int32_t use_graph, void* stream);

/* Release a plan (its graph included).  NULL is a no-op. */
void subapsnap_multi_plan_destroy(sas_multi_plan* plan);

/* Release a context and everything it allocated.  NULL is a no-op. */
void subapsnap_destroy(sas_ctx* ctx);

/* Message for the last failed call on this host thread ("" if none). */
const char* subapsnap_last_error(void);

/* Device status word of a context: 0, or a SAS_* code recorded by a kernel
 * (e.g. SAS_ETIMEOUT from a bounded wait).  Synchronises the context's
 * work on `stream` and clears the word. */
sas_status subapsnap_device_status(sas_ctx* ctx, void* stream);

/* Self-test of the device-side failure path (not in the paper): a kernel waits,
 * through the bounded wait every pipelined kernel of the library uses, on a
 * barrier that nothing arrives on; after `seconds` (0 < seconds <= 2) the
 * wait gives up and records SAS_ETIMEOUT in the context's status word, which
 * this call then reads (synchronising `stream`) and clears.  Returns
 * SAS_ETIMEOUT when the mechanism works; the context stays usable. */
sas_status subapsnap_selftest_wait(sas_ctx* ctx, double seconds, void* stream);

/* Library version string. */
const char* subapsnap_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SUBAPSNAP_H */
