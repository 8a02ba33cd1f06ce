/*
 * sppc.h - C ABI of the GB300 (sm_103a) SPPC eigensolver library (libsppc.so).
 *
 * SPPC (Subspace Projection with Perturbative Corrections) computes the k lowest
 * eigenpairs of a large sparse symmetric matrix H split as H = H0 + V with
 * H0 = diag(H0_hat, 0), H0_hat the leading n1 x n1 block (the small configuration
 * space) and V = H - H0 (paper Sec. 2, Eqs. split/split2; Algorithm 2).  Each order
 * p adds k perturbative correction vectors Psi^(p) (Eq. exp_seq2), computed from
 * small shifted solves in the leading block (Eqs. bl_diag, sm_first, sm_lin_proj),
 * to an orthonormal basis Q (Eqs. blkGS, QR, Qp) and extracts Ritz pairs from the
 * projected matrix Q^T H Q (Eqs. tilde_H, proj), costing k products with H per
 * order (Sec. 4.3, Eqs. avoid_SpMV2, HPsip).
 *
 * Conventions (every entry point):
 *  - Returns an sppc_status; never aborts.  On failure sppc_last_error(h) (or
 *    sppc_last_error(NULL) for failures before a handle exists) gives a message.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Work is enqueued on it; calls that return host results synchronise it.
 *  - Device buffers passed in are owned by the caller and only read or written
 *    during the call.  Host buffers likewise.  The library owns everything it
 *    allocates (matrix copy, basis Q, W = HQ, scratch) and frees it in
 *    sppc_destroy.
 *  - Dense blocks are row-major n x ncols with a leading dimension (elements).
 *  - All values crossing the ABI are IEEE FP64.  Internally the library stores
 *    matrix values and vectors by default as double-float pairs (two fp32 whose
 *    sum carries ~48 significant bits) and computes with error-free fp32
 *    transformations, because native FP64 throughput on this GPU is ~1/70 of
 *    FP32; opts.precision = -1 selects native FP64 storage and arithmetic
 *    (DFMA) for the whole path instead.
 *  - A handle is not thread-safe: one host thread at a time.
 */
#ifndef SPPC_H_
#define SPPC_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sppc_ctx* sppc_handle;

typedef enum {
  SPPC_OK = 0,
  SPPC_ERR_ARG = 1,           /* bad argument (null pointer, size, k range, ...) */
  SPPC_ERR_NOT_SYMMETRIC = 2, /* H != H^T (only when opts.check_symmetry) */
  SPPC_ERR_LEVELS = 3,        /* level_offsets malformed or n1 not a level boundary */
  SPPC_ERR_OOM = 4,           /* device or host allocation failed */
  SPPC_ERR_CUDA = 5,          /* a CUDA call failed (message has the CUDA error) */
  SPPC_ERR_BREAKDOWN = 6,     /* Cholesky breakdown / rank loss in orthogonalisation */
  SPPC_ERR_MINRES = 7,        /* a small solve hit its iteration limit */
  SPPC_ERR_TIMEOUT = 8,       /* a bounded device-side wait gave up */
  SPPC_NOT_CONVERGED = 9,     /* p_max reached; outputs hold the last order's pairs */
  SPPC_ERR_STATE = 10,        /* call out of sequence (e.g. correct before start) */
  SPPC_ERR_NAN = 11           /* a NaN/Inf appeared in the input or iteration */
} sppc_status;

/* Caller-owned CSR matrix, only read by sppc_create.  Rows must have strictly
 * increasing column indices; the diagonal may be stored or absent. */
typedef struct {
  int64_t n;              /* rows = columns */
  int64_t nnz;            /* stored entries */
  const int64_t* row_ptr; /* n+1 offsets, row_ptr[0] = 0, row_ptr[n] = nnz */
  const int32_t* col;     /* nnz column indices in [0, n) */
  const double* val;      /* nnz values */
  int32_t on_device;      /* 0: host pointers, 1: device pointers */
} sppc_csr;

typedef struct {
  int32_t p_max;          /* maximum correction order (default 15; paper Sec. 4.3, 6) */
  double tol;             /* scaled residual ||Hz - theta z|| / |theta| (Eq. rrn), default 1e-6 */
  double minres_tol;      /* small solve: stop at ||r|| <= minres_tol ||b1|| (default 1e-12) */
  int32_t minres_maxit;   /* small solve iteration cap (default 20*n1, at most 200000) */
  double small_tol;       /* small eigensolve residual tolerance, relative to ||H0_hat|| (1e-12) */
  int32_t small_block;    /* vectors in the small eigensolve (default 2k, >= k+1) */
  double degeneracy_tol;  /* psi_hat_j also deflated for column k if |E_j - E_k| <= tol*||H0_hat|| (1e-10) */
  int32_t check_symmetry; /* 1: verify H == H^T bit for bit at create (default 0) */
  uint64_t seed;          /* seed of the small eigensolve's start block (default 0) */
  int32_t timing;         /* 1: time kernels with CUDA events into sppc_stats (default 0) */
  int64_t spmm_chunk_cols; /* SpMM column tile: 0 (default) = 1310720 columns, 80 MB of an 8-column
                              double-float block (keeps the gathered rows of X in L2), untiled with
                              precision -1 when an 8-column X fits in L2 (the FP64 product is then
                              DFMA-bound), -1 = untiled, > 0 = that many
                              columns (at most 255 tiles), -2 = autotuned at create (untiled and
                              2.6M/1.31M/655k/328k-column tiles timed on two 8-column products each;
                              the fastest kept, see sppc_spmm_tiling) */
  int32_t hybrid;          /* 0: plain SPPC (Alg. 2, default); 1: after switch_order SPPC orders continue
                              by block extension with preconditioned Ritz residuals (Sec. 5: SPPC
                              combined with a second eigensolver started from its approximations);
                              2: after switch_order orders, per-pair RMM-DIIS from the Ritz vectors
                              (Sec. 6: DIIS over the last min(8, p_max + 1) iterates, Jacobi-
                              preconditioned step; needs precision 0; Z returns each pair's vector) */
  int32_t switch_order;    /* SPPC orders before the continuation (default 15, Sec. 6) */
  int32_t hybrid_maxit;    /* continuation steps, k SpMVs each (default 1000) */
  int32_t precond;         /* 1: residual_j / (diag(H) - theta_j) (default); 0: none (block Krylov);
                              2: as 1, then the leading rows replaced by precond_iters MINRES steps on
                              P (H_L - theta_j) P t = P r_j[:nL], H_L the leading block (H0_hat, or more
                              levels by precond_levels), P deflating the Ritz vector's leading part
                              (shifted block-diagonal preconditioner, Sec. 5) */
  double precond_clamp;    /* denominators of the preconditioner clamped to |.| >= this (1e-2) */
  int32_t hybrid_blocks;   /* continuation basis limit in blocks of k vectors before a thick restart
                              to 2k Ritz vectors (default 0 = p_max + 1; at least 3) */
  int32_t spmm_kernel;     /* SpMM kernel for 8-column blocks: 1 = rows of X gathered into registers
                              (default), 0 = gathered into shared memory by the tensor memory
                              accelerator; both give identical results (other widths always use 1) */
  int32_t reorth;          /* continuation's block Gram-Schmidt: 0 = second projection only when the
                              first kept less than half of some column's norm (default), 1 = always
                              twice (SPPC orders always project twice: Eq. blkGS applied twice) */
  int32_t precond_iters;   /* MINRES steps of the leading-block preconditioner (precond 2; default 20) */
  int32_t precision;       /* 0: FP64-quality path in double-float (default).  -1: native FP64: H's
                              values, every vector and coefficient stored as IEEE doubles, every
                              product, Gram, update, MINRES step and the projected eigensolve's
                              Householder part in FP64 arithmetic (DFMA); not with hybrid = 2 or
                              the proposal; spmm_kernel 0 falls back to 1.  1: mixed precision: H's values
                              rounded to FP32 everywhere; the products with H during the solve in FP32
                              (X rounded to FP32, FP32 accumulation); Gram, CholeskyQR2, the projected
                              eigensolve and MINRES in double-float; at the end the Ritz values and
                              residuals are recomputed with double-float products (Rayleigh
                              quotients) and the continuation goes on with double-float products
                              if they miss tol.  2: as 1 with BF16 values: off-diagonal values
                              rounded to FP32 and then to BF16 (nearest, ties to even), the
                              diagonal to FP32, everywhere; the FP32 products read the BF16 values
                              (2 bytes per entry) and the FP32 diagonal.  1 and 2 need k in {3, 4, 7, 8}. */
  int32_t proposal;        /* 0: none (default).  1: learned correction proposal (not in the paper):
                              each continuation step extends the basis by the network's block
                              g_j = (r_j / (diag(H) - theta_j)) (1 + m_j) instead of the plain
                              preconditioned residuals (leading n1 rows still from the precond 2
                              solve); kept iff the largest scaled residual drops, else the step is
                              redone with the plain block.  Needs hybrid = 1, precond 1 or 2 and
                              sppc_set_proposal before the solve. */
  int32_t precond_levels;  /* precond 2: the MINRES-solved leading block spans levels [0, precond_levels)
                              (rows [0, max(n1, level_offsets[precond_levels])); default 1 = the
                              small space H0_hat).  More levels: a stronger preconditioner (fewer
                              continuation steps) for more work per MINRES step. */
  int32_t minres_deflate;  /* 1 (default): the small solves of Eq. sm_lin_proj take the solution's
                              components along the small eigensolve's other eigenvectors in closed
                              form and run MINRES on the remainder (same solution, fewer
                              iterations; 8-column blocks, k = 7 or 8); 0: plain MINRES */
  int32_t small_degree;    /* degree of the Chebyshev filter in the small eigensolve (default 30; halved
                              and redone when the filtered block is too ill-conditioned for
                              CholeskyQR) */
  double switch_stall;     /* hybrid: also leave SPPC (before switch_order) at the first order p >= 2
                              where some eigenpair's scaled residual exceeds switch_stall times its
                              value at order p - 1 (Sec. 6: switch when a residual starts to
                              stagnate); 0 (default) = off */
  int32_t minres_ctas;     /* cap on the CTAs of the small-space MINRES kernel (0 = one per 64 rows,
                              at most the resident limit; default) */
  int32_t spin_cap;        /* polls after which a grid barrier of the persistent MINRES kernel gives
                              up: the kernel raises its error flag, every CTA leaves, and the call
                              returns SPPC_ERR_TIMEOUT (0 = default, 4,194,304 polls, a few seconds;
                              a tiny value forces that path, for tests).  With spmm_kernel = 0 it
                              also bounds each mbarrier wait of the TMA-gather SpMM to spin_cap - 1
                              non-blocking tests (1 = give up at the first wait; 0 = about a second
                              of clock): the warp gives up, waits for its copies in flight, raises
                              the handle's flag, and sppc_spmm_host (or the next correction order)
                              returns SPPC_ERR_TIMEOUT */
  int32_t value_rounding;  /* with precision 0 or -1: 1 rounds H's values to FP32, 2 rounds them as
                              precision 2 does (diagonal FP32, other entries BF16), before anything
                              else; the solve then runs on that matrix in the chosen format (the
                              reference of the mixed-precision runs).  0 (default): as given;
                              ignored with precision 1 or 2, which round this way themselves */
  int32_t minres_fp32;     /* 1: the small solves of Eq. sm_lin_proj by iterative refinement: each sweep
                              runs MINRES in FP32 (to minres_fp32_tol relative, or 2,000 iterations)
                              on the current residual, adds its solution and recomputes the residual
                              b1 - (H0_hat - E) x in double-float, until ||r|| <= minres_tol ||b1||
                              (at most 8 sweeps).  Not with precision -1.  0 (default): MINRES in the
                              value format */
  double minres_fp32_tol;  /* FP32 MINRES stopping tolerance of one refinement sweep (default 1e-6) */
  int32_t tensor_gram;     /* 1: the Gram products against the orthonormal basis (the projections of
                              Eq. blkGS and the border Q^T W of Eq. proj) run on the tensor cores:
                              entries cut into 62-bit fixed point, eight 8-bit digits each, exact
                              FP16 digit products summed exactly, combined in FP64 (error below one
                              FP64 rounding of the largest terms; see sppc_block_gram).  Used where
                              the block width is 8 (k = 7 or 8); a basis entry that is not finite
                              makes the solve return SPPC_ERR_NAN.  0 (default): CUDA cores */
  int32_t sell_sigma;      /* rows of the windows inside which H's SELL-16 layout sorts the rows of a
                              level by decreasing entry count (less padding against more reordering of
                              the X gathers): a multiple of 16 in [16, 1024]; 0 (default) = 1024; -2 =
                              autotuned at create (64, 256 and 1024 built and timed on two 8-column
                              products each at the column tile in use, the fastest kept; see
                              sppc_sell_sigma) */
} sppc_opts;

typedef struct {
  int32_t orders;            /* correction orders run (p of the last Rayleigh-Ritz) */
  int32_t converged;         /* 1 if every scaled residual <= tol */
  int64_t spmv_h;            /* products of H with one vector (k per order, k(P+1) total) */
  int64_t spmv_h11;          /* products of H0_hat with one vector (small eigensolve + MINRES) */
  int64_t minres_iters;      /* total MINRES iterations (max over the k columns, summed over orders) */
  int64_t small_eig_iters;   /* Chebyshev filter degree summed over outer iterations */
  int32_t spmm_launches;     /* launches of the big SpMM kernel */
  double spmm_ms;            /* summed CUDA-event time of the big SpMM launches (timing=1) */
  double minres_ms;          /* small solves (timing=1) */
  double small_eig_ms;       /* small eigensolve (timing=1) */
  double dense_ms;           /* Gram / orthogonalisation / Rayleigh-Ritz kernels (timing=1) */
  double total_ms;           /* whole call (timing=1) */
  int32_t refine_steps;      /* continuation steps run (hybrid) */
  int32_t restarts;          /* thick restarts of the continuation */
  int32_t switched_at;       /* SPPC order at which the continuation started */
  int32_t reorth_passes;     /* appended blocks that needed the second Gram-Schmidt pass */
  int32_t refine_df;         /* mixed precision: continuation steps run with double-float products
                                after the FP32 phase */
  int32_t proposals_tried;   /* learned proposal: continuation steps that tried the network's block */
  int32_t proposals_kept;    /* ... and kept it (the largest scaled residual dropped) */
  int32_t small_filter_retries; /* small eigensolve: filters redone with half the degree after a
                                   CholeskyQR breakdown of the filtered block */
} sppc_stats;

/* Fill `o` with the defaults listed above. */
void sppc_default_opts(sppc_opts* o);

/* Build a handle for H (paper Sec. 2: H0_hat = leading n1 x n1 block).
 *  level_offsets[0..n_levels]: 0 = off_0 < off_1 < ... < off_n = n, the row ranges
 *    of the hierarchy levels (Sec. 1: leading submatrix = smaller N_max space);
 *  n1 must equal level_offsets[j] for some j >= 1 (Sec. 6.1: H0_hat is the whole
 *    smaller configuration space), else SPPC_ERR_LEVELS;
 *  1 <= k <= 8 eigenpairs, k < n1.
 * Copies and reformats H into library-owned device memory (level-blocked SELL-16
 * layout plus a separate copy of H0_hat).  Allocates the basis for opts.p_max
 * orders up front (SPPC_ERR_OOM if it does not fit).  opts may be NULL. */
sppc_status sppc_create(const sppc_csr* H, const int64_t* level_offsets, int32_t n_levels, int64_t n1,
                        int32_t k, const sppc_opts* opts, void* stream, sppc_handle* out);

/* Y = H X for ncols <= 8 columns (the SpMM of Sec. 4.2, "k SpMVs in Hq^(p)").
 * X, Y: caller-owned DEVICE buffers, row-major n x ncols, leading dims ldx, ldy
 * (>= ncols).  X and Y must not overlap. */
sppc_status sppc_spmm(sppc_handle h, const double* X, int64_t ldx, double* Y, int64_t ldy, int32_t ncols,
                      void* stream);

/* Y = H X like sppc_spmm, but the call allocates no device memory: for callers
 * that cannot allocate while they multiply (a framework that owns all device
 * memory through its own allocator and budget, a service that forbids growth
 * after start-up, a loop that must not pay the synchronisation cudaMalloc or
 * cudaFree may imply).  The paper has no counterpart; this is a property of the
 * library.  Scratch (double-float copies of X and of the result) lives in a fixed
 * 32 MiB device array that every GPU loading the library holds until exit; a call
 * needs 2*n*kp*8 bytes of it (kp = ncols rounded up to even), so n*kp must be
 * <= 2,097,152, else SPPC_ERR_ARG (nothing is launched).  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress) with that
 * device current; make that first call before any stream capture.  All calls
 * share the array and it keeps the last call's contents: calls whose work
 * overlaps on the GPU race on it.  X, Y: caller-owned DEVICE buffers as in
 * sppc_spmm. */
sppc_status sppc_spmm_noalloc(sppc_handle h, const double* X, int64_t ldx, double* Y, int64_t ldy, int32_t ncols,
                              void* stream);

/* Same product with HOST buffers: copies X to the device, multiplies, copies Y back
 * (synchronises the stream). */
sppc_status sppc_spmm_host(sppc_handle h, const double* X, int64_t ldx, double* Y, int64_t ldy, int32_t ncols,
                           void* stream);

/* Algorithm 2 steps 1-4: the k lowest eigenpairs (E^(0), psi_hat) of H0_hat
 * (Eq. EP_small), Q^(0) = Psi^(0), W = H Q^(0), projected matrix and Ritz pairs.
 * theta, resid: optional host arrays of k (NULL to skip). */
sppc_status sppc_start(sppc_handle h, double* theta, double* resid, void* stream);

/* One correction order p -> p+1 (Alg. 2 loop body, first half): right-hand side
 * of Eq. exp_seq2 from the recycled H Psi^(p-1) (Eqs. avoid_SpMV2, HPsip), the
 * correction energies E^(p) (Eq. exp_seq), x2 = -b2/E^(0) (Eq. sm_first), the k
 * deflated small solves by MINRES (Eq. sm_lin_proj), block Gram-Schmidt (Eq.
 * blkGS; a second pass when the first removed more than half of some column's
 * norm) and CholeskyQR2 (Eq. QR), appending q^(p) to Q (Eq. Qp). */
sppc_status sppc_correct(sppc_handle h, void* stream);

/* Rayleigh-Ritz after sppc_correct (second half of the loop body): W_p = H q^(p)
 * (the k SpMVs of the order), bordered projected matrix (Eq. proj), its k lowest
 * eigenpairs, Ritz vectors and scaled residuals (Eq. rrn).  theta, resid: optional
 * host arrays of k. */
sppc_status sppc_rayleigh_ritz(sppc_handle h, double* theta, double* resid, void* stream);

/* Algorithm 2 end to end: start, then correct + rayleigh_ritz until every scaled
 * residual <= tol or p_max orders (switch_order orders when opts.hybrid, followed
 * by sppc_refine_step until converged or hybrid_maxit steps, or by per-pair
 * RMM-DIIS when opts.hybrid = 2).  Each order's Rayleigh-Ritz step runs beside
 * the next order's correction on a second stream the handle owns; that stream
 * is joined to `stream` before the call returns.  Results equal the step-by-step
 * calls.  Outputs (any may be NULL):
 *   theta[k], resid[k]: host arrays;
 *   Z: caller-owned DEVICE buffer n x k (ldz >= k), the Ritz vectors (each
 *      pair's own iterate after RMM-DIIS);
 *   stats: host struct.
 * tol <= 0 or p_max < 0 take the handle's options.  Returns SPPC_NOT_CONVERGED
 * (with the last order's pairs filled in) when p_max is reached first. */
sppc_status sppc_solve(sppc_handle h, double tol, int32_t p_max, double* theta, double* Z, int64_t ldz,
                       double* resid, sppc_stats* stats, void* stream);

/* One continuation step (after at least one Rayleigh-Ritz step): extend the basis
 * by the k Ritz residuals of the current pairs, divided by diag(H) - theta_j when
 * opts.precond (block Davidson; block Krylov otherwise; with precond 2 the leading
 * rows come from the deflated leading-block solve), orthogonalised against
 * the basis (Eq. blkGS twice, CholeskyQR2); k SpMVs; Rayleigh-Ritz.  When the
 * basis holds opts.hybrid_blocks blocks it first restarts from the 2k lowest
 * Ritz vectors.
 * After the first step sppc_correct is no longer allowed.  theta, resid: optional
 * host arrays of k. */
sppc_status sppc_refine_step(sppc_handle h, double* theta, double* resid, void* stream);

/* Per-step record of the last solve: E^(p) (k values), sine of the angle between
 * Psi_j^(p) and M^(p-1) after orthogonalisation (k values; Sec. 6.2), Ritz values
 * and scaled residuals after order p (k values each), MINRES iterations per column.
 * Steps 0..orders are SPPC orders; continuation steps follow (E and MINRES counts
 * zero, angle of the appended residual block).  Any output may be NULL. */
sppc_status sppc_order_info(sppc_handle h, int32_t p, double* E, double* angle, double* theta, double* resid,
                            int32_t* minres_iters);

/* Current statistics of the handle (cumulative since sppc_start). */
sppc_status sppc_get_stats(sppc_handle h, sppc_stats* stats);

/* Copies of internal state for tests (host buffers, FP64):
 *   which = 0: psi_hat, n1 x k;   1: Q, n x m (m = k * (orders+1));   2: W = H Q, n x m;
 *           3: projected matrix, m x m;   4: Psi^(p) of the last order, n x k;
 *           5: E^(0), k;   6: the learned proposal's block of the last continuation step,
 *           n x k;   7: the plain preconditioned block of that step, n x k (its leading n1
 *           rows from the precond 2 solve; after sppc_proposal_samples: the raw residuals);
 *           8: the block the last continuation step appended to the basis, before its
 *           orthogonalisation, n x k (hybrid = 1; SPPC_ERR_STATE before the first step).
 * `count` is the number of doubles the buffer holds; returns SPPC_ERR_ARG if too small. */
sppc_status sppc_get_state(sppc_handle h, int32_t which, double* out, int64_t count);

/* Integer layout of the device matrix copy, for bit-exact checks.  Host buffers:
 *   slice_ptr[n_slices+1] (int64), slice_rows[16*n_slices] (int32, -1 = padding row),
 *   h11 same for the leading block (one column chunk), n_chunks and
 *   chunk_slice[n_chunks+1] (first slice of each column chunk of H).
 * Query sizes with NULL buffers. */
sppc_status sppc_get_layout(sppc_handle h, int64_t* n_slices, int64_t* slice_ptr, int32_t* slice_rows,
                            int64_t* n11_slices, int64_t* h11_slice_ptr, int32_t* h11_slice_rows, int32_t* n_chunks,
                            int64_t* chunk_slice);

/* The nev lowest eigenpairs of a small dense symmetric matrix: the projected
 * eigensolve of the Rayleigh-Ritz step (Alg. 2; Eqs. tilde_H, rrn) on its own.
 * S: device, m x m row-major with leading dimension lds (symmetrised as
 * (S + S^T)/2), 1 <= m <= 144; theta: device, nev values ascending; V: device,
 * m x nev row-major with leading dimension ldv >= nev, orthonormal columns.
 * 1 <= nev <= min(16, m).  flags: 0 = Householder tridiagonalisation and
 * back-transformation in double-float (the default path's form), 1 = in FP64
 * (the native FP64 path's); other bits SPPC_ERR_ARG.  One launch of a cluster
 * of 8 CTAs; Sturm-count brackets, inverse iteration (FP32 steps, then FP64).
 * Asynchronous on `stream`; SPPC_ERR_ARG on bad sizes.  All buffers are
 * caller-owned. */
sppc_status sppc_small_syev(const double* S, int32_t m, int32_t lds, int32_t nev, double* theta, double* V,
                            int32_t ldv, int32_t flags, void* stream);

/* The block Gram product of block Gram-Schmidt (Eq. blkGS) and of the border of
 * the projected matrix (Eq. proj), as the solve computes it:
 *   G[(8a + i) * 8 + j] = sum_{r < n} A_a[r][i] B[r][j],
 * A: device, nblocks (1 .. 40) blocks of n x 8 row-major FP64, block a at A + 8 a n;
 * B: device, n x 8 row-major FP64 (A and B may be NULL when n = 0); G: device,
 * 8 nblocks x 8 row-major FP64.
 * flags bit 0 (SPPC_GRAM_TENSOR): on the tensor cores.  Every entry of A must have
 *   |a| < 2 (columns of an orthonormal basis); a = sign X 2^-61 with X < 2^62 an
 *   integer, b = sign X' 2^(f_j - 61) with 2^f_j above |b| in column j (per group
 *   of rows), X and X' cut into eight 8-bit digits; every digit product with
 *   digit levels s + t <= 8 is formed exactly in FP16 x FP16 -> FP32 (sums of 256
 *   rows stay below 2^24) and summed in 64-bit integers; the result is one FP64
 *   rounding per row group away from the exact Gram of the rounded inputs, whose
 *   rounding and dropped levels add at most about 2^-60 |b|_max per row.
 *   Otherwise (bit 0 clear): FP64 or double-float fused multiply-adds.
 * flags bit 1 (SPPC_GRAM_DF): the values are first converted to double-float pairs
 *   and the product runs in that format (FP64 slots otherwise).
 * Synchronises `stream`; temporaries are allocated and freed per call.  SPPC_ERR_ARG
 * on bad sizes, SPPC_ERR_NAN if (tensor cores) an entry of A has |a| >= 2 or a value
 * is not finite, SPPC_ERR_TIMEOUT if a device-side wait gave up. */
#define SPPC_GRAM_TENSOR 1
#define SPPC_GRAM_DF 2
sppc_status sppc_block_gram(const double* A, int32_t nblocks, const double* B, int64_t n, int32_t flags, double* G,
                            void* stream);

/* The block update of block Gram-Schmidt (Eq. blkGS: T = S - Q C) and of the
 * restart's Q Y, as the solve computes it:
 *   Y[r][j] = alpha[j] X[r][j] + sum_a sum_i A_a[r][i] C[(8a + i) * 8 + j],
 * A: device, nblocks (1 .. 40) blocks of n x 8 row-major FP64, block a at A + 8 a n;
 * C: device, 8 nblocks x 8 row-major FP64; alpha: device, 8 FP64 or NULL (1);
 * X: device, n x 8 FP64 or NULL (the term is absent); Y: device, n x 8 FP64, may
 * be X.  flags as for sppc_block_gram: bit 0 (SPPC_GRAM_TENSOR) on the tensor
 * cores (needs |A| < 2; the basis digits of sppc_block_gram, C cut into
 * balanced 8-bit digits with one power of two per column, levels s + t <= 9 of
 * the digit products summed exactly, each output rounded once to FP64), bit 1
 * (SPPC_GRAM_DF) in double-float slots.  Synchronises `stream`; temporaries are
 * allocated per call; SPPC_ERR_ARG on bad sizes, SPPC_ERR_NAN if (tensor cores)
 * an entry of A has |a| >= 2 or a value is not finite, SPPC_ERR_TIMEOUT if a
 * device-side wait gave up. */
sppc_status sppc_block_update(const double* A, int32_t nblocks, const double* C, const double* alpha, const double* X,
                              double* Y, int64_t n, int32_t flags, void* stream);

/* ---- Learned correction proposal (not in the paper; the continuation of
 * Sec. 5-6 extended by a network's block).  Network: per (row i, Ritz pair j),
 * features f = (H_ii, level(i), ||H_i,:||_2, rhat_ij = r_ij sqrt(n)/||r_j||, theta_j,
 * (|H| |rhat_j|)_i), x = (f - mu) / sd, h1 = gelu(W1 x + b1), h2 = gelu(W2 h1 + b2),
 * m = w3 . h2 + b3 (64 hidden units, tanh-form GELU).  Parameters: one FP32
 * vector of SPPC_NET_PARAMS values, W1 (64 x 6 row-major), b1 (64), W2 (64 x 64,
 * W2[o][i] at o*64 + i), b2 (64), w3 (64), b3.  Training minimises
 * mean (rhat (1 + m) - y)^2 with y the exact correction in rhat's scale (see
 * sppc_proposal_samples). */
#define SPPC_NET_PARAMS 4673
#define SPPC_NET_FEATURES 6

/* Install a trained network in h (host arrays: params[SPPC_NET_PARAMS], mu[6],
 * sd[6] > 0), copied into library memory; the solve then uses BF16 inference
 * (weights, inputs and hidden activations rounded to BF16, FP32 sums).
 * SPPC_ERR_ARG on non-finite values or sd <= 0. */
sppc_status sppc_set_proposal(sppc_handle h, const float* params, const float* mu, const float* sd);

/* Training samples from h's current Rayleigh-Ritz state (after sppc_start or
 * sppc_rayleigh_ritz) and exact eigenvectors psi (device, n x k row-major, leading
 * dimension ldpsi >= k, column j the converged eigenvector of pair j): for rows
 * i >= n1 and pairs j < k, sample s = (i - n1) k + j gets raw features F[s*6 + f]
 * (device float), rhat[s] and target y[s] = -(H_ii - theta_j) t_ij sqrt(n)/||r_j||,
 * t_j = psi_j / (z_j^T psi_j) - z_j the exact correction of the Ritz vector z_j
 * (denominator clamped as by precond_clamp); rhat and y are 0 for the pairs with
 * |z_j^T psi_j| < 1/2 (a Ritz vector far from its eigenvector: zero loss and
 * gradient).  *count = (n - n1) k.  Does not change
 * the SPPC state.  Synchronises `stream`. */
sppc_status sppc_proposal_samples(sppc_handle h, const double* psi, int64_t ldpsi, float* F, float* rhat, float* y,
                                  int64_t* count, void* stream);

/* Network output m for `count` standardised samples X (device, count x 6) into
 * out (device); bf16 != 0 selects the solve's BF16 inference, else FP32.
 * Asynchronous on `stream`. */
sppc_status sppc_mlp_forward(const float* params, const float* X, int64_t count, int32_t bf16, float* out,
                             void* stream);

/* FP32 loss L = mean_s (rhat_s (1 + m_s) - y_s)^2 over `count` samples (device
 * X count x 6 standardised, rhat, y) and its gradient grad[SPPC_NET_PARAMS]
 * (device); *loss (device, may be NULL).  Deterministic (fixed summation order).
 * Synchronises `stream`. */
sppc_status sppc_mlp_loss_grad(const float* params, const float* X, const float* rhat, const float* y, int64_t count,
                               float* grad, float* loss, void* stream);

/* One Adam step (Kingma and Ba 2015) with bias correction, step number t >= 1:
 * mom, vel (device, SPPC_NET_PARAMS each) updated in place with params. */
sppc_status sppc_mlp_adam(float* params, float* mom, float* vel, const float* grad, int32_t t, float lr, float beta1,
                          float beta2, float eps, void* stream);

/* One epoch: minibatches of `batch` samples in the order perm[0..nsamples)
 * (device int64, NULL = 0, 1, 2, ...), each a gradient (mean over the batch) and
 * an Adam step; *step counts Adam steps (in/out); *mean_loss (host) = mean of the
 * batch losses.  Synchronises `stream`. */
sppc_status sppc_mlp_train_epoch(float* params, float* mom, float* vel, const float* X, const float* rhat,
                                 const float* y, const int64_t* perm, int64_t nsamples, int32_t batch, int32_t* step,
                                 float lr, float beta1, float beta2, float eps, double* mean_loss, void* stream);

/* Per-feature mean and (population) spread of `count` raw samples F (device,
 * count x 6) into host mean[6], sd[6] (FP64 sums).  Synchronises `stream`. */
sppc_status sppc_feature_moments(const float* F, int64_t count, double* mean, double* sd, void* stream);

/* X = (F - mu) / sd per feature (F, X device count x 6; mu, sd host, sd > 0). */
sppc_status sppc_standardize(const float* F, int64_t count, const float* mu, const float* sd, float* X,
                             void* stream);

/* Solve `count` independent problems (handles created beforehand, each with its
 * own matrix and options) concurrently: `workers` host threads, each with its own
 * non-blocking CUDA stream, take problems in decreasing order of stored entries
 * and run sppc_solve(tol, p_max of the handle) on them; results equal solving
 * them one by one.  Host outputs: theta, resid (count x kmax row-major, row i
 * holds problem i's k values, the rest 0), converged[count], stats[count] (may
 * be NULL).  kmax >= every handle's k.  Returns the first hard error by problem
 * index, else SPPC_NOT_CONVERGED if some problem missed tol, else SPPC_OK.
 * Handles must not be used by other threads during the call. */
sppc_status sppc_solve_batch(sppc_handle* handles, int32_t count, double tol, int32_t workers, int32_t kmax,
                             double* theta, double* resid, int32_t* converged, sppc_stats* stats);

/* The SpMM column tile of h's layout (*chunk_cols: -1 untiled, else columns per
 * tile) and, when it was autotuned (spmm_chunk_cols = -2), the measured ms per
 * 8-column product of each candidate, in the order untiled, 2.6M, 1.31M, 655k,
 * 328k columns (0 for a candidate not tried; candidate_ms[5], may be NULL). */
sppc_status sppc_spmm_tiling(sppc_handle h, int64_t* chunk_cols, double* candidate_ms);

/* The sort window (opts.sell_sigma) of H's SELL-16 layout: *sigma gets the rows
 * of the window in use; with sell_sigma = -2, candidate_ms[3] (may be NULL) the
 * autotuner's ms per 8-column product at windows 64, 256 and 1024 (zeros
 * otherwise).  Host pointers; SPPC_ERR_ARG for a null handle. */
sppc_status sppc_sell_sigma(sppc_handle h, int32_t* sigma, double* candidate_ms);

/* ---- Batched SpMM: Y_i = H_i X_i for `count` handles (1..1024, untiled layouts,
 * i.e. at most 1,310,720 columns each by default) in one persistent launch: the
 * slices of all matrices form one index space that warps drain through a
 * device work queue; results equal per-handle sppc_spmm bit for bit.  The
 * plan captures the launch and the FP64 <-> double-float conversions in a CUDA
 * graph once; each run replays it.  X[i], Y[i]: device FP64, n_i x ncols
 * row-major (ncols in [1, 8], leading dimension ncols), fixed per plan; the
 * handles' SpMM scratch is used, so a handle must not run other calls while a
 * plan that holds it runs. */
typedef struct sppc_batch_plan_s* sppc_batch_plan;
sppc_status sppc_spmm_batch_plan(sppc_handle* handles, int32_t count, const double* const* X, double* const* Y,
                                 int32_t ncols, sppc_batch_plan* out);
sppc_status sppc_spmm_batch_run(sppc_batch_plan plan, void* stream);
sppc_status sppc_spmm_batch_destroy(sppc_batch_plan plan);

/* Release everything the handle owns.  NULL is a no-op. */
sppc_status sppc_destroy(sppc_handle h);

/* Number of CUDA kernel launches this library has issued since it was loaded
 * (all handles, all threads).  Lets a caller count the kernels of a timed region. */
int64_t sppc_kernel_launches(void);

/* Last error message of h (or of the calling thread's last failed create when
 * h == NULL).  The string is owned by the library and valid until the next call. */
const char* sppc_last_error(sppc_handle h);

#ifdef __cplusplus
}
#endif

#endif /* SPPC_H_ */
