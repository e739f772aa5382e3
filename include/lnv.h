/*
 * lnv.h -- C ABI of liblnv, a GB300 (sm_103a) library for the range-truncated
 * block-sparse products of the LNV density-matrix method (Bowler & Miyazaki,
 * "Calculations on millions of atoms with DFT", Sec. 2).
 *
 * Method (Sec. 2): the density matrix in the support-function basis is
 * K = 3LSL - 2LSLSL (Eq. 3) with S the overlap matrix (Eq. 2) and L the
 * auxiliary density matrix, truncated as L_ij = 0 for |R_i - R_j| > R_L.  The
 * electron count is N_e = 2 Tr[KS] (Sec. 2, condition 2); the band energy at
 * fixed H is E = 2 Tr[KH]; the minimisation over L uses
 *     dE/dL = 6(SLH + HLS) - 4(SLSLH + SLHLS + HLSLS)
 * restricted to L's range.  The main cost is sparse matrix multiplication
 * (Sec. 3), which this library runs on the GPU.
 *
 * Conventions shared by every call:
 *  - Matrices are block-CSR over atoms: one NSF x NSF block per stored atom
 *    pair, blocks row-major, a matrix's values one contiguous array of
 *    nnzb * NSF * NSF elements in the block order of its pattern.
 *  - A pattern holds row_ptr (int64, n+1), col (int32, nnzb, ascending inside
 *    each row) and, for symmetric patterns, a transpose map tr (int64, nnzb):
 *    tr[p] is the position of block (j, i) when p holds block (i, j).
 *  - Range patterns keep block (i, j) iff d_ij^2 < R^2, with d the
 *    minimum-image distance in an orthorhombic periodic cell, summed as
 *    ((dx*dx)+(dy*dy))+(dz*dz) in IEEE FP64 without fused multiply-adds.
 *  - "_dev" pointers are device memory on the context's device; "_host"
 *    pointers are host memory.  Value arrays are caller-owned; patterns,
 *    plans and systems are library-owned opaque handles.  Device value
 *    arrays start on a 16-byte boundary (as cudaMalloc's do): the kernels
 *    move blocks in 16-byte pieces.
 *  - Every call is asynchronous on the context's stream unless it says it
 *    synchronises.  Calls that build handles (pattern, plan, system)
 *    allocate device memory and synchronise the stream.
 *  - No exception crosses the ABI.  A call returns LNV_OK or a negative
 *    status; lnv_last_error() gives the calling thread's last message.
 *    On error no output is guaranteed and handles stay valid.
 */
#ifndef LNV_H
#define LNV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int lnv_status;
#define LNV_OK 0
#define LNV_ERR_ARG (-1)         /* null pointer, bad size, bad enum        */
#define LNV_ERR_CUDA (-2)        /* a CUDA runtime call or launch failed    */
#define LNV_ERR_OOM (-3)         /* device allocation failed                */
#define LNV_ERR_PATTERN (-4)     /* patterns of different sizes, unsorted or
                                    non-symmetric where symmetry is needed  */
#define LNV_ERR_UNSUPPORTED (-5) /* NSF or precision not built, row too long */
#define LNV_ERR_TIMEOUT (-6)     /* a bounded device-side wait ran out (see
                                    lnv_ctx_device_status)                  */

/* Arithmetic of a call.  LNV_FP64: values, products and sums in FP64.
 * LNV_FP32: values stored and multiplied in FP32 with FP32 accumulation of
 * the block products; traces, energies and the gradient combination are
 * accumulated in FP64 from the FP32 operands. */
typedef enum { LNV_FP64 = 0, LNV_FP32 = 1 } lnv_prec;

/* Operand flags of lnv_plan_product: use the block transpose of A or B,
 * (A^T)_ik = (A_ki)^T, read through the pattern's transpose map. */
#define LNV_TRANS_A 1
#define LNV_TRANS_B 2
#define LNV_SYM_C 4   /* the product is symmetric: form one triangle, mirror the other */

typedef struct lnv_ctx lnv_ctx;
typedef struct lnv_pattern lnv_pattern;
typedef struct lnv_plan lnv_plan;
typedef struct lnv_system lnv_system;

/* ---- context ---------------------------------------------------------- */

/* Bind a context to CUDA device `device` and the caller's stream
 * (a cudaStream_t, may be NULL for the legacy default stream; the stream
 * stays owned by the caller). */
lnv_status lnv_ctx_create(int device, void *cuda_stream, lnv_ctx **out);
lnv_status lnv_ctx_set_stream(lnv_ctx *ctx, void *cuda_stream);
lnv_status lnv_ctx_destroy(lnv_ctx *ctx);
/* Last error message of the calling thread ("" if none).  Valid until the
 * thread's next failing call. */
const char *lnv_last_error(void);
/* Library version string, static storage. */
const char *lnv_version(void);
/* Kernels this library has launched in this process so far (all threads). */
int64_t lnv_launch_count(void);

/* Device-side status of the context.  The tensor-core product kernel (kernel
 * 9 below) synchronises its warps with barriers whose waits are bounded in
 * time: a wait that runs out (which only a fault elsewhere, e.g. a kernel
 * killed mid-way, can cause) makes the kernel drain its in-flight work, free
 * its tensor memory and exit, with its outputs undefined, and raises the
 * context's status word.  lnv_ctx_device_status synchronises the context
 * stream, returns LNV_ERR_TIMEOUT if the word was raised since the last call
 * (and clears it), else LNV_OK.  lnv_ctx_set_wait_limit sets the limit of one
 * wait in nanoseconds (default 1 s; > 0). */
lnv_status lnv_ctx_device_status(lnv_ctx *ctx);
lnv_status lnv_ctx_set_wait_limit(lnv_ctx *ctx, uint64_t ns);
/* Measured rate of the fused multiply-add pipe of the context's GPU in the
 * given precision (TFLOP/s, 2 flop per FMA): eight independent FMA chains per
 * thread, eight 256-thread CTAs per SM, best of three timed launches.  The
 * SIMT block products (Sec. 3: the main load is sparse matrix
 * multiplication) are bound by this pipe; it is the measured denominator of
 * their rooflines beside the nominal one.  Allocates a small buffer and
 * synchronises. */
lnv_status lnv_probe_fma_rate(lnv_ctx *ctx, lnv_prec prec, double *tflops);
/* Exercise the bounded-wait path: one CTA waits on a barrier that nothing
 * completes, gives up after the context's wait limit and raises the status
 * word (no fault, no trap).  Asynchronous; read the result with
 * lnv_ctx_device_status. */
lnv_status lnv_debug_expire_wait(lnv_ctx *ctx);

/* ---- a0: range patterns (Sec. 2, locality of L and of the products) ---- */

/* Build {(i, j): d_ij^2 < cutoff^2} for n_atoms positions pos_dev[n][3]
 * (FP64, Angstrom) in the periodic box cell_host[3].  Positions may lie
 * outside the box; the minimum image is taken of the raw difference.  Uses a
 * cell list, so the cost is linear in n_atoms at fixed density.  Rows are
 * sorted, the diagonal is present, the transpose map is filled.  Fails with
 * LNV_ERR_UNSUPPORTED if a row exceeds 16384 blocks.  Synchronises. */
lnv_status lnv_pattern_build(lnv_ctx *ctx, const double *pos_dev, int64_t n_atoms,
                             const double *cell_host, double cutoff, lnv_pattern **out);

/* Same for n_seg independent systems concatenated along the atom index:
 * system s owns atoms [seg_off_host[s], seg_off_host[s+1]) and the box
 * cells_host[3s..3s+2]; no block couples two systems.  The result is the
 * block-diagonal union, used for batched evaluation. */
lnv_status lnv_pattern_build_batched(lnv_ctx *ctx, const double *pos_dev, int n_seg,
                                     const int64_t *seg_off_host, const double *cells_host,
                                     double cutoff, lnv_pattern **out);

/* Adopt a caller-built pattern (copied).  Columns must be ascending inside
 * each row and in [0, n); otherwise LNV_ERR_PATTERN.  The transpose map is
 * built when the pattern is symmetric (else tr entries are -1).
 * Synchronises. */
lnv_status lnv_pattern_from_csr(lnv_ctx *ctx, int64_t n, const int64_t *row_ptr_dev,
                                const int32_t *col_dev, lnv_pattern **out);

/* Borrowed views of a pattern's device arrays (valid until destroy). */
lnv_status lnv_pattern_info(const lnv_pattern *p, int64_t *n, int64_t *nnzb,
                            const int64_t **row_ptr_dev, const int32_t **col_dev,
                            const int64_t **tr_dev, int *symmetric);
lnv_status lnv_pattern_destroy(lnv_pattern *p);
/* Carry block values from one pattern onto another of the same atoms (e.g.
 * L of an earlier geometry onto the pattern of the next one, to start the
 * next minimisation from it): block (i, j) of `to` takes block (i, j) of
 * `from`, zeros where `from` has none.  from_vals_dev and to_vals_dev are
 * device arrays in `prec` with NSF x NSF blocks; they must not alias.
 * Asynchronous on the context stream; LNV_ERR_PATTERN if the atom counts
 * differ. */
lnv_status lnv_pattern_remap(lnv_ctx *ctx, const lnv_pattern *from, const lnv_pattern *to, int nsf,
                             lnv_prec prec, const void *from_vals_dev, void *to_vals_dev);

/* ---- a1-a3, a5, a6: masked block products (Sec. 2 operation (i)) ----- */

/* Plan C = mask_C(op(A) op(B)): for each block (i, j) of C's pattern,
 * C_ij = sum_k op(A)_ik op(B)_kj; nothing outside C's pattern is formed.
 * flags: LNV_TRANS_A / LNV_TRANS_B (needs a symmetric pattern).
 * LNV_SYM_C declares the product symmetric (as S L S is for symmetric S and
 * L; C's pattern must be symmetric, else LNV_ERR_PATTERN): the kernels that
 * can skip work form only C's blocks with col >= row, and every element below
 * the diagonal of the full matrix is then set to its mirror element (blocks
 * (i, j), j < i, to the transpose of block (j, i)), so the result is exactly
 * symmetric.  The caller vouches for the symmetry: the lower triangle is not
 * computed.  The plan chooses its kernel from the patterns' symbolic work
 * counts (see lnv_plan_info).  The patterns must outlive the plan.
 * Synchronises. */
lnv_status lnv_plan_product(lnv_ctx *ctx, const lnv_pattern *A, const lnv_pattern *B,
                            const lnv_pattern *C, int flags, lnv_plan **out);
/* Symbolic counts of a plan: block triples (i, k, j) that contribute, and
 * the kernel chosen: 0 push (shared-memory row accumulator), 1 pull with a
 * binary search of B's row k per output, 2 pull walking B's row j
 * (merge-join; needs a symmetric B pattern), 3 row groups of 4 atoms with a
 * 16-bit position table of op(B), 4 row groups with per-column hit lists,
 * 5 row groups with the table, per-warp lists of the k's its columns hit and
 * a cp.async shared-memory ring of op(B) blocks (FP32 values, NSF = 4; other
 * cases run kernel 3), 6 row groups on tensor cores (mma.sync TF32 with
 * a hi/lo split of both operands, FP32 accumulation; FP32 values, NSF = 4;
 * other cases run kernel 3), 7 listed triples: per block of C the stored
 * (op(A)_ik, op(B)_kj) pairs, k ascending, listed once per plan (NSF = 4;
 * other NSF run kernel 0), 8 kernel 5 with warp slices of half the width (8
 * output columns per warp for two fused products, 16 for one): a warp lists
 * only the k's its columns hit, and groups with few columns give more warps
 * (other cases run kernel 3), 9 row groups of 8 atoms as dense tiles on the
 * tcgen05 tensor cores: C_g^T = op(B)^T op(A)_g^T with 128-row tiles of 32
 * output columns j, op(B) rows gathered into tensor memory, op(A) in shared
 * memory, every operand split into TF32 high and low parts (hi*hi + hi*lo +
 * lo*hi, FP32 accumulation: FP32-level accuracy); needs op(B) = B^T (plans
 * without LNV_TRANS_B fail with LNV_ERR_UNSUPPORTED); FP32 values with NSF =
 * 4 (other cases run kernel 0), 10 the same for 9 x 9 blocks: row groups of
 * 7 atoms (N = 63 of 64), 128-row tiles of 14 output columns (M = 126 of
 * 128), K in stages of 8 k-atoms; either op(B); FP32 values with NSF = 9
 * (other cases run kernel 0), 11 kernel 9's 8-row groups and tcgen05
 * pipeline taken one 128-row tile (32 output columns) at a time over only
 * the k's at which one of the tile's columns holds op(B)_kj, for the tables
 * that are sparse as a whole but dense per tile (T = SX, U = SY); either
 * op(B); a symmetric first output is formed on the tiles of its upper part
 * and mirrored; FP32 values with NSF = 4 (other cases run kernel 0), 12
 * and 13 the single-pass forms of 9 and 11: operands rounded to TF32 (round
 * to nearest), one MMA per K step, FP32 accumulation, no low parts; their
 * error (about 1e-4 relative) misses the FP32-level bound, so the
 * autotuner never picks them: they measure the precision trade-off.
 * Kernels 9-13 need value arrays 16-byte aligned (else LNV_ERR_UNSUPPORTED
 * from the multiply).
 * The default is 3 when at least half of the table's candidates hit, else 4,
 * when the tables fit a third of the free device memory. */
lnv_status lnv_plan_info(const lnv_plan *plan, int64_t *triples, int *mode);
/* Number of product kernels (0 .. LNV_NUM_KERNELS - 1). */
#define LNV_NUM_KERNELS 14
/* Select the kernel of a plan (0..13 as above); 0-11 give the same result up
 * to rounding order (12 and 13 to single-pass TF32 accuracy).  Kernels 3-13
 * build their tables on first selection
 * (allocates, synchronises).  LNV_ERR_UNSUPPORTED if the kernel cannot run
 * this plan. */
lnv_status lnv_plan_set_kernel(lnv_ctx *ctx, lnv_plan *plan, int kernel);
lnv_status lnv_plan_destroy(lnv_plan *plan);

/* Numeric product on the context stream (Sec. 2 operation (i), the sparse
 * matrix multiplication of Sec. 3): C = alpha mask_C(op(A) op(B)) + beta C.
 * A_dev, B_dev, C_dev are value arrays in `prec` (double or float) with
 * NSF x NSF blocks, NSF in {1, 2, 4, 9}.  beta = 0: C is overwritten (its
 * old values are not read, NaN included) and nothing is allocated.  beta !=
 * 0: the product is formed in a scratch buffer the context keeps (allocated
 * or grown on the first such call, which then synchronises; later calls of
 * the same size allocate nothing) and combined with C elementwise in FP64
 * arithmetic, rounded to the value precision. */
lnv_status lnv_bsr_multiply(lnv_ctx *ctx, const lnv_plan *plan, int nsf, lnv_prec prec,
                            const void *A_dev, const void *B_dev, void *C_dev, double alpha,
                            double beta);

/* ---- a4: traces (N_e = 2 Tr[KS], Sec. 2; E = 2 Tr[KH]) ----------------- */

/* out_dev[0] = Tr[A B] = sum_ij <A_ij, (B_ji)^T>, A and B on the same
 * symmetric pattern, accumulated in FP64 in a fixed order (deterministic).
 * `scratch_dev` holds n doubles (per-row partial sums). */
lnv_status lnv_trace_product(lnv_ctx *ctx, const lnv_pattern *P, int nsf, lnv_prec prec,
                             const void *A_dev, const void *B_dev, double *scratch_dev,
                             double *out_dev);

/* Tr[A B] like lnv_trace_product, for callers that cannot allocate device
 * memory or pass scratch: for example code held to a fixed device-memory
 * budget by its own pool, or an interface with no room for a scratch
 * buffer.  The paper has no counterpart; this is a library convenience.
 * The per-row partial sums live in a static device array of 262144 doubles
 * (2 MiB) that every GPU loading the library keeps until exit; patterns with
 * more rows fail with LNV_ERR_UNSUPPORTED.  The call allocates nothing.  It
 * looks the array's device address up (cudaGetSymbolAddress) on every call
 * made outside a stream capture, so the address stays right after a
 * cudaDeviceReset, and keeps the last one for calls made during a capture:
 * make one call on the device before capturing.  All calls on a device share
 * the array, so calls whose kernels overlap on the GPU race; serialise them.
 * Every row's partial sum is written before it is read, so the array needs no
 * clearing between calls. */
lnv_status lnv_trace_product_noalloc(lnv_ctx *ctx, const lnv_pattern *P, int nsf,
                                     lnv_prec prec, const void *A_dev, const void *B_dev,
                                     double *out_dev);

/* ---- a1-a7 fused: LNV energy, electron count and gradient -------------- */

/* A system: positions, S and H on the range-r_sh pattern, L on the range-r_l
 * pattern, plus every intermediate pattern and product plan of the
 * evaluation.  n_seg > 1 batches independent systems (block-diagonal,
 * seg_off_host / cells_host as in lnv_pattern_build_batched); n_seg = 1
 * takes seg_off_host = NULL and one box.  Synchronises. */
lnv_status lnv_system_create(lnv_ctx *ctx, int nsf, lnv_prec prec, const double *pos_dev,
                             int64_t n_atoms, int n_seg, const int64_t *seg_off_host,
                             const double *cells_host, double r_sh, double r_l,
                             lnv_system **out);
/* As lnv_system_create, with the intermediates truncated below their exact
 * ranges (Sec. 2: the matrices' sparsity is an approximation; the paper notes
 * that carefully constructed sparse-matrix methods make the cost linear):
 * X = LS, Y = LH and Z = LSLS kept within r_x (exact: r_l + r_sh), T = SLS
 * and U = SLH within r_t (exact: r_l + 2 r_sh).  r_x <= 0 or r_t <= 0 selects
 * the exact range; otherwise r_l <= r_x <= r_l + r_sh and r_l <= r_t <=
 * r_l + 2 r_sh (LNV_ERR_ARG outside).  Every product is still formed exactly
 * on its truncated pattern, in the same association as the exact plan, so E,
 * N_e and G become approximations whose error vanishes at the exact ranges. */
lnv_status lnv_system_create_truncated(lnv_ctx *ctx, int nsf, lnv_prec prec, const double *pos_dev,
                                       int64_t n_atoms, int n_seg, const int64_t *seg_off_host,
                                       const double *cells_host, double r_sh, double r_l, double r_x,
                                       double r_t, lnv_system **out);
/* Patterns of S/H and of L (borrowed). */
lnv_status lnv_system_patterns(const lnv_system *sys, const lnv_pattern **sh,
                               const lnv_pattern **l);
/* Device bytes of workspace one evaluation needs (intermediates X, Y, T, U,
 * Z, W, Q and trace partials). */
lnv_status lnv_system_workspace_size(const lnv_system *sys, int with_grad, size_t *bytes);
/* Block size, precision and number of independent systems of a system
 * (any output may be NULL). */
lnv_status lnv_system_info(const lnv_system *sys, int *nsf, lnv_prec *prec, int *n_seg);
/* Algorithmic block triples of one evaluation (sum over its products).  T =
 * SLS is symmetric when X is exact (r_x = r_l + r_sh): only the triples of
 * its upper triangle (col >= row) count, as only those are formed. */
lnv_status lnv_system_triples(const lnv_system *sys, int with_grad, int64_t *triples);
/* The same per stage (XY, TU, Z, traces, Q, W, G; 7 values, the TU entry
 * counting both T and U). */
lnv_status lnv_system_stage_triples(const lnv_system *sys, int64_t *t7);
lnv_status lnv_system_destroy(lnv_system *sys);

/* Kernel of each product stage (XY, TU, Z, -, Q, W, -; -1 for non-products),
 * in the numbering of lnv_plan_info. */
lnv_status lnv_system_stage_kernels(const lnv_system *sys, int *k7);

/* Select the kernel of one product stage (0 XY, 1 TU, 2 Z, 4 Q, 5 W) by
 * hand, in the numbering of lnv_plan_info; as lnv_plan_set_kernel. */
lnv_status lnv_system_set_stage_kernel(lnv_ctx *ctx, lnv_system *sys, int stage, int kernel);

/* T = SLS is symmetric when X is exact (r_x = r_l + r_sh).  Such a system
 * forms by default only T's upper triangle (col >= row) where the TU kernel
 * can skip the rest (push, row groups), then mirrors the lower triangle.
 * on = 0 forms T whole instead (faster when the kernel's cost does not follow
 * its multiply-adds); on = 1 on a system with truncated X is
 * LNV_ERR_UNSUPPORTED.  A change rebuilds the TU plan's row-group tables,
 * whose column order follows the setting (synchronises).  lnv_system_mirror
 * reports the setting. */
lnv_status lnv_system_set_mirror(lnv_ctx *ctx, lnv_system *sys, int on);
lnv_status lnv_system_mirror(const lnv_system *sys, int *on);

/* Autotuner: runs one evaluation on S, H, L, then times every applicable
 * kernel of each product stage (XY, TU, Z, Q, W) on those intermediates
 * (reps launches each, CUDA events on the context stream) and keeps the
 * fastest; for TU each kernel with and without the mirror of T.  ms_out (5 x LNV_NUM_KERNELS values, may be NULL) receives the
 * time of every (stage, kernel) pair tried, -1 for kernels that do not
 * apply.  Allocates and synchronises; results do not change beyond rounding
 * order.  Uses the system's own workspace. */
lnv_status lnv_system_autotune(lnv_ctx *ctx, lnv_system *sys, const void *S_dev, const void *H_dev,
                               const void *L_dev, int reps, double *ms_out);

/* Stage timing: with enable != 0, lnv_energy_grad records CUDA events on the
 * context stream around its stages XY, TU, Z, traces, Q, W, G.
 * lnv_system_stage_ms waits for the last evaluation's final event and writes
 * the 7 stage durations in milliseconds (0 for stages that did not run). */
lnv_status lnv_system_profile(lnv_system *sys, int enable);
lnv_status lnv_system_stage_ms(lnv_system *sys, double *ms7);

/* One evaluation (Sec. 2, Eq. 3).  S_dev, H_dev (on the r_sh pattern) and
 * L_dev (on the r_l pattern) are value arrays in the system's precision.
 * All three must be symmetric (block (j, i) the transpose of block (i, j)),
 * as the overlap and Hamiltonian of real basis functions are and as L is
 * taken, so that K is a symmetric density matrix.  The
 * evaluation relies on it (T = SLS is formed on one triangle and mirrored, and
 * Z = L T is read as L T^T); the results for a non-symmetric L are
 * undefined.
 * Writes, per system s, out_dev[6 s + 0..5] = {E, N_e, Tr[LSLH],
 * Tr[LSLSLH], Tr[LSLS], Tr[LSLSLS]} (FP64); when G_dev is not NULL, dE/dL
 * = 6(SLH + HLS) - 4(SLSLH + SLHLS + HLSLS) on L's pattern; when GN_dev is
 * not NULL, dN_e/dL = 12(SLS - SLSLS) on L's pattern (both in the system's
 * precision, FP64-combined, every stored entry of L independent).
 * Workspace: ws_dev of ws_bytes >= lnv_system_workspace_size(with_grad =
 * G_dev != NULL), or NULL to use a buffer the system allocates on first use
 * and keeps.  Asynchronous on the context stream. */
lnv_status lnv_energy_grad(lnv_ctx *ctx, lnv_system *sys, const void *S_dev,
                           const void *H_dev, const void *L_dev, double *out_dev,
                           void *G_dev, void *GN_dev, void *ws_dev, size_t ws_bytes);

/* The same evaluation (Sec. 2, Eq. 3) from host memory: S_host, H_host and
 * L_host (the layouts and symmetry of lnv_energy_grad) are copied to device
 * buffers the system allocates on first use and keeps, the evaluation runs
 * on the context stream with the system's own workspace, and out_host[6 s +
 * 0..5] and, when G_host is not NULL, dE/dL are copied back.  Synchronises:
 * the host arrays are read and written before the call returns.  Pinned
 * (page-locked) host memory copies fastest; any host memory is accepted.
 * Errors as lnv_energy_grad; LNV_ERR_OOM when the device buffers cannot be
 * allocated. */
lnv_status lnv_energy_grad_host(lnv_ctx *ctx, lnv_system *sys, const void *S_host, const void *H_host,
                                const void *L_host, double *out_host, void *G_host);

/* ------------------------------------------------------------------ minimisation
 * The search for the ground state around the evaluation: vary L on its
 * pattern to minimise the energy with the electron count set (Sec. 2,
 * conditions 2 and 3, Eq. 3).  The paper prints no algorithm; lnv_minimize
 * takes the usual one.  The count is set by a chemical potential mu: the
 * function minimised is Omega = E - mu N_e = 2 Tr[K (H - mu S)], the band
 * energy of H - mu S.  Polak-Ribiere conjugate gradients run on L's stored
 * entries, and each line search is exact: Omega(L + tD) is a cubic in t,
 * fitted from its value and slope at 0 and two more evaluations.
 *
 * Vector kernels on value arrays of n elements in `prec` (device pointers):
 * out = a x + b y (x or y is not read when its factor is 0; out may alias x
 * or y), and *out_dev = x . y summed in FP64 in a fixed order (one device
 * double; uses a scratch buffer the context keeps).  Asynchronous. */
lnv_status lnv_vec_axpby(lnv_ctx *ctx, lnv_prec prec, int64_t n, double a, const void *x_dev,
                         double b, const void *y_dev, void *out_dev);
lnv_status lnv_vec_dot(lnv_ctx *ctx, lnv_prec prec, int64_t n, const void *x_dev, const void *y_dev,
                       double *out_dev);
/* Minimise Omega = E - mu N_e over L_dev (updated in place; the system's
 * precision, L's pattern) for one system (n_seg = 1, else
 * LNV_ERR_UNSUPPORTED), until the root-mean-square of dOmega/dL is <= tol,
 * a line search finds no step, or after max_iter iterations.  With mu in a
 * gap of the spectrum of (H, S) and no truncation the minimum is the
 * projector on the states below mu.  hist_host (may be NULL) receives up to
 * max_iter + 1 rows of {Omega, E, N_e, rms of dOmega/dL, previous step
 * length}; *iters_out the iterations done (rows written = iters + 1).
 * Allocates five L-sized arrays and one of S's size for the call;
 * synchronises. */
lnv_status lnv_minimize(lnv_ctx *ctx, lnv_system *sys, const void *S_dev, const void *H_dev,
                        void *L_dev, double mu, int max_iter, double tol, double *hist_host,
                        int *iters_out);

#ifdef __cplusplus
}
#endif
#endif /* LNV_H */
