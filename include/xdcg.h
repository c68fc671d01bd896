/*
 * xdcg -- adapted deflated conjugate gradients for XFEM/GFEM crack systems
 * on one GB300 GPU (sm_103a).
 *
 * Solves K u = f, K symmetric positive definite (Section 2.4, Eq.
 * linear_system), by conjugate gradients (Algorithm 1) preconditioned by
 * the multiplicative A-DEF2 combination (Section 3.2) of
 *   - subdomain deflation: per box subdomain the six rigid-body modes of
 *     Eq. dcg_deflation_space, plus, in boxes holding jump-enriched nodes,
 *     the six enriched modes of Eqs. dcg_deflation_space_enr_std and
 *     dcg_deflation_space_enr_enr (Section 3.3), and
 *   - block Jacobi over node blocks that include the enriched dofs
 *     (Section 3.4, Eqs. block_jacobi, block_jacobi_enr),
 * started from the initial solution of Algorithm 2 (with u_-1 = 0) and
 * stopped when ||r_i||_2 <= tol ||f||_2 (relative tolerance, Section 4).
 *
 * Conventions shared by every entry point:
 *   - All functions return an xdcg_status; nothing is thrown across the ABI.
 *   - "device" pointers are CUDA global-memory addresses on the device that
 *     is current when xdcg_setup is called; "host" pointers are ordinary
 *     (pageable or pinned) host memory.
 *   - A context is bound to the CUDA stream given at set-up; every call on
 *     it is ordered on that stream.  A context is not thread-safe.
 *   - dof layout: node I owns the contiguous dofs [dof_ptr[I], dof_ptr[I+1]),
 *     ordered [3 standard | 3 jump] or [3 standard | 12 branch]; so every
 *     node block has b_I in {3, 6, 15} dofs.
 */
#ifndef XDCG_H
#define XDCG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct xdcg_ctx xdcg_ctx;   /* opaque; owns all of its device memory */

typedef enum {
    XDCG_OK = 0,
    XDCG_INVALID_ARG = 1,      /* bad pointer, size, index, pattern or option */
    XDCG_NOT_SPD_BLOCK = 2,    /* a node block failed its Cholesky factorisation;
                                  xdcg_setup's bad_index names the node */
    XDCG_COARSE_NOT_SPD = 3,   /* E = Z^T K Z failed its factorisation;
                                  xdcg_setup's bad_index names the coarse pivot */
    XDCG_BREAKDOWN = 4,        /* p^T K p <= 0 or not finite during the iteration */
    XDCG_NO_CONVERGENCE = 5,   /* max_iter reached; u holds the last iterate */
    XDCG_CUDA_ERROR = 6,       /* a CUDA runtime call failed */
    XDCG_OOM = 7,              /* device allocation failed */
    XDCG_TOO_LARGE = 8,        /* the problem needs more than the fixed scratch of
                                  xdcg_spmv_noalloc */
    XDCG_TIMEOUT = 9           /* a kernel's bounded wait on its own asynchronous copies ran
                                  out; the results of that call are invalid and the
                                  context must be destroyed */
} xdcg_status;

enum { XDCG_HOST = 0, XDCG_DEVICE = 1 };       /* memory space of input arrays */
enum { XDCG_FP64 = 0, XDCG_MIXED = 1 };        /* solve precision */
enum { XDCG_BLOCK_JACOBI = 0, XDCG_POINT_JACOBI = 1 };   /* M of Algorithm 3 */

/* Stiffness matrix K in node-blocked CSR, full symmetric storage, FP64.
 * Row I lists the nodes J coupled to I (sharing an element), sorted, with
 * the diagonal J = I present; block (I, J) is b_I x b_J, row-major, at
 * val[val_ptr[p] .. val_ptr[p+1]).  The pattern and the values must be
 * symmetric (checked at set-up to 1e-12 relative).  Read-only; copied at
 * set-up, so the caller may free it when xdcg_setup returns. */
typedef struct {
    int32_t n_nodes;
    const int32_t *dof_ptr;    /* [n_nodes + 1], dof_ptr[0] = 0 */
    const int32_t *row_ptr;    /* [n_nodes + 1] */
    const int32_t *col;        /* [row_ptr[n_nodes]] */
    const int64_t *val_ptr;    /* [row_ptr[n_nodes] + 1] */
    const double *val;         /* [val_ptr[row_ptr[n_nodes]]] */
    int32_t mem;               /* XDCG_HOST or XDCG_DEVICE, for all six arrays */
} xdcg_matrix;

/* The deflation space Z (Section 3.3), one box subdomain s = sub_of_node[I]
 * per node, in one of two forms.
 *
 * Valued form (values != NULL): Z itself.  Box s owns sub_cols[s] (6 or 12)
 * consecutive coarse columns, boxes in order; node I's block of Z is b_I x
 * sub_cols[sub[I]] doubles, row-major (rows: I's dofs, columns: its box's
 * columns), and the blocks of nodes 0, 1, ... follow one another in values.
 * Z is zero outside each node's own box columns.  coords, hsign, centre and
 * enriched_modes are then ignored and may be NULL.
 *
 * Geometric form (values == NULL): the
 * library builds Z on the device from it: for node I in box s = sub[I] and
 * x = coords[I] - centre[s], the rigid block R(x) of Eq. dcg_deflation_space
 * on I's standard dofs (columns 6 s' .. 6 s' + 5 of box s); if
 * enriched_modes is set and the jump-enriched nodes (b_I = 6) of box s are
 * not all on one line, six more columns holding hsign[I] * R(x) on the
 * standard dofs (Eq. dcg_deflation_space_enr_std), R(x) on the jump dofs
 * (Eq. dcg_deflation_space_enr_enr) and 0 on branch dofs.  hsign[I] is
 * H(x_I) = +-1, the side of the box's crack on which node I lies.  The
 * resulting Z must have full column rank (checked through E). */
typedef struct {
    int32_t n_sub;
    const int32_t *sub_of_node;  /* [n_nodes], values in [0, n_sub) */
    const double *coords;        /* [3 n_nodes], x y z per node */
    const int8_t *hsign;         /* [n_nodes], +1 or -1 */
    const double *centre;        /* [3 n_sub] */
    int32_t enriched_modes;      /* 0: rigid modes only; 1: add enriched modes */
    int32_t mem;                 /* XDCG_HOST or XDCG_DEVICE, for all the arrays */
    const int32_t *sub_cols;     /* valued form: [n_sub] columns of each box, 6 or 12 */
    const double *values;        /* valued form: the node blocks of Z; NULL: geometric form */
} xdcg_deflation;

/* Block-Jacobi blocks chosen by the caller (Section 3.4, Eqs. block_jacobi,
 * block_jacobi_enr): M is the block diagonal of K over these blocks.  The
 * paper's own choice is one block per subdomain, enriched dofs included;
 * number the dofs subdomain by subdomain and give each subdomain's range.
 * Block b is the contiguous dof range [dof_ptr[b], dof_ptr[b+1]) of K's
 * numbering; every boundary must fall between two nodes, and no block may
 * hold more than XDCG_MAX_BLOCK_DOFS dofs (else XDCG_INVALID_ARG).  At set-up
 * each block's part of K is gathered as a dense matrix and inverted in FP64;
 * every iteration applies the inverses as dense products (in FP64, or for
 * MIXED in FP32 on the block-scaled system).  A block whose inversion meets a
 * pivot <= 1e-14 times its largest diagonal entry gives XDCG_NOT_SPD_BLOCK
 * with bad_index = the block.  Passing NULL selects one block per node
 * (3, 6 or 15 dofs, factored by Cholesky), the library's default.  Not
 * combinable with XDCG_POINT_JACOBI or with a batched context (max_batch >
 * 0).  Copied at set-up. */
#define XDCG_MAX_BLOCK_DOFS 4096
typedef struct {
    int32_t n_blocks;
    const int32_t *dof_ptr;    /* [n_blocks + 1], dof_ptr[0] = 0, dof_ptr[n_blocks] = n */
    int32_t mem;               /* XDCG_HOST or XDCG_DEVICE */
} xdcg_blocks;

typedef struct {
    double tol;              /* relative residual target, default 1e-8 */
    int32_t max_iter;        /* total CG iterations (inner ones for MIXED), default 10000 */
    int32_t precision;       /* XDCG_FP64 (default) or XDCG_MIXED */
    double inner_tol;        /* MIXED: residual replacement each time the FP32 recursive
                                residual has dropped by this factor, default 1e-3 */
    int32_t max_outer;       /* MIXED: residual replacements (FP64 residual evaluations),
                                default 30.  When two replacements in a row shorten the FP64
                                residual by less than 2x (the FP32 recurrence's rounding floor,
                                near 1e-11 relative on large systems), when the FP32 run stalls
                                (200 iterations without its residual dropping by 10 %: the
                                FP32 rounding of K~ hides what is left to resolve), or when
                                max_outer is reached, the solve folds in the FP32 correction and
                                finishes with the FP64 iteration from its current u (Algorithm
                                2 with u_-1 = u) */
    int32_t time_spmv;       /* 1: bracket every SpMV launch of the iteration by CUDA events;
                                2: bracket every kernel of the iteration (t_phase_ms) */
    int32_t jacobi;          /* XDCG_BLOCK_JACOBI (default): one block per node (3/6/15 dofs,
                                Eqs. block_jacobi, block_jacobi_enr); XDCG_POINT_JACOBI: the
                                diagonal of K, the paper's comparison preconditioner
                                (Section 4.1).  MIXED scales K~ by the same factors; with point
                                Jacobi its FP32 run can break down (XDCG_BREAKDOWN) */
    int32_t record_history;  /* 1: keep ||r_i|| / ||f|| of every iteration of FP64 solves
                                (xdcg_get_history); default 0 */
    int32_t max_batch;       /* MIXED: right-hand sides one xdcg_solve_batch call may take
                                together (0..8; 0 = no batched buffers), default 0 */
    int32_t coarse_fp64;     /* MIXED: 1 applies E^-1 in FP64 inside the FP32 iteration (an FP64
                                GEMV whose result is rounded to FP32); default 0: an FP32 copy
                                of E^-1 (half the bytes; A-DEF2 tolerates the inexact coarse
                                solve).  Single right-hand-side solves; the batched FP32
                                iteration of xdcg_solve_batch uses the FP32 copy.  The FP64
                                path always applies E^-1 in FP64 */
    double wait_s;           /* limit of every bounded device wait on the SpMV's own bulk copies,
                                in seconds, default 2.  A wait that runs out ends the call with
                                XDCG_TIMEOUT after the copies in flight have landed (their own
                                limit, 0.1 s, is fixed).  0 gives up at the first wait: it
                                exists to exercise that status, not for use */
    int32_t autotune;        /* 1: set-up times every compiled pipeline shape of the SpMV (steps
                                per bulk-copy stage, stages per warp, blocks per SM) on this
                                matrix and keeps the fastest (info.spmv_shape_*); a few ms.
                                Default 0: the default shape (FP32 5, FP64 0).  Two contexts
                                with different shapes may round the fused dot differently */
    int32_t graph;           /* 1: the loops of the solves enqueue their iterations as CUDA
                                graphs: a batch of 8 iterations of xdcg_solve / xdcg_solve_x0
                                (FP64, and MIXED's FP32 iteration) is recorded by stream capture
                                once per context (on a private stream of the context, so the
                                context's own stream may be the legacy default stream) and
                                replayed with one graph launch per batch; xdcg_solve_batch and
                                xdcg_solve_systems (the first context's option) record the 2
                                iterations of each tick, again whenever the set of systems still
                                iterating changes.  The graphs hold the same launches in the same
                                order, with the same programmatic ordering between them, so the
                                results are the same bits.  Ignored with time_spmv (its events
                                sit between the kernels).  Default 0 */
    int32_t spmv_shape_fp32; /* >= 0: the FP32 SpMV runs this pipeline shape (xdcg_info_t lists
                                them), whatever autotune found; -1 (default): the default
                                shape (5), or the autotuner's pick.  XDCG_INVALID_ARG beyond
                                the last shape */
    int32_t spmv_shape_fp64; /* the same for the FP64 SpMV (default shape 0) */
} xdcg_options;

typedef struct {
    int32_t iterations;          /* loop bodies run (products K p), summed over cycles */
    int32_t outer_cycles;        /* MIXED: FP64 residual evaluations; FP64: 1 */
    double rel_res_recursive;    /* FP64: last recursive ||r|| / ||f||; MIXED: ||L^-1 r|| / ||f||
                                    of the FP32 recursive residual before the last replacement */
    double rel_res_true;         /* ||f - K u|| / ||f|| in FP64 after the solve */
    double t_solve_ms;           /* CUDA-event time of the solve on the context stream */
    int32_t bad_index;           /* failing node or coarse pivot, else -1 */
    int32_t n_spmv_timed;        /* SpMV launches timed (time_spmv) */
    double t_spmv_ms;            /* their summed CUDA-event time */
    int64_t n_launches;          /* kernels launched by this call */
    int32_t n_phase_timed;       /* iterations whose kernels were timed (time_spmv = 2) */
    double t_phase_ms[5];        /* their summed CUDA-event time per kernel of the iteration:
                                    FP64: SpMV, update, restriction, coarse solve, prolongation;
                                    MIXED: SpMV, restriction+update, coarse solve, prolongation */
    int32_t n_fp64_iterations;   /* MIXED: iterations of the FP64 finish (included in
                                    iterations), 0 when the FP32 cycles alone met tol */
    int32_t n_graph_launches;    /* graph launches made by this call (xdcg_options.graph); the
                                    kernels they ran are counted in n_launches */
} xdcg_result;

typedef struct {
    int64_t n;                   /* dofs */
    int32_t n_nodes;
    int32_t k;                   /* coarse dimension */
    int64_t nnz;                 /* scalar nonzeros of K */
    int64_t nnzb3;               /* 3x3 blocks of the chunked SpMV layout */
    int64_t spmv_bytes_fp64;     /* bytes one FP64 SpMV reads and writes in the library's
                                    chunked layout (one index per 3x3 chunk block, row data,
                                    p read once, q written once; slot padding excluded) */
    int64_t spmv_bytes_fp32;     /* the same for the FP32 SpMV */
    int64_t iter_bytes_fp64;     /* algorithmic bytes of one FP64 iteration */
    int64_t iter_bytes_fp32;     /* algorithmic bytes of one FP32 inner iteration (MIXED) */
    double t_setup_ms;           /* wall time of xdcg_setup */
    int64_t restrict_bytes_fp32; /* ... of its restriction + update kernel (MIXED) */
    int64_t coarse_bytes_fp32;   /* ... of its coarse solve kernel (MIXED) */
    int64_t prolong_bytes_fp32;  /* ... of its prolongation kernel (MIXED) */
    int64_t nnzb;                /* node blocks of K (entries of the caller's block CSR) */
    int64_t spmv_alg_bytes_fp64; /* bytes one product q = K p must move at least, counted on
                                    the node-blocked matrix: 8 nnz + 4 nnzb + 4 (n_nodes + 1)
                                    + 2 * 8 n (values, block indices, row pointers, p read
                                    once, q written once) */
    int64_t spmv_alg_bytes_fp32; /* the same with 4-byte values and vectors */
    int64_t block_entries;       /* caller blocks: sum of their squared sizes (entries of the
                                    dense inverses applied per iteration); 0 for node blocks */
    double t_setup_phase_ms[8];  /* wall time of xdcg_setup's phases: validation; host layout
                                    (integer maps); uploads and SpMV value gathers; node-block
                                    factors, W and E; E^-1; the FP32 level (MIXED); caller
                                    blocks; work vectors */
    int32_t reused_node_factors; /* xdcg_setup_update: node-block factors carried over */
    int32_t reused_coarse_inverse; /* xdcg_setup_update: 1 if E^-1 was carried over */
    int32_t spmv_shape_fp64;     /* SpMV pipeline shape in use (default FP64 0, FP32 5; the
                                    FP32 one for MIXED contexts) */
    int32_t spmv_shape_fp32;
    double spmv_shape_us_fp64[8]; /* autotune: median time of each shape's product, -1 untimed;
                                    FP64 shapes (steps per stage, stages, blocks per SM):
                                    (1,3,3) (1,4,2) (2,2,2) (1,2,4) */
    double spmv_shape_us_fp32[8]; /* FP32 shapes: (2,3,3) (1,4,4) (2,4,2) (1,6,3) (3,3,2), and
                                    the lean kernel's (2,3,3) (1,6,3) (2,2,4): stages that run
                                    across slice boundaries, the copy schedule walked by every
                                    lane, no per-stage record; the same products and, at the
                                    same grid, the same dot */
} xdcg_info_t;

/* Fill *opt with the defaults listed above. */
xdcg_status xdcg_default_options(xdcg_options *opt);

/* Validate K and the deflation description, copy them to the device, lay K
 * out for the SpMV (FP64 and, for MIXED, FP32 copies), factor the node
 * blocks (FP64 Cholesky), build Z, W = K Z and E = Z^T K Z, and invert E in
 * FP64 (MIXED also keeps an FP32 copy of E^-1).  blocks: NULL (one block per
 * node) or the caller's blocks (xdcg_blocks), inverted in FP64.  stream: a
 * cudaStream_t (NULL = legacy default stream).  On error *out is NULL and,
 * if bad_index is not NULL, *bad_index names the failing node or caller
 * block (XDCG_NOT_SPD_BLOCK) or coarse pivot (XDCG_COARSE_NOT_SPD), else -1. */
xdcg_status xdcg_setup(xdcg_ctx **out, const xdcg_matrix *K, const xdcg_deflation *Z,
                       const xdcg_blocks *blocks, const xdcg_options *opt, void *stream,
                       int32_t *bad_index);

/* Set-up for the next crack-front position of a propagation (the paper's
 * crack propagation studies, Section 4: the preconditioner is updated rather
 * than rebuilt from nothing).  Same arguments and result as xdcg_setup, plus
 * prev, a context of the same mesh (the same nodes, in the same order) for
 * the previous front.  The new context is built as by xdcg_setup, except
 * that every node whose dofs and diagonal block of K are unchanged (bitwise)
 * takes its block-Jacobi factor from prev instead of refactoring it (so only
 * the blocks the front changed are factored), and that an unchanged E
 * (bitwise, same k) takes prev's E^-1 instead of inverting it.  The results
 * are bit for bit those of xdcg_setup on the same input.  prev is only read
 * (its stream is synchronised first) and stays valid; destroy it when it is
 * no longer needed.  info.reused_node_factors and info.reused_coarse_inverse
 * say what was carried over. */
xdcg_status xdcg_setup_update(xdcg_ctx **out, const xdcg_ctx *prev, const xdcg_matrix *K,
                              const xdcg_deflation *Z, const xdcg_blocks *blocks,
                              const xdcg_options *opt, void *stream, int32_t *bad_index);

/* Solve K u = f with the options given at set-up, tol overriding opt.tol
 * when > 0.  f, u: caller-owned device arrays of n doubles (may not alias).
 * res may be NULL.  On NO_CONVERGENCE u holds the last iterate. */
xdcg_status xdcg_solve(xdcg_ctx *ctx, const double *f, double *u, double tol, xdcg_result *res);

/* As xdcg_solve, started from the caller's guess: on entry u holds u_-1, and
 * Algorithm 2 gives u_0 = u_-1 + Z E^-1 Z^T (f - K u_-1) (the paper's start
 * with a nonzero u_-1; reusing the previous solution is the paper's stated
 * future work).  The mixed path starts its FP64 solution at u_-1 and its
 * FP32 run on the scaled residual f - K u_-1.  A guess that already meets
 * tol returns it unchanged with 0 iterations.  Iteration counts and the
 * stopping test are as for xdcg_solve. */
xdcg_status xdcg_solve_x0(xdcg_ctx *ctx, const double *f, double *u, double tol,
                          xdcg_result *res);

/* Solve K U_j = F_j for m right-hand sides of the set-up system (several load
 * cases of one crack configuration).  F, U: device arrays of m * n doubles,
 * column j at offset j * n (may not alias).  With MIXED and opt.max_batch >= m
 * the columns run as one batched FP32 iteration: each iteration reads K~, Z~,
 * W~ and E^-1 once for all columns.  Each column advances on its own: when
 * its FP32 recursive residual has dropped by inner_tol (or its p^T K p is not
 * positive, or it reaches max_iter iterations) it is held while the others
 * iterate, its FP32 correction is folded into U_j and its FP64 residual
 * f_j - K U_j replaces the recursive one; it leaves once that residual meets
 * tol (or is not finite: BREAKDOWN with bad_index = j; or after max_outer
 * replacements or at max_iter: NO_CONVERGENCE).  A column's result does not
 * depend on the other columns.  Otherwise (FP64, or max_batch = 0) the
 * columns are solved one after another.  res: NULL or m results, iterations
 * counted per column.  Returns the worst status over the columns. */
xdcg_status xdcg_solve_batch(xdcg_ctx *ctx, const double *F, double *U, int32_t m, double tol,
                             xdcg_result *res);

/* xdcg_solve_batch for several systems at once (the crack fronts of a
 * propagation sweep, Section 4: each front has its own K, Z and
 * preconditioner), run as one batched FP32 iteration: every iteration is one
 * launch per kernel over all systems' blocks, on ctxs[0]'s stream (ordered
 * after the work already queued on the other contexts' streams, and before
 * what is queued on them later).  ctxs: n_sys distinct MIXED contexts on one
 * device, set up with the same max_batch rounding (1..4 or 5..8); F[s], U[s]:
 * device arrays of m[s] * n_s doubles as for xdcg_solve_batch, 1 <= m[s] <=
 * that context's max_batch.  tol <= 0 takes each context's opt.tol.  Every
 * column's result is the same bits as from xdcg_solve_batch on its own
 * context.  res: NULL or sum(m) results, system by system; status: NULL or
 * n_sys statuses.  Contexts must not be used by another thread meanwhile.
 * Returns INVALID_ARG, CUDA_ERROR or TIMEOUT for the call, else the worst
 * system status. */
xdcg_status xdcg_solve_systems(xdcg_ctx *const *ctxs, int32_t n_sys, const double *const *F,
                               double *const *U, const int32_t *m, double tol,
                               xdcg_result *res, xdcg_status *status);

/* As xdcg_solve with host arrays: copies f to the device, solves, copies u
 * back, all on the context stream; returns after u is on the host. */
xdcg_status xdcg_solve_host(xdcg_ctx *ctx, const double *f_host, double *u_host, double tol,
                            xdcg_result *res);

xdcg_status xdcg_get_info(const xdcg_ctx *ctx, xdcg_info_t *info);

/* Recursive relative residuals ||r_i|| / ||f||, i = 0 .. iterations, of the
 * last FP64 solve (the curves of the paper's Section 4.1 residual figure).
 * Needs opt.record_history at set-up (else XDCG_INVALID_ARG).  Writes
 * min(cap, *count) values to out (host) and the number recorded to *count.
 * MIXED solves record nothing (their FP32 recursion lives in a scaled norm). */
xdcg_status xdcg_get_history(xdcg_ctx *ctx, double *out, int32_t cap, int32_t *count);

/* The operator of one solve path applied to x.  XDCG_FP64: y = K x with
 * double arrays.  XDCG_MIXED: y = K~ x with float arrays, where
 * K~ = L^-1 K L^-T is the block-scaled matrix of the FP32 inner solve (L the
 * FP64 Cholesky factors of the node blocks), stored and accumulated in FP32.
 * x, y: device, length n, in the caller's dof numbering (the FP32 operator
 * is stored box by box; x and y are renumbered through the context's FP32
 * work vectors).  If xty is not NULL it receives x^T y (FP64 reduction) on
 * the host. */
xdcg_status xdcg_spmv(xdcg_ctx *ctx, int32_t precision, const void *x, void *y, double *xty);

/* Same result as xdcg_spmv, for callers that cannot allocate device memory
 * at the point of the call: code that runs while another allocator (a
 * framework's caching allocator, or a memory pool sized to the whole device)
 * holds the device memory budget, so that a cudaMalloc would fail; and code
 * on a latency-critical path, where cudaMalloc and cudaFree can synchronise
 * the device and stall its other streams.  The paper has no counterpart;
 * this is a property of the library, not of the method.
 *
 * It allocates nothing.  The SpMV's reduction scratch (block partial sums
 * and its scalar block) lives in one file-scope device array of
 * XDCG_NOALLOC_MAX_BLOCKS doubles plus one scalar block (about 33 KB), which
 * every GPU that loads the library keeps until the process exits.  The
 * first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current, so make that first call
 * before any stream capture.  The device current at the call must be the
 * context's (the one current at xdcg_setup), else XDCG_INVALID_ARG.  All
 * calls share the array, which keeps the last call's contents; each call
 * clears what must start at zero, but calls that overlap on the GPU (other
 * streams, other contexts) race on it.  The XDCG_MIXED product also uses the
 * context's own FP32 work vectors (it renumbers x and y, see xdcg_spmv), so
 * it must not overlap another call on the same context.
 *
 * x, y: device arrays of n values (double for XDCG_FP64, float for
 * XDCG_MIXED, as in xdcg_spmv).  xty_dev: NULL or a device double that
 * receives x^T y.  Asynchronous on the context stream, so the call returns
 * before the product is done and reports no device-side failure itself: if
 * a bounded wait of the product on its own copies ran out (the condition
 * xdcg_spmv reports as XDCG_TIMEOUT), *xty_dev is set to NaN and y is not
 * valid; a caller that must detect this passes xty_dev.  Returns
 * XDCG_TOO_LARGE when the context's SpMV grid exceeds
 * XDCG_NOALLOC_MAX_BLOCKS blocks (the SpMV runs a persistent grid of at
 * most a few blocks per SM, so this does not happen on current GPUs). */
#define XDCG_NOALLOC_MAX_BLOCKS 4096
xdcg_status xdcg_spmv_noalloc(xdcg_ctx *ctx, int32_t precision, const void *x, void *y,
                              double *xty_dev);

/* z = A-DEF2 preconditioner applied to r (Algorithm 3, one merged coarse
 * solve), FP64.  r, z: device, length n. */
xdcg_status xdcg_precond(xdcg_ctx *ctx, const double *r, double *z);

/* Sensitivity of a loss J(u), u = K^-1 f, to each element's Young's modulus
 * (for differentiable use of the solver; not part of the paper's method).
 * With K = sum_e E_e Khat_e, Khat_e the element stiffness for E = 1 at fixed
 * Poisson ratio, the adjoint of the solve gives
 *     out[e] = dJ/dE_e = -lam_e^T Khat_e u_e,   K lam = dJ/du
 * (lam: a second solve on this context; K is symmetric).
 *
 * n_el elements.  Element e's local dofs are elem_dofs[elem_dof_ptr[e] ..
 * elem_dof_ptr[e+1]) (at most 120: 8 nodes x 15 dofs), each the global dof
 * (0 <= d < n) of that local dof or -1 for an eliminated one (its u and lam
 * entries count as 0).  Its d_e x d_e row-major Khat_e starts at
 * elem_mat[elem_mat_off[e]] and must lie within the mat_len doubles of
 * elem_mat; elements may share a matrix.  u, lam: length n.  All arrays are
 * device arrays owned by the caller; out (device, n_el doubles) is written
 * in FP64, each element's sum in a fixed order.
 *
 * Synchronises the context stream.  XDCG_INVALID_ARG for a null pointer, a
 * negative n_el, a global dof >= n, more than 120 local dofs or a matrix
 * outside elem_mat; the offending elements' out entries are then NaN and the
 * others are valid. */
xdcg_status xdcg_element_sensitivity(xdcg_ctx *ctx, int64_t n_el, const int64_t *elem_dof_ptr,
                                     const int32_t *elem_dofs, const int64_t *elem_mat_off,
                                     const double *elem_mat, int64_t mat_len, const double *u,
                                     const double *lam, double *out);

/* Gradient of a loss J(u), u = K^-1 f, with respect to K's stored entries
 * (for differentiable use of the solver; not part of the paper's method):
 *     dJ/dK_ij = -lam_i u_j,   K lam = dJ/du
 * (lam: a second solve on this context, K being symmetric), sampled at the
 * positions K stores: out[val_ptr[p] + a * b_J + b] receives -lam[dof_ptr[I]
 * + a] * u[dof_ptr[J] + b] for the stored block p = (I, J).  The per-element
 * modulus sensitivities of xdcg_element_sensitivity are the contractions
 * <dJ/dK, Khat_e>.
 *
 * K: the context's matrix structure as device arrays (mem = XDCG_DEVICE,
 * n_nodes as at set-up; val is not read).  lam, u: device, length n.  out:
 * device, val_ptr[nnzb] doubles, written in FP64 (each entry one product).
 * Synchronises the context stream.  XDCG_INVALID_ARG for a null pointer, a
 * host-memory structure or a node count other than the context's, and for
 * a stored block whose column, dofs or value range are out of bounds (that
 * block's entries are left unwritten). */
xdcg_status xdcg_stiffness_gradient(xdcg_ctx *ctx, const xdcg_matrix *K, const double *lam,
                                    const double *u, double *out);

/* Copy the coarse matrix E (k x k, row-major, FP64) to host memory E_host. */
xdcg_status xdcg_coarse_matrix(xdcg_ctx *ctx, double *E_host);

xdcg_status xdcg_destroy(xdcg_ctx *ctx);

const char *xdcg_status_string(xdcg_status s);

#ifdef __cplusplus
}
#endif
#endif /* XDCG_H */
