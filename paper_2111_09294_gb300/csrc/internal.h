// Internal declarations of the xdcg library: device layouts, the per-solve
// scalar block, and the kernel launchers shared by the translation units.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "xdcg.h"

namespace xdcg {

constexpr int kThreads = 256;      // threads per block of the streaming kernels
constexpr int kWarps = kThreads / 32;
constexpr int kSpmvThreads = 256;  // threads per block of the SpMV (8 persistent warps)
constexpr int kSpmvWarps = kSpmvThreads / 32;

// done flags written by the kernels
enum : int { kRunning = 0, kConverged = 1, kBreakdown = 2, kMaxIter = 3, kFault = 4 };

// what the last block of a reduction does with the reduced value(s)
enum Fin : int {
    kFinAlpha = 0,   // value = p^T q: alpha = rho / pq, its += 1, breakdown test
    kFinRR = 1,      // value = ||r||^2: store rr, converged test against tol2ff
    kFinStore = 2,   // value stored into scratch[slot]
    kFinDefer = 3,   // each block's sum stored at partials[block]; the next kernel adds them
};

// Scalars of one CG run, in device memory.  Written only by the last block
// of a reduction kernel (single writer), read by all later kernels.
struct Scalars {
    double rho;       // r^T z
    double pq;        // p^T K p
    double alpha, beta;
    double rr;        // ||r||^2
    double ry;        // r^T y, y = M^-1 r
    double tol2ff;    // tol^2 ||f||^2
    double scratch[4];
    int its;          // loop bodies run
    int done;         // kRunning / kConverged / kBreakdown / kMaxIter / kFault
    int max_it;
    int fault;        // set by a kernel whose bounded wait ran out
    unsigned int ticket[4];   // last-block tickets, reset by the last block
    double *hist;     // if not null: ||r_i||^2 of iteration i, i < histCap
    int histCap;
    int pad2;
};

// Chunked 3x3 BSR over the chunk rows (3 consecutive dofs) in sliced-ELL
// form with TPR threads per row: a warp holds 32 / TPR rows; at step s,
// lane (rr + (32 / TPR) h) handles slot s * TPR + h of row rr of its slice,
// and the slot's column index and its 9 values sit in 32-wide runs, so
// a slice's steps are one contiguous run of memory (columns at
// slicePtr[sl] + 32 st + lane, value e at 9 slicePtr[sl] + (9 st + e) 32 +
// lane), which the SpMV streams into shared memory with bulk copies.
// Partial rows are combined by shuffles.  Every slice has at least one step.
template <typename T>
struct SellDev {
    int nRows, nSlices;
    const int *row;            // [nRows] chunk row
    const int *len;            // [nRows] blocks in the row
    const long long *slicePtr; // [nSlices + 1] first slot (lane-slot) of each slice
    const int *col;            // [slots] chunk column
    const T *val;              // [9 slots]
};

// Rows whose blocks all couple standard dofs of standard nodes ("S": 27 or
// fewer blocks, natural order, 2 threads per row) and the remaining rows
// ("X": enriched chunks and standard chunks next to enriched nodes, sorted
// by length, 16 threads per row).
constexpr int kTprS = 2;
constexpr int kTprX = 16;
// the SpMV pipeline shape a context runs unless autotuned or pinned
// (spmv_cfg.cuh): FP32 the lean kernel's 2 steps x 3 stages x 3 blocks per
// SM (measured fastest on the 48^3 two-crack system), FP64 1 x 3 x 3
constexpr int kSpmvDefaultShapeF32 = 5;
constexpr int kSpmvDefaultShapeF64 = 0;
constexpr int kXBucket = 8;     // X rows are grouped by len / kXBucket

// ---- batched FP32 iteration (several right-hand sides of one system) ------

constexpr int kMaxBatch = 8;   // right-hand sides per batched solve

// Scalars of a batched FP32 run; column j of every vector is right-hand side j
// (vectors interleaved: entry (dof d, column j) at d * MB + j).  Columns
// advance independently: a column whose recursive residual reaches its
// trigger, whose p^T K p is not positive or that reaches the iteration limit
// is held (pend) with its vectors carried unchanged while the others keep
// iterating, until the host replaces its residual; it leaves (active = 0) at
// a replacement that finds it converged, not finite or out of cycles.  So a
// column's arithmetic does not depend on the other columns, on the other
// systems of a launch over several systems, nor on when its replacement runs.
enum : int { kColOk = 0, kColBad = 1, kColLimit = 2 };
constexpr double kMinGroupDrop2 = 1e-2;   // (1/10)^2: least drop per replacement cycle
struct BatchScalars {
    double rho[kMaxBatch], pq[kMaxBatch], alpha[kMaxBatch], beta[kMaxBatch], rr[kMaxBatch];
    double trig[kMaxBatch];     // column j is held once rr_j <= trig_j
    double rrRep[kMaxBatch];    // rr_j before its last replacement (restart test)
    double scale[kMaxBatch];    // per-column scale of the FP64 <-> FP32 transforms
    double ff[kMaxBatch];       // ||f_j||^2
    double rn2[kMaxBatch];      // ||f_j - K u_j||^2 at column j's last replacement
    double tol, delta2;         // relative tolerance; squared inner drop per cycle
    int active[kMaxBatch];      // 1 until column j leaves
    int pend[kMaxBatch];        // held until its replacement
    int last[kMaxBatch];        // held at the iteration limit: its replacement is its last
    int broken[kMaxBatch];      // p_j^T K p_j <= 0 seen (restart at the replacement)
    int repl[kMaxBatch];        // replaced by the replacement now running (all at the start)
    int itsc[kMaxBatch];        // iterations column j has taken
    int cycles[kMaxBatch];      // replacements of column j
    int outcome[kMaxBatch];     // kColOk, kColBad (not finite), kColLimit (no convergence)
    int its;                    // iterations the system ran: residual buffer its & 1 is current
    int done;                   // kRunning while a column iterates, else kConverged; kFault
    int max_it, max_outer, fault;
    int hold;                   // held for a replacement running on its own stream
    int go;                     // the iteration in progress runs this system (set by the gate)
    int pad;
    unsigned int ticket[4];
};

template <typename T>
struct SpmvDev {
    SellDev<T> S, X;
    int shape;                 // pipeline shape (spmv_cfg.cuh)
    int grid;                  // persistent blocks (kSpmvThreads each)
    const int *warpSlice;      // [grid * kSpmvWarps + 1] slice range of each warp
                               // (S slices, then X slices offset by S.nSlices)
    unsigned long long waitNs; // limit of each launch's bounded waits on its bulk copies
};

// Node-level data: node lists per block size, packed Cholesky factors of
// the node blocks (lower triangle row by row, the diagonal stored as its
// reciprocal), stored structure-of-arrays: entry e of node t of a list at
// L[e * count + t].
template <typename T>
struct NodeDev {
    int nNodes;
    int nStd, nH, nT;
    const int *stdNodes, *hNodes, *tNodes;
    const int *dofStart;      // [nNodes + 1]
    const T *Lstd, *Lh, *Lt;  // 6 / 21 / 120 entries per node
    const int *sub;           // [nNodes] box of each node
    const T *xrel;            // [3 nNodes] coordinates relative to the box centre
    const signed char *hsign; // [nNodes]
    const int *col0;          // [nBox] first coarse column of each box
    const int *menr;          // [nBox] 1 if the box carries enriched modes
};

// Box-level data, node data in box order ("slots": the nodes of box s are
// slots ownPtr[s] .. ownPtr[s+1]-1), and the W entries of each box (nodes
// coupled to the box, W block b_I x M_s row-major at wOff[e]).  Z is
// matrix-free (ownX, ownH) in the FP64 path and explicit (Zt at ownZ[t],
// b_I x M_s row-major) in the block-scaled FP32 path.
template <typename T>
struct BoxDev {
    int nBox;
    const int *col0, *menr;       // first coarse column / enriched-mode flag per box
    const int *ownPtr;            // [nBox + 1]
    const int *ownDof;            // [slots] first dof of the node
    const unsigned char *ownB;    // [slots] dofs of the node (3, 6, 15)
    const signed char *ownH;      // [slots] H(x_I)
    const T *ownX;                // [3 slots] position relative to the box centre
    const long long *ownZ;        // [slots] offset of the explicit Z~ block
    const T *Zt;                  // explicit Z~ (scaled path only)
    const int *extPtr;            // [nBox + 1]
    const int *extDof;            // [entries] first dof of the entry's node
    const unsigned char *extB;    // [entries] dofs of the entry's node
    const long long *wOff;        // [entries]
    const T *W;
};

// ---- launchers (defined in the .cu files) --------------------------------

// Multiprocessors of the current device (queried once per device, then
// cached); grids of the streaming kernels are sized from it.
int device_sm_count();

template <typename T>
void launch_spmv(const SpmvDev<T> &A, const T *x, T *y, const T *b, int residual_mode,
                 double *partials, Scalars *sc, int fin, int slot, cudaStream_t st);
// persistent grid of pipeline shape `shape` (< 0 on a CUDA error), and the
// number of compiled shapes per precision (spmv_cfg.cuh)
template <typename T>
int spmv_persistent_grid(int nSlicesTotal, int shape);
template <typename T>
int spmv_shape_count();

template <typename T>
void launch_update(const NodeDev<T> &N, T *u, T *r, const T *p, const T *q, T *y, int mode,
                   double *partials, Scalars *sc, cudaStream_t st);

// Row-parallel form of the block-scaled FP32 path: per box, the rows of its
// own nodes (Z~, column-major: column c of box s at Z + zBase[s] + c * R_s;
// own row r is dof r of the box-major numbering) and the rows of the nodes
// coupled to it (W~, column-major likewise, each row mapped to its dof).
// The restriction splits each box's own rows followed by its coupled rows
// into balanced units of at most kUnitRows rows (a box near the crack front
// holds several times the rows of an average box; most boxes are one unit).
// When a box has several units, the last to finish (per-box ticket) adds
// their partial sums in unit order.
struct RowBoxDev {
    int nBox;
    const int *col0, *menr;
    const int *ownRowPtr;               // [nBox + 1]: box s owns dofs [ownRowPtr[s], ownRowPtr[s + 1])
    const long long *zBase;             // [nBox]
    const float *Z;
    const int *extRowPtr, *extRowDof;   // [nBox + 1], [coupled rows]
    float *g32;                         // [k] FP32 copy of g for the FP32 coarse solve
    const long long *wBase;             // [nBox]
    const float *W;
    int nUnits;
    const int *unitBox;                 // [nUnits]
    const int *unitOwnBegin, *unitOwnEnd, *unitExtBegin, *unitExtEnd;   // [nUnits] row ranges
    const int *boxUnit;                 // [nBox + 1] first unit of each box
    int nPUnits;                        // prolongation units (own rows, <= kProlongRows)
    const int *pUnitBox, *pUnitBegin, *pUnitEnd;
    double *unitPart;                   // [nUnits * 24] partial sums (scratch)
    unsigned int *boxTicket;            // [nBox] (scratch, kept at zero between launches)
};
constexpr int kUnitRows = 3072;     // own + coupled rows per restriction unit
constexpr int kProlongRows = 512;
constexpr int kUnitRowsBatch = 1024;     // the same for the batched kernels (MB threads per row)
constexpr int kProlongRowsBatch = 64;

void launch_restrict(const BoxDev<double> &B, const double *a, const double *b, int withW,
                     double *g, double *zr, const Scalars *sc, cudaStream_t st);
void launch_prolong(const BoxDev<double> &B, const double *nu, const double *y, double *p,
                    int mode, Scalars *sc, cudaStream_t st);
// mode 0 (iteration): r' = r - alpha q and u += alpha p on own rows (r' written
// to r_next), g = Z~^T r' - W~^T r', zr = Z~^T r', ||r'||^2 with the
// convergence and iteration-cap tests; mode 1 (start): the same without the
// update (alpha = 0, nothing written but g, zr, ||r||^2); mode 2 (Algorithm
// 2): g = Z~^T r only; mode 3 (caller blocks, y = M~^-1 r given): g = Z~^T r
// - W~^T y and zr = Z~^T r, nothing else.
void launch_restrict_update(const RowBoxDev &B, float *u, const float *r_cur, float *r_next,
                            const float *p, const float *q, int mode, double *g, double *zr,
                            double *partials, Scalars *sc, cudaStream_t st,
                            const float *y = nullptr);
void launch_prolong_rows(const RowBoxDev &B, const float *nu32, const float *y, float *p,
                         int mode, Scalars *sc, cudaStream_t st);
// The FP32 iteration's restriction (mode 0) after a product launched with
// kFinDefer: it adds the product's block sums of p^T q (pqPart, pqN of them)
// itself, takes alpha from them and counts the iteration in sc->its.
void launch_restrict_update_deferred(const RowBoxDev &B, float *u, const float *r_cur,
                                     float *r_next, const float *p, const float *q, double *g,
                                     double *zr, double *partials, Scalars *sc,
                                     const float2 *pqPart, int pqN, cudaStream_t st);
void launch_to_colmajor(int nItems, const int *itemBox, const int *rowStart,
                        const unsigned char *itemB, const long long *srcOff,
                        const int *boxRowPtr, const long long *boxBase, const int *menr,
                        const float *src, float *dst, cudaStream_t st);

// nu = E^-1 g (FP64; nu32 optional FP32 copy)
void launch_coarse(const double *Einv, int k, const double *g, const double *zr, double *nu,
                   float *nu32, int mode, double *partials, Scalars *sc, cudaStream_t st);

template <typename T>
void launch_dot(const T *a, const T *b, long long n, double *partials, Scalars *sc, int fin,
                int slot, cudaStream_t st);

// mixed precision helpers

// ---- block-scaled FP32 path (mixed precision) -------------------------------

// FP64 node-block Cholesky factors of all nodes: node I's factor is list
// nodeList[I] (0: 3x3, 1: 6x6, 2: 15x15), position nodeIdx[I] in that list.
struct FacDev {
    const double *L[3];
    int cnt[3];
    const int *nodeList, *nodeIdx;
};

// Z given by value (the valued deflation form): node I's b_I x M_s block
// (M_s = 12 if menr[s] else 6), row-major, at v + off[I].  v == nullptr: Z is
// built from the geometry (Eqs. dcg_deflation_space, dcg_deflation_space_enr_std,
// dcg_deflation_space_enr_enr).
struct ZvalDev {
    const double *v;
    const long long *off;
};

void launch_gather(const int *src, long long n, const double *v, double *out64, float *out32,
                   cudaStream_t st);
void launch_build_Zt(int nSlots, const int *slotNode, const int *dofStart, const int *sub,
                     const double *xrel, const signed char *hsign, const int *menr,
                     const ZvalDev &Zv, const FacDev &F, const long long *zOff, float *Zt,
                     cudaStream_t st);
// node-wise transforms between the caller's dof numbering (nat, which also
// gives the node sizes) and the box-major FP32 numbering: in / ot are the
// numberings of the input / output vector
void launch_fwd_scale(int nNodes, const int *nat, const int *in, const int *ot, const FacDev &F,
                      const double *r, double s, float *out, cudaStream_t st);
void launch_bwd_accum(int nNodes, const int *nat, const int *in, const int *ot, const FacDev &F,
                      const float *ut, double scale, double *u, cudaStream_t st);
void launch_renumber(int nNodes, const int *nat, const int *in, const int *ot, const float *x,
                     float *out, cudaStream_t st);

// ---- batched dense SPD inversion (set-up; dense_inv.cu) ---------------------

// nMat row-major matrices, matrix m (dim[m] x dim[m]) at A + off[m], inverted
// in place.  Tile tables: rowTileOff = prefix of T_m, tileOff = prefix of
// T_m (T_m + 1) / 2 (upper 64 x 64 tiles), T_m = ceil(dim[m] / 64).  Scratch:
// D (nMat x 64 x 64), C (panel rows of matrix m at cOff[m], dim[m] x 64),
// thr (nMat).  A pivot that is not above rel times the matrix's largest
// diagonal entry sets *bad (atomic min) to the matrix index (badByMatrix) or
// to the pivot's index within its matrix.
struct DenseBatch {
    int nMat, nTiles, nRowTiles;
    const int *dim;
    const long long *off;
    const int *tileOff, *rowTileOff;
    double *A, *D, *C, *thr;
    const long long *cOff;
    int *bad;
    int badByMatrix;
};
size_t dense_inv_panel_doubles(int dim);
size_t dense_inv_pivot_doubles();
int dense_inv_tiles(int dim);
cudaError_t launch_dense_inverse(const DenseBatch &B, int maxDim, long long nEntries, double rel,
                                 cudaStream_t st);

// ---- set-up kernels -------------------------------------------------------


struct KinDev {   // node-blocked input matrix on the device (FP64)
    int nNodes;
    const int *dofStart, *rowPtr, *col;
    const long long *valPtr;
    const double *val;
};

// ---- caller-given block-Jacobi blocks (blocks.cu) ----------------------------

// Dense inverses of the caller's blocks, block b (positions bPos[b] ..
// bPos[b+1]-1, row-major, at A + aOff[b]); position p is entry idx[p] of this
// path's vectors.  Apply units: rows [unitRow0[u], unitRow1[u]) of block
// unitBlk[u].
template <typename T>
struct BlkDev {
    int nBlk, nUnits;
    const long long *aOff;
    const int *bPos, *idx;
    const T *A;
    const int *unitBlk, *unitRow0, *unitRow1;
};
constexpr int kBlkUnitRows = 64;

void launch_gather_blocks(const KinDev &K, long long nnzb, const int *blockRow,
                          const int *blockOfNode, const int *bStart, const int *bDim,
                          const long long *aOff, double *A, cudaStream_t st);
void launch_scale_block_inverse(int n, const int *rowBlock, const int *bStart, const int *bDim,
                                const int *bNode0, const int *bNode1, const long long *aOff,
                                const int *dofStart, const FacDev &F, const double *X, double *Y,
                                float *Z, cudaStream_t st);
template <typename T>
void launch_block_apply(const BlkDev<T> &B, const T *r, T *y, double *partials, Scalars *sc,
                        cudaStream_t st);
template <typename T>
void launch_update_plain(T *u, T *r, const T *p, const T *q, long long n, int mode,
                         double *partials, Scalars *sc, cudaStream_t st);


// pos (optional): node t of the list is written to position pos[t] of a list
// of total nodes (default: position t of count)
int launch_block_cholesky(int B, int count, const int *nodes, const double *Dsoa, double *L64,
                          float *L32, int *bad, cudaStream_t st, const int *pos = nullptr,
                          int total = 0);
void launch_copy_factors(int count, int ents, const int *src, const int *dst, const double *prev,
                         int prevTotal, double *L, int total, cudaStream_t st);
void launch_differ(const double *a, const double *b, long long n, int *differ, cudaStream_t st);
void launch_xrel(int nNodes, const double *coords, const double *centre, const int *sub,
                 double *x64, float *x32, cudaStream_t st);
void launch_build_W(const KinDev &K, int nExt, const int *extBox, const int *extNode,
                    const long long *wOff, const int *sub, const double *xrel,
                    const signed char *hsign, const int *menr, const ZvalDev &Zv, double *W,
                    cudaStream_t st);
void launch_build_E(int nSeg, const int *segBox, const int *segOwner, const int *segBegin,
                    const int *segEnd, const int *extNode, const long long *wOff,
                    const double *W, const int *dofStart, const double *xrel,
                    const signed char *hsign, const int *col0, const int *menr,
                    const ZvalDev &Zv, int k, double *E, cudaStream_t st);
void launch_symmetrize(double *E, int k, cudaStream_t st);
void launch_coarse32(const float *Einv, int k, const float *g32, const double *zr, double *nu,
                     float *nu32, int mode, double *partials, Scalars *sc, cudaStream_t st);
void launch_cast_f32(const double *a, float *b, long long n, cudaStream_t st);
void launch_scale_blocks(const KinDev &K, const int *blockRow, long long nnzb, const FacDev &F,
                         double *Kt, cudaStream_t st);
void launch_scale_W(int nExt, const int *extBox, const int *extNode, const long long *wOff,
                    const int *menr, const int *dofStart, const FacDev &F, const double *W,
                    float *Wt, cudaStream_t st);

// ---- batched FP32 iteration (batch.cu); MB = 4 or 8 ------------------------
//
// Arguments of one system's batched kernels.  The residual is double
// buffered: buffer (bs->its & 1 ? rB : rA) is current, so the kernels pick
// their buffers from the system's own iteration count and one set of
// arguments serves every iteration.
struct SpmmArgs {
    SpmvDev<float> A;
    int m, fin;                // fin 0: iteration (p_j^T K p_j); 1: start (||b_j - K x_j||^2)
    const float *x, *b;
    float *y;
    double *partials;
    BatchScalars *bs;
};
struct RestrictBArgs {
    RowBoxDev B;
    int m, mode;               // 0 iteration; 1 G from the current residual; 2 G = Z~^T f
    float *u, *rA, *rB;
    const float *f;            // mode 2 input
    const float *p, *q;
    double *G, *ZR, *unitPart, *partials;
    float *G32;                // column j at G32 + j * gld (the coarse solve stages it)
    int gld;                   // a multiple of 4, >= k
    BatchScalars *bs;
};
struct CoarseBArgs {
    const float *Einv, *G32;
    int k, m, mode;            // 0 nu only; 1 start; 2 iteration; 3 replacement
    int gld;
    const double *ZR;
    double *NU, *partials;
    float *NU32;
    BatchScalars *bs;
    unsigned long long waitNs; // limit of the bounded waits on the bulk copies of G
};
struct ProlongBArgs {
    RowBoxDev B;
    int m, mode;               // 0 iteration; 1 p = Z~ nu; 2 start; 3 replacement
    const float *NU32, *rA, *rB;
    float *p;
    const BatchScalars *bs;
};
// One iteration over several systems: per kernel a device table of the
// systems' arguments and of their first blocks (system s runs blocks
// off[s] .. off[s + 1] - 1 of a launch of off[nSys] blocks, as block
// b - off[s] of its own grid).
struct BatchSysTab {
    int nSys;
    const SpmmArgs *spmm;
    const RestrictBArgs *rst;
    const CoarseBArgs *crs;
    const ProlongBArgs *pro;
    const int *off[4];         // spmm, restriction, coarse, prolongation
    int blocks[4];
};

template <int MB>
void launch_spmm(const SpmmArgs &a, cudaStream_t st);
bool spmm_prepare();
// persistent grid of the batched product (resident blocks per SM x SMs); < 0 on error
int spmm_persistent_grid(int MB, int nSlicesTotal);
template <int MB>
void launch_restrict_b(const RestrictBArgs &a, cudaStream_t st);
template <int MB>
void launch_coarse_b(const CoarseBArgs &a, cudaStream_t st);
template <int MB>
void launch_prolong_b(const ProlongBArgs &a, cudaStream_t st);
template <int MB>
void launch_iteration_sys(const BatchSysTab &t, cudaStream_t st);
int coarse_b_blocks(int k, int MB);
// column scalars: fresh FP64 reduction slots for the columns in mask; open a
// replacement of the columns in mask; judge their FP64 residuals; arm the
// triggers (first: after the start, every column)
void launch_batch_slots(Scalars *slots, unsigned mask, cudaStream_t st);
void launch_batch_open(BatchScalars *bs, Scalars *slots, unsigned mask, cudaStream_t st);
void launch_batch_judge(BatchScalars *bs, const Scalars *slots, int m, cudaStream_t st);
void launch_batch_arm(BatchScalars *bs, int m, int first, cudaStream_t st);
void launch_batch_hold(BatchScalars *bs, cudaStream_t st);
// FP64 <-> FP32 transforms of the columns being replaced (repl_j)
template <int MB>
void launch_fwd_scale_b(int nNodes, int m, const int *nat, const int *ot, const FacDev &F,
                        const double *r, long long ldr, const BatchScalars *bs, float *outA,
                        float *outB, cudaStream_t st);
template <int MB>
void launch_bwd_accum_b(int nNodes, int m, const int *nat, const int *in, const FacDev &F,
                        float *ut, const BatchScalars *bs, double *u, long long ldu,
                        cudaStream_t st);

// element sensitivities -lam_e^T Khat_e u_e (sensitivity.cu)
constexpr int kSensMaxDofs = 120;   // 8 nodes x 15 dofs
void launch_element_sensitivity(long long nEl, long long n, const int64_t *dofPtr,
                                const int32_t *dofs, const int64_t *matOff, long long matLen,
                                const double *mats, const double *u, const double *lam,
                                double *out, int *bad, cudaStream_t st);
void launch_stiffness_gradient(int nNodes, long long nnzb, long long n, long long nval,
                               const int32_t *dofStart, const int32_t *rowPtr, const int32_t *col,
                               const int64_t *valPtr, const double *lam, const double *u,
                               double *out, int *bad, cudaStream_t st);

}  // namespace xdcg
