// Host side of the xdcg C ABI: input validation, layout planning (integer
// structure only; every floating-point operation runs in a kernel), set-up
// kernels, and the solve drivers for the FP64 and the FP32-inner / FP64-
// refinement paths.
#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "internal.h"

using namespace xdcg;

namespace {

constexpr int kBatch = 8;              // iterations enqueued between convergence polls
constexpr int kMaxGrid = 1 << 16;      // partial-sum slots per reduction value

struct Level64 {
    SpmvDev<double> A;
    NodeDev<double> N;
    BoxDev<double> B;
    BlkDev<double> J;         // caller blocks (when given): dense FP64 inverses
};
struct Level32 {          // block-scaled system K~ = L^-1 K L^-T in FP32
    SpmvDev<float> A;
    SpmvDev<float> Ab;        // the same matrix with the batched product's persistent grid
    RowBoxDev R;
    RowBoxDev Rb;            // the same boxes with the batched kernels' unit tables
    FacDev F;
    const int *dofStart64;    // [nNodes + 1] node dofs in the FP64 (caller's) numbering
    const int *dofStart32;    // [nNodes + 1] node dofs in the box-major FP32 numbering
    BlkDev<float> J;          // caller blocks: FP32 inverses of the block-scaled blocks
};

// A batch of iterations recorded once by stream capture and replayed as one
// graph launch (xdcg_options.graph); key holds the pointers and sizes the
// batch was recorded with.
using LoopKey = std::array<const void *, 8>;
struct LoopGraph {
    cudaGraphExec_t exec = nullptr;
    LoopKey key{};
    long long launches = 0;   // kernels in one replay
};

}  // namespace

struct xdcg_ctx {
    int device = 0;
    cudaStream_t st = nullptr;
    xdcg_options opt{};
    xdcg_info_t info{};
    bool mixed = false;
    bool userBlocks = false;       // M from the caller's blocks (dense inverses)
    long long blkEntries = 0;      // sum of the caller blocks' squared sizes

    int nNodes = 0, nBox = 0, k = 0;
    long long n = 0;
    std::vector<void *> allocs;

    Level64 L64{};
    Level32 L32{};
    double *Einv = nullptr;
    float *Einv32 = nullptr;       // FP32 copy for the mixed path's FP32 iteration
    float *g32 = nullptr;          // FP32 copy of the coarse right-hand side g
    // batched FP32 run (opt.max_batch > 0): vectors n x bMB interleaved by column
    int bMB = 0;
    float *bF32 = nullptr, *bU32 = nullptr, *bRA = nullptr, *bRB = nullptr, *bP = nullptr,
          *bQ = nullptr, *bG32 = nullptr, *bNU32 = nullptr;
    double *bG = nullptr, *bZR = nullptr, *bNU = nullptr, *bUnitPart = nullptr, *bR64 = nullptr;
    BatchScalars *bs = nullptr, *h_bs = nullptr;
    Scalars *bSlots = nullptr, *h_slots = nullptr;   // per-column FP64 reductions (device, pinned)
    // kept for xdcg_setup_update: each node's dofs, its (Jacobi-filtered)
    // diagonal block (host) and its position in its factor list
    std::vector<int> hostKind, hostListPos;
    std::vector<long long> hostDiagOff;
    std::vector<double> hostDiag;
    int reusedFactors = 0, reusedCoarse = 0;
    double *hist = nullptr;        // record_history: ||r_i||^2 of the last FP64 solve
    int histLen = 0;
    double histFF = 0.0;
    long long extRows32 = 0, zEnt32 = 0, wEnt32 = 0;   // sizes of the FP32 box layouts
    double *E = nullptr;                      // E = Z^T K Z as assembled (diagnostics)
    std::vector<void *> temps;                // set-up temporaries

    // FP64 work vectors
    double *u64 = nullptr, *r64 = nullptr, *p64 = nullptr, *q64 = nullptr, *y64 = nullptr;
    double *f64 = nullptr, *uh64 = nullptr;   // host-path staging
    // FP32 work vectors (inner solve)
    float *f32 = nullptr, *u32 = nullptr, *r32 = nullptr, *p32 = nullptr, *q32 = nullptr,
          *y32 = nullptr;
    double *g = nullptr, *zr = nullptr, *nu = nullptr;
    float *nu32 = nullptr;
    double *partials = nullptr;
    Scalars *sc = nullptr, *sc32 = nullptr, *aux = nullptr;
    Scalars *h_sc = nullptr;   // pinned
    int *h_done = nullptr;     // pinned, 2 slots
    Scalars *h_poll = nullptr; // pinned, 2 slots: the FP32 run's scalars at each poll
    cudaEvent_t ev0 = nullptr, ev1 = nullptr, evb[2] = {nullptr, nullptr};
    std::vector<cudaEvent_t> evS, evE;
    std::vector<cudaEvent_t> evP;      // per-kernel marks of timed iterations (time_spmv = 2)
    long long launches = 0;
    // opt.graph: the captures are recorded on a private stream (the context's
    // own may be the legacy default stream, which cannot be captured)
    cudaStream_t capSt = nullptr;
    LoopGraph loop32[2];               // FP32 iteration batch, by residual-buffer parity
    LoopGraph loop64;                  // FP64 iteration batch
    long long graphLaunches = 0;       // graph launches made (diagnostics)
};

namespace {

#define CK(call)                                      \
    do {                                              \
        cudaError_t e_ = (call);                      \
        if (e_ != cudaSuccess) return XDCG_CUDA_ERROR; \
    } while (0)

// opt.graph: (re)record the batch of iterations that enqueue(stream) issues,
// unless G already holds it for this key.  Recording runs nothing; the graph
// holds the same launches, with the same programmatic (PDL) ordering between
// them, as the uncaptured loop, so replaying it gives the same bits.
template <typename F>
xdcg_status loop_graph(xdcg_ctx *c, LoopGraph &G, const LoopKey &key, F &&enqueue) {
    if (G.exec && G.key == key) return XDCG_OK;
    if (G.exec) {
        cudaGraphExecDestroy(G.exec);
        G.exec = nullptr;
    }
    if (!c->capSt) CK(cudaStreamCreateWithFlags(&c->capSt, cudaStreamNonBlocking));
    CK(cudaStreamBeginCapture(c->capSt, cudaStreamCaptureModeThreadLocal));
    const long long l0 = c->launches;
    enqueue(c->capSt);
    G.launches = c->launches - l0;   // counted when replayed, not when recorded
    c->launches = l0;
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(c->capSt, &g);
    if (e != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        return XDCG_CUDA_ERROR;
    }
    const cudaError_t e2 = cudaGraphInstantiate(&G.exec, g, 0);
    cudaGraphDestroy(g);
    if (e2 != cudaSuccess) {
        G.exec = nullptr;
        return XDCG_CUDA_ERROR;
    }
    G.key = key;
    return XDCG_OK;
}

// A named range on the profiler timeline (NVTX) for the life of a scope, so
// that a profiler can select the set-up or one solve; a no-op when no
// profiler is attached.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

template <typename T>
T *dalloc(xdcg_ctx *c, size_t count) {
    void *p = nullptr;
    if (count == 0) count = 1;
    if (cudaMalloc(&p, count * sizeof(T)) != cudaSuccess) return nullptr;
    c->allocs.push_back(p);
    return (T *)p;
}

template <typename T>
T *dalloc_tmp(xdcg_ctx *c, size_t count) {
    void *p = nullptr;
    if (count == 0) count = 1;
    if (cudaMalloc(&p, count * sizeof(T)) != cudaSuccess) return nullptr;
    c->temps.push_back(p);
    return (T *)p;
}

template <typename T>
T *upload_tmp(xdcg_ctx *c, const std::vector<T> &v) {
    T *d = dalloc_tmp<T>(c, v.size());
    if (!d) return nullptr;
    if (!v.empty() && cudaMemcpyAsync(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice,
                                      c->st) != cudaSuccess)
        return nullptr;
    return d;
}

template <typename T>
T *upload(xdcg_ctx *c, const std::vector<T> &v) {
    T *d = dalloc<T>(c, v.size());
    if (!d) return nullptr;
    if (!v.empty() && cudaMemcpyAsync(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice,
                                      c->st) != cudaSuccess)
        return nullptr;
    return d;
}

template <typename T>
bool fetch(std::vector<T> &dst, const T *src, size_t count, int mem) {
    dst.resize(count);
    if (count == 0) return true;
    if (!src) return false;
    if (mem == XDCG_DEVICE)
        return cudaMemcpy(dst.data(), src, count * sizeof(T), cudaMemcpyDeviceToHost) == cudaSuccess;
    std::memcpy(dst.data(), src, count * sizeof(T));
    return true;
}

// f(begin, end) over [0, n) split into contiguous pieces, one host thread
// each (at most 16, and none for small n): the set-up's validation and
// layout loops, whose pieces write disjoint outputs.
template <typename F>
void parallel_for(long long n, F &&f) {
    static const int hw = (int)std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    const int T = (int)std::min<long long>(hw, (n + 8191) / 8192);
    if (T <= 1) {
        f(0LL, n);
        return;
    }
    std::vector<std::thread> th;
    th.reserve(T);
    for (int t = 0; t < T; ++t) th.emplace_back([&f, n, t, T] { f(n * t / T, n * (t + 1) / T); });
    for (auto &x : th) x.join();
}

// Every point of x (p x 3) on one line?  (true for fewer than 3 points)
bool points_collinear(const std::vector<double> &x) {
    const size_t p = x.size() / 3;
    if (p < 3) return true;
    const double *a = &x[0];
    size_t far = 0;
    double best = -1.0;
    for (size_t i = 0; i < p; ++i) {
        double d = 0;
        for (int e = 0; e < 3; ++e) d += (x[3 * i + e] - a[e]) * (x[3 * i + e] - a[e]);
        if (d > best) { best = d; far = i; }
    }
    double ab[3];
    for (int e = 0; e < 3; ++e) ab[e] = x[3 * far + e] - a[e];
    const double ab2 = ab[0] * ab[0] + ab[1] * ab[1] + ab[2] * ab[2];
    for (size_t i = 0; i < p; ++i) {
        double v[3];
        for (int e = 0; e < 3; ++e) v[e] = x[3 * i + e] - a[e];
        const double c0 = v[1] * ab[2] - v[2] * ab[1];
        const double c1 = v[2] * ab[0] - v[0] * ab[2];
        const double c2 = v[0] * ab[1] - v[1] * ab[0];
        if (c0 * c0 + c1 * c1 + c2 * c2 > 1e-12 * ab2 * ab2) return false;
    }
    return true;
}

__global__ void k_init_scalars(Scalars *sc, double tol2, const double *ffsrc, int max_it,
                               double *hist, int histCap) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        Scalars z{};
        z.tol2ff = ffsrc ? tol2 * (*ffsrc) : tol2;
        z.max_it = max_it;
        z.hist = hist;
        z.histCap = histCap;
        *sc = z;
    }
}

void init_scalars(xdcg_ctx *c, Scalars *sc, double tol2, const double *ffsrc, int max_it,
                  double *hist = nullptr, int histCap = 0) {
    k_init_scalars<<<1, 32, 0, c->st>>>(sc, tol2, ffsrc, max_it, hist, histCap);
    c->launches++;
}

xdcg_status map_done(int done) {
    switch (done) {
        case kConverged: return XDCG_OK;
        case kBreakdown: return XDCG_BREAKDOWN;
        case kMaxIter: return XDCG_NO_CONVERGENCE;
        case kFault: return XDCG_TIMEOUT;
        default: return XDCG_NO_CONVERGENCE;
    }
}

// Kernel timing of the iteration loop (time_spmv = 2): mark m of iteration it
// is recorded before the iteration's kernel m, mark P after its last kernel.
constexpr int kMarks = 6;

xdcg_status phase_mark(xdcg_ctx *c, int it, int m) {
    const size_t idx = (size_t)it * kMarks + m;
    while (c->evP.size() <= idx) {
        cudaEvent_t e;
        CK(cudaEventCreate(&e));
        c->evP.push_back(e);
    }
    CK(cudaEventRecord(c->evP[idx], c->st));
    return XDCG_OK;
}

// sums the phase times of the first n timed iterations into res
xdcg_status phase_collect(xdcg_ctx *c, int n, int P, xdcg_result *res) {
    for (int it = 0; it < n; ++it)
        for (int m = 0; m < P; ++m) {
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, c->evP[(size_t)it * kMarks + m],
                                    c->evP[(size_t)it * kMarks + m + 1]));
            res->t_phase_ms[m] += ms;
        }
    res->n_phase_timed += n;
    return XDCG_OK;
}

#define MARK(it, m)                                                             \
    do {                                                                        \
        if (timeKernels) {                                                      \
            xdcg_status ms_ = phase_mark(c, (it), (m));                         \
            if (ms_ != XDCG_OK) return ms_;                                     \
        }                                                                       \
    } while (0)

// ---- one preconditioned CG run (Algorithms 1-3) ----------------------------

// Unscaled path: block-Jacobi applied by the node-block factors, Z from
// coordinates.  Used in FP64.
struct PlainPath {
    xdcg_ctx *c;
    Level64 &L;
    cudaStream_t st;          // the stream its kernels are enqueued on
    void spmv(const double *x, double *y, const double *b, int res, int fin, Scalars *sc) {
        launch_spmv<double>(L.A, x, y, b, res, c->partials, sc, fin, 0, st);
    }
    void update(double *u, double *r, const double *p, const double *q, double *y, int mode,
                Scalars *sc) {
        if (c->userBlocks) {
            // caller blocks: the update, then y = M^-1 r by the blocks' dense inverses
            launch_update_plain<double>(u, r, p, q, c->n, mode, c->partials, sc, st);
            launch_block_apply<double>(L.J, r, y, c->partials, sc, st);
            c->launches++;
        } else {
            launch_update<double>(L.N, u, r, p, q, y, mode, c->partials, sc, st);
        }
    }
    void restrict_(const double *a, const double *b, int withW, double *zr, Scalars *sc) {
        launch_restrict(L.B, a, b, withW, c->g, zr, sc, st);
    }
    void coarse(const double *zr, int mode, Scalars *sc) {
        launch_coarse(c->Einv, c->k, c->g, zr, c->nu, nullptr, mode, c->partials, sc, st);
    }
    void prolong(const double *y, double *p, int mode, Scalars *sc) {
        launch_prolong(L.B, c->nu, y, p, mode, sc, st);
    }
};

template <typename T, typename Path>
xdcg_status run_pcg(xdcg_ctx *c, Path path, const T *f, T *u, T *r, T *p, T *q, T *y,
                    Scalars *sc, int max_it, bool guess, int *its_out, int *done_out,
                    xdcg_result *res) {
    cudaStream_t st = c->st;
    const bool timeSpmv = c->opt.time_spmv == 1, timeKernels = c->opt.time_spmv == 2;
    if (guess) {
        // Algorithm 2 with the caller's u_-1 (in u): u_0 = u_-1 + Z E^-1 Z^T (f - K u_-1)
        path.spmv(u, r, f, 1, kFinStore, sc);
        path.restrict_(r, nullptr, 0, nullptr, sc);
        path.coarse(nullptr, 0, sc);
        path.prolong(u, u, 2, sc);
        c->launches += 4;
    } else {
        // Algorithm 2 with u_-1 = 0: u_0 = Z E^-1 Z^T f
        path.restrict_(f, nullptr, 0, nullptr, sc);
        path.coarse(nullptr, 0, sc);
        path.prolong(nullptr, u, 1, sc);
        c->launches += 3;
    }
    // r_0 = f - K u_0, z_0 by Algorithm 3, p_0 = z_0
    path.spmv(u, r, f, 1, kFinRR, sc);
    path.update(u, r, nullptr, nullptr, y, 1, sc);
    path.restrict_(r, y, 1, c->zr, sc);
    path.coarse(c->zr, 1, sc);
    path.prolong(y, p, 2, sc);
    c->launches += 5;

    int launched = 0;
    const int max_batches = max_it / kBatch + 2;
    // opt.graph: the batch's kernels as one recorded graph (not with the
    // timing modes, whose events sit between the kernels)
    const bool useGraph = c->opt.graph && !timeSpmv && !timeKernels;
    if (useGraph) {
        const LoopKey key{u, r, p, q, y, sc, c->zr, nullptr};
        xdcg_status s = loop_graph(c, c->loop64, key, [&](cudaStream_t cs) {
            Path rec = path;
            rec.st = cs;
            for (int i = 0; i < kBatch; ++i) {
                rec.spmv(p, q, nullptr, 0, kFinAlpha, sc);
                rec.update(u, r, p, q, y, 0, sc);
                rec.restrict_(r, y, 1, c->zr, sc);
                rec.coarse(c->zr, 2, sc);
                rec.prolong(y, p, 0, sc);
                c->launches += 5;
            }
        });
        if (s != XDCG_OK) return s;
    }
    for (int b = 0; b < max_batches; ++b) {
        if (useGraph) {
            CK(cudaGraphLaunch(c->loop64.exec, st));
            c->launches += c->loop64.launches;
            c->graphLaunches++;
            launched += kBatch;
        }
        for (int i = 0; i < kBatch && !useGraph; ++i) {
            if (timeSpmv) {
                if ((int)c->evS.size() <= launched) {
                    cudaEvent_t e0, e1;
                    CK(cudaEventCreate(&e0));
                    CK(cudaEventCreate(&e1));
                    c->evS.push_back(e0);
                    c->evE.push_back(e1);
                }
                CK(cudaEventRecord(c->evS[launched], st));
            }
            MARK(launched, 0);
            path.spmv(p, q, nullptr, 0, kFinAlpha, sc);
            if (timeSpmv) CK(cudaEventRecord(c->evE[launched], st));
            MARK(launched, 1);
            path.update(u, r, p, q, y, 0, sc);
            MARK(launched, 2);
            path.restrict_(r, y, 1, c->zr, sc);
            MARK(launched, 3);
            path.coarse(c->zr, 2, sc);
            MARK(launched, 4);
            path.prolong(y, p, 0, sc);
            MARK(launched, 5);
            c->launches += 5;
            ++launched;
        }
        CK(cudaMemcpyAsync(&c->h_done[b & 1], &sc->done, sizeof(int), cudaMemcpyDeviceToHost, st));
        CK(cudaEventRecord(c->evb[b & 1], st));
        if (b >= 1) {
            CK(cudaEventSynchronize(c->evb[(b - 1) & 1]));
            if (c->h_done[(b - 1) & 1] != kRunning) break;
        }
    }
    CK(cudaMemcpyAsync(c->h_sc, sc, sizeof(Scalars), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    CK(cudaGetLastError());
    *its_out = c->h_sc->its;
    *done_out = c->h_sc->done;
    const int nt = std::min(launched, c->h_sc->its);
    if (timeSpmv) {
        for (int i = 0; i < nt; ++i) {
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, c->evS[i], c->evE[i]));
            res->t_spmv_ms += ms;
        }
        res->n_spmv_timed += nt;
    }
    if (timeKernels) {
        xdcg_status s = phase_collect(c, nt, 5, res);
        if (s != XDCG_OK) return s;
        res->t_spmv_ms = res->t_phase_ms[0];
        res->n_spmv_timed = res->n_phase_timed;
    }
    return XDCG_OK;
}

// The FP32 inner solve on the block-scaled system: four kernels per
// iteration (SpMV with p^T q; restriction fused with the u, r update and
// ||r||^2; coarse solve; prolongation), the residual double-buffered so that
// the restriction can read the old residual of neighbouring boxes while it
// writes the new one of its own.  Iteration i reads residual buffer
// (i & 1 ? rB : rA) and writes the other.

__global__ void k_set_trigger(Scalars *sc, int mode, double delta2, double floor2) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        if (mode == 0) {            // re-arm without a convergence test; keep the
            sc->done = kRunning;    // recursive ||r||^2 for the restart test
            sc->tol2ff = -1.0;
            sc->scratch[3] = sc->rr;
        } else {                    // next residual replacement when ||r||^2 drops below this
            sc->tol2ff = fmax(delta2 * sc->rr, floor2);
        }
    }
}

// nu = E^-1 g inside the FP32 iteration: the FP32 copy of E^-1 (default) or
// the FP64 one (opt.coarse_fp64), both writing nu and its FP32 copy nu32
void coarse_inner(xdcg_ctx *c, const double *zr, int mode, Scalars *sc, cudaStream_t st) {
    if (c->opt.coarse_fp64)
        launch_coarse(c->Einv, c->k, c->g, zr, c->nu, c->nu32, mode, c->partials, sc, st);
    else
        launch_coarse32(c->Einv32, c->k, c->g32, zr, c->nu, c->nu32, mode, c->partials, sc, st);
}

// Algorithm 2 and the first direction: u~ = Z~ E^-1 Z~^T f~, r = f~ - K~ u~ (rA),
// z = r + Z~ nu, p = z.
void scaled_init(xdcg_ctx *c, const float *f, float *u, float *rA, float *p, Scalars *sc) {
    cudaStream_t st = c->st;
    Level32 &L = c->L32;
    launch_restrict_update(L.R, nullptr, f, nullptr, nullptr, nullptr, 2, c->g, nullptr,
                           c->partials, sc, st);
    coarse_inner(c, nullptr, 0, sc, st);
    launch_prolong_rows(L.R, c->nu32, nullptr, u, 1, sc, st);
    launch_spmv<float>(L.A, u, rA, f, 1, c->partials, sc, kFinRR, 0, st);
    if (c->userBlocks) {
        // y = M~^-1 r by the caller blocks, then g = Z~^T r - W~^T y
        launch_block_apply<float>(L.J, rA, c->y32, c->partials, sc, st);
        launch_restrict_update(L.R, nullptr, rA, nullptr, nullptr, nullptr, 3, c->g, c->zr,
                               c->partials, sc, st, c->y32);
        coarse_inner(c, c->zr, 1, sc, st);
        launch_prolong_rows(L.R, c->nu32, c->y32, p, 2, sc, st);
        c->launches += 8;
        return;
    }
    launch_restrict_update(L.R, nullptr, rA, nullptr, nullptr, nullptr, 1, c->g, c->zr,
                           c->partials, sc, st);
    coarse_inner(c, c->zr, 1, sc, st);
    launch_prolong_rows(L.R, c->nu32, rA, p, 2, sc, st);
    c->launches += 7;
}

// A stall of the FP32 run: kStallIts iterations without the recursive
// ||r|| dropping by 10 % (||r||^2 by 19 %) below its best.  A healthy run
// drops it by 1e-3 in some tens of iterations; a stall means that the FP32
// rounding of K~ hides the components still to be resolved.
constexpr int kStallIts = 200;

// Run iterations (in batches, polling the device flag) until a kernel stops
// the run (the replacement trigger, breakdown, the iteration cap) or the run
// stalls (*stalled, the device flag still running).
xdcg_status scaled_iterate(xdcg_ctx *c, float *u, float *rA, float *rB, float *p, float *q,
                           Scalars *sc, int max_it, int *its_out, int *done_out,
                           xdcg_result *res, bool *stalled) {
    cudaStream_t st = c->st;
    Level32 &L = c->L32;
    const bool timeSpmv = c->opt.time_spmv == 1, timeKernels = c->opt.time_spmv == 2;
    CK(cudaMemcpyAsync(c->h_sc, sc, sizeof(Scalars), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    const int it0 = c->h_sc->its;
    int i = it0, launched = 0;
    const int max_batches = (max_it - it0) / kBatch + 2;
    double bestRR = c->h_sc->rr;
    int lastGain = it0;
    *stalled = false;
    // kernel m (0..3) of iteration it of the FP32 iteration, enqueued on s
    auto kernel = [&](int m, int it, cudaStream_t s) {
        float *rc = (it & 1) ? rB : rA;
        float *rn = (it & 1) ? rA : rB;
        // without caller blocks the product leaves its blocks' sums of
        // p^T q for the restriction to add (no ticketed reduction at the
        // product's end), past the region the restriction's own
        // reduction uses
        float2 *pqPart = reinterpret_cast<float2 *>(c->partials + kMaxGrid);
        if (m == 0) {
            launch_spmv<float>(L.A, p, q, nullptr, 0,
                               c->userBlocks ? c->partials : c->partials + kMaxGrid, sc,
                               c->userBlocks ? kFinAlpha : kFinDefer, 0, s);
        } else if (m == 1) {
            if (c->userBlocks) {
                // residual in place (no neighbour reads before the apply), y
                // = M~^-1 r by the caller blocks, then the restriction
                launch_update_plain<float>(u, rA, p, q, c->n, 0, c->partials, sc, s);
                launch_block_apply<float>(L.J, rA, c->y32, c->partials, sc, s);
                launch_restrict_update(L.R, nullptr, rA, nullptr, nullptr, nullptr, 3, c->g, c->zr,
                                       c->partials, sc, s, c->y32);
                c->launches += 2;
            } else {
                launch_restrict_update_deferred(L.R, u, rc, rn, p, q, c->g, c->zr, c->partials, sc,
                                                pqPart, L.A.grid, s);
            }
        } else if (m == 2) {
            coarse_inner(c, c->zr, 2, sc, s);
        } else {
            launch_prolong_rows(L.R, c->nu32, c->userBlocks ? c->y32 : rn, p, 0, sc, s);
            c->launches += 4;
        }
    };
    // opt.graph: a batch's kernels as one recorded graph per residual-buffer
    // parity of its first iteration (kBatch is even), not with the timing
    // modes, whose events sit between the kernels
    const bool useGraph = c->opt.graph && !timeSpmv && !timeKernels;
    LoopGraph &G = c->loop32[it0 & 1];
    if (useGraph) {
        const LoopKey key{u, rA, rB, p, q, sc, c->zr, c->userBlocks ? c->y32 : nullptr};
        xdcg_status s = loop_graph(c, G, key, [&](cudaStream_t cs) {
            for (int j = 0; j < kBatch; ++j)
                for (int m = 0; m < 4; ++m) kernel(m, it0 + j, cs);
        });
        if (s != XDCG_OK) return s;
    }
    for (int b = 0; b < max_batches; ++b) {
        if (useGraph) {
            CK(cudaGraphLaunch(G.exec, st));
            c->launches += G.launches;
            c->graphLaunches++;
            i += kBatch;
            launched += kBatch;
        }
        for (int j = 0; j < kBatch && !useGraph; ++j, ++i, ++launched) {
            if (timeSpmv) {
                if ((int)c->evS.size() <= launched) {
                    cudaEvent_t e0, e1;
                    CK(cudaEventCreate(&e0));
                    CK(cudaEventCreate(&e1));
                    c->evS.push_back(e0);
                    c->evE.push_back(e1);
                }
                CK(cudaEventRecord(c->evS[launched], st));
            }
            MARK(launched, 0);
            kernel(0, i, st);
            if (timeSpmv) CK(cudaEventRecord(c->evE[launched], st));
            MARK(launched, 1);
            kernel(1, i, st);
            MARK(launched, 2);
            kernel(2, i, st);
            MARK(launched, 3);
            kernel(3, i, st);
            MARK(launched, 4);
        }
        // one copy per poll: the stop flag and ||r||^2 for the stall test
        CK(cudaMemcpyAsync(&c->h_poll[b & 1], sc, sizeof(Scalars), cudaMemcpyDeviceToHost, st));
        CK(cudaEventRecord(c->evb[b & 1], st));
        if (b >= 1) {
            CK(cudaEventSynchronize(c->evb[(b - 1) & 1]));
            if (c->h_poll[(b - 1) & 1].done != kRunning) break;
            const double rrNow = c->h_poll[(b - 1) & 1].rr;
            const int itNow = it0 + b * kBatch;
            if (rrNow < 0.81 * bestRR) {
                bestRR = rrNow;
                lastGain = itNow;
            } else if (itNow - lastGain >= kStallIts) {
                *stalled = true;
                break;
            }
        }
    }
    CK(cudaMemcpyAsync(c->h_sc, sc, sizeof(Scalars), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    CK(cudaGetLastError());
    *its_out = c->h_sc->its;
    *done_out = c->h_sc->done;
    if (*done_out != kRunning) *stalled = false;
    const int nt = std::min(launched, c->h_sc->its - it0);
    if (timeSpmv) {
        for (int e = 0; e < nt; ++e) {
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, c->evS[e], c->evE[e]));
            res->t_spmv_ms += ms;
        }
        res->n_spmv_timed += nt;
    }
    if (timeKernels) {
        const double t0 = res->t_phase_ms[0];
        const int n0 = res->n_phase_timed;
        xdcg_status s = phase_collect(c, nt, 4, res);
        if (s != XDCG_OK) return s;
        res->t_spmv_ms += res->t_phase_ms[0] - t0;
        res->n_spmv_timed += res->n_phase_timed - n0;
    }
    return XDCG_OK;
}

xdcg_status read_aux(xdcg_ctx *c, double *vals, int count) {
    CK(cudaMemcpyAsync(c->h_sc, c->aux, sizeof(Scalars), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    for (int i = 0; i < count; ++i) vals[i] = c->h_sc->scratch[i];
    return c->h_sc->done == kFault ? XDCG_TIMEOUT : XDCG_OK;
}

xdcg_status solve_fp64(xdcg_ctx *c, const double *f, double *u, double tol, bool guess,
                       xdcg_result *res) {
    cudaStream_t st = c->st;
    init_scalars(c, c->aux, -1.0, nullptr, INT_MAX);
    launch_dot<double>(f, f, c->n, c->partials, c->aux, kFinStore, 0, st);
    init_scalars(c, c->sc, tol * tol, &c->aux->scratch[0], c->opt.max_iter, c->hist,
                 c->hist ? c->opt.max_iter + 1 : 0);
    c->launches += 1;
    int its = 0, done = 0;
    xdcg_status s = run_pcg<double>(c, PlainPath{c, c->L64, c->st}, f, u, c->r64, c->p64, c->q64,
                                    c->y64, c->sc, c->opt.max_iter, guess, &its, &done, res);
    if (s != XDCG_OK) return s;
    const double rr = c->h_sc->rr;
    // true residual f - K u in FP64
    launch_spmv<double>(c->L64.A, u, c->r64, f, 1, c->partials, c->aux, kFinStore, 1, st);
    c->launches += 1;
    double v[2];
    if ((s = read_aux(c, v, 2)) != XDCG_OK) return s;
    const double ff = v[0];
    c->histLen = c->hist ? std::min(its, c->opt.max_iter) + 1 : 0;
    c->histFF = ff;
    res->iterations = its;
    res->outer_cycles = 1;
    res->rel_res_recursive = ff > 0 ? std::sqrt(rr / ff) : 0.0;
    res->rel_res_true = ff > 0 ? std::sqrt(v[1] / ff) : 0.0;
    return map_done(done);
}

// FP32-inner / FP64-refinement solve with residual replacement ("reliable
// updates"): one FP32 A-DEF2 CG run on the block-scaled system; whenever its
// recursive residual has dropped by the factor inner_tol since the last
// replacement, the FP32 correction is added to the FP64 solution, the true
// residual f - K u is recomputed in FP64, and its scaled image replaces the
// recursive residual while the search direction and rho carry on, so the
// Krylov space is not restarted.
xdcg_status solve_mixed(xdcg_ctx *c, const double *f, double *u, double tol, bool guess,
                        xdcg_result *res) {
    cudaStream_t st = c->st;
    Level32 &L = c->L32;
    init_scalars(c, c->aux, -1.0, nullptr, INT_MAX);
    launch_dot<double>(f, f, c->n, c->partials, c->aux, kFinStore, 0, st);
    c->launches += 1;
    double v[2];
    xdcg_status s;
    if ((s = read_aux(c, v, 1)) != XDCG_OK) return s;
    const double ff = v[0];
    if (!guess || ff == 0.0) CK(cudaMemsetAsync(u, 0, c->n * sizeof(double), st));
    res->iterations = 0;
    res->outer_cycles = 0;
    res->rel_res_recursive = 0.0;
    res->rel_res_true = 0.0;
    if (ff == 0.0) return XDCG_OK;
    if (!std::isfinite(ff)) return XDCG_BREAKDOWN;
    double rn2 = ff;
    const double *rhs = f;
    if (guess) {
        // start from the caller's u: the FP32 run solves for the correction of
        // r = f - K u (Algorithm 2 with u_-1 = u, applied to the correction)
        init_scalars(c, c->aux, -1.0, nullptr, INT_MAX);
        launch_spmv<double>(c->L64.A, u, c->r64, f, 1, c->partials, c->aux, kFinStore, 0, st);
        c->launches += 1;
        if ((s = read_aux(c, v, 1)) != XDCG_OK) return s;
        rn2 = v[0];
        res->rel_res_true = std::sqrt(rn2 / ff);
        if (!std::isfinite(rn2)) return XDCG_BREAKDOWN;
        if (rn2 <= tol * tol * ff) return XDCG_OK;
        rhs = c->r64;
    }
    const double s0 = 1.0 / std::sqrt(ff);
    const double delta2 = c->opt.inner_tol * c->opt.inner_tol;
    float *rA = c->r32, *rB = c->y32;
    // f~ = s0 L^-1 f (or of the starting residual), and the FP32 run from Algorithm 2
    launch_fwd_scale(c->nNodes, L.dofStart64, L.dofStart64, L.dofStart32, L.F, rhs, s0, c->f32,
                     st);
    CK(cudaMemsetAsync(c->u32, 0, c->n * sizeof(float), st));
    init_scalars(c, c->sc32, -1.0, nullptr, c->opt.max_iter);
    scaled_init(c, c->f32, c->u32, rA, c->p32, c->sc32);
    k_set_trigger<<<1, 32, 0, st>>>(c->sc32, 1, delta2, 0.0);
    c->launches += 2;
    double last_rec = 1.0;
    int cycles = 0, its = 0, done = 0, breakdowns = 0, slow = 0;
    bool finishFp64 = false, stalled = false;
    xdcg_status status = XDCG_NO_CONVERGENCE;
    while (true) {
        s = scaled_iterate(c, c->u32, rA, rB, c->p32, c->q32, c->sc32, c->opt.max_iter, &its,
                           &done, res, &stalled);
        if (s != XDCG_OK) return s;
        if (done == kFault) return XDCG_TIMEOUT;
        last_rec = std::sqrt(c->h_sc->rr);
        // fold the FP32 correction into u (FP64): u += L^-T u~ / s0
        launch_bwd_accum(c->nNodes, L.dofStart64, L.dofStart32, L.dofStart64, L.F, c->u32, 1.0 / s0,
                         u, st);
        CK(cudaMemsetAsync(c->u32, 0, c->n * sizeof(float), st));
        init_scalars(c, c->aux, -1.0, nullptr, INT_MAX);
        launch_spmv<double>(c->L64.A, u, c->r64, f, 1, c->partials, c->aux, kFinStore, 0, st);
        c->launches += 3;
        if ((s = read_aux(c, v, 1)) != XDCG_OK) return s;
        const double prev = rn2;
        rn2 = v[0];
        cycles++;
        if (!std::isfinite(rn2)) { status = XDCG_BREAKDOWN; break; }
        if (rn2 <= tol * tol * ff) { status = XDCG_OK; break; }
        if (done == kMaxIter) { status = XDCG_NO_CONVERGENCE; break; }
        // two replacements in a row that shortened the FP64 residual by less
        // than 2x (or the replacement budget spent): the FP32 recurrence has
        // reached its rounding floor; the FP64 iteration finishes from u
        slow = rn2 > 0.25 * prev ? slow + 1 : 0;
        if (stalled || slow >= 2 || cycles >= c->opt.max_outer) { finishFp64 = true; break; }
        if (done == kBreakdown) {
            if (rn2 >= prev || ++breakdowns > 2) { status = XDCG_BREAKDOWN; break; }
        }
        // replace the recursive residual by the scaled true residual and finish
        // the interrupted iteration: z = r + Z~ nu, beta, p = z + beta p (beta =
        // 0 if the replacement moved the residual far: see k_coarse mode 3)
        float *rbuf = (c->userBlocks || !(its & 1)) ? rA : rB;
        launch_fwd_scale(c->nNodes, L.dofStart64, L.dofStart64, L.dofStart32, L.F, c->r64, s0, rbuf,
                         st);
        k_set_trigger<<<1, 32, 0, st>>>(c->sc32, 0, 0.0, 0.0);
        if (c->userBlocks) {
            launch_update_plain<float>(nullptr, rbuf, nullptr, nullptr, c->n, 1, c->partials,
                                       c->sc32, st);
            launch_block_apply<float>(L.J, rbuf, c->y32, c->partials, c->sc32, st);
            launch_restrict_update(L.R, nullptr, rbuf, nullptr, nullptr, nullptr, 3, c->g, c->zr,
                                   c->partials, c->sc32, st, c->y32);
            c->launches += 2;
        } else {
            launch_restrict_update(L.R, nullptr, rbuf, nullptr, nullptr, nullptr, 1, c->g, c->zr,
                                   c->partials, c->sc32, st);
        }
        coarse_inner(c, c->zr, done == kBreakdown ? 1 : 3, c->sc32, st);
        launch_prolong_rows(L.R, c->nu32, c->userBlocks ? c->y32 : rbuf, c->p32,
                            done == kBreakdown ? 2 : 0, c->sc32, st);
        c->launches += 5;
        CK(cudaMemcpyAsync(c->h_sc, c->sc32, sizeof(Scalars), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        // next replacement: a further factor inner_tol, or sooner when the
        // scaled residual, at the ratio just observed between the scaled and
        // the true norm, should be at half the target -- but not before it has
        // dropped by a factor 10: near the target a few CG steps shorten the
        // scaled residual without shortening the true one
        const double gamma2 = c->h_sc->rr / (s0 * s0 * rn2);
        const double floor2 = std::min(0.25 * tol * tol * ff * s0 * s0 * gamma2,
                                       kMinGroupDrop2 * c->h_sc->rr);
        k_set_trigger<<<1, 32, 0, st>>>(c->sc32, 1, delta2, floor2);
        c->launches += 1;
    }
    res->iterations = its;
    res->outer_cycles = cycles;
    res->rel_res_recursive = last_rec;
    res->rel_res_true = std::sqrt(rn2 / ff);
    if (finishFp64) {
        // Algorithm 2 with u_-1 = u, then FP64 A-DEF2 PCG to tol; its iterations
        // and its one FP64 residual evaluation are added to the counts
        xdcg_result r64{};
        r64.bad_index = -1;
        s = solve_fp64(c, f, u, tol, true, &r64);
        res->iterations = its + r64.iterations;
        res->outer_cycles = cycles + 1;
        res->rel_res_recursive = r64.rel_res_recursive;
        res->rel_res_true = r64.rel_res_true;
        res->n_fp64_iterations = r64.iterations;
        return s;
    }
    return status;
}

// ---- batched mixed solve: m right-hand sides per system, one or several systems ----
//
// The start (||f_j||^2, Algorithm 2 and the first directions for every
// column) is enqueued for every system after one wait.  Then each tick
// enqueues kTick FP32 iterations (one launch per kernel over all systems
// when there are several), reads the snapshot of every system's scalars
// taken at the end of the previous tick (so the device works on this tick
// meanwhile) and enqueues a replacement of the columns held there: fold of
// the FP32 correction into U, FP64 residual f_j - K U_j, the test against
// tol, the transform of the new residual and Algorithm 3 on it.  The held
// columns of a system wait for that while its other columns and the other
// systems iterate; a system whose columns have all left drops out.

constexpr int kTick = 2;    // batched iterations enqueued between snapshots

struct BatchRun {
    xdcg_ctx *c = nullptr;
    const double *F = nullptr;
    double *U = nullptr;
    int m = 0;
    double tol = 0.0;
    bool live = false;         // columns left
    SpmmArgs spmm{};
    RestrictBArgs rst{};
    CoarseBArgs crs{};
    ProlongBArgs pro{};
};

int g_ld(const xdcg_ctx *c) { return (std::max(c->k, 1) + 3) & ~3; }
RestrictBArgs restrict_args(xdcg_ctx *c, int m, int mode) {
    return RestrictBArgs{c->L32.Rb, m, mode, c->bU32, c->bRA, c->bRB, c->bF32, c->bP, c->bQ,
                         c->bG, mode == 2 ? nullptr : c->bZR, c->bUnitPart, c->partials,
                         c->bG32, g_ld(c), c->bs};
}
CoarseBArgs coarse_args(xdcg_ctx *c, int m, int mode) {
    return CoarseBArgs{c->Einv32, c->bG32, c->k, m, mode, g_ld(c), mode == 0 ? nullptr : c->bZR,
                       c->bNU, c->partials, c->bNU32, c->bs, c->L32.A.waitNs};
}
ProlongBArgs prolong_args(xdcg_ctx *c, int m, int mode) {
    return ProlongBArgs{c->L32.Rb, m, mode, c->bNU32, c->bRA, c->bRB,
                        mode == 1 ? c->bU32 : c->bP, c->bs};
}

// host scalars from the columns' ||f_j||^2 (fresh slots), then the start
template <int MB>
xdcg_status batch_start(BatchRun &R, cudaStream_t st) {
    xdcg_ctx *c = R.c;
    Level32 &L = c->L32;
    const long long n = c->n;
    const int m = R.m;
    BatchScalars &hb = *c->h_bs;
    hb = BatchScalars{};
    hb.max_it = c->opt.max_iter;
    hb.max_outer = c->opt.max_outer;
    hb.tol = R.tol;
    hb.delta2 = c->opt.inner_tol * c->opt.inner_tol;
    int nActive = 0;
    for (int j = 0; j < m; ++j) {
        if (c->h_slots[j].done == kFault) return XDCG_TIMEOUT;
        const double ff = c->h_slots[j].scratch[0];
        hb.ff[j] = hb.rn2[j] = ff;
        hb.repl[j] = 1;
        hb.trig[j] = -1.0;
        if (!std::isfinite(ff)) {
            hb.outcome[j] = kColBad;
            continue;
        }
        hb.active[j] = ff > 0.0;
        hb.scale[j] = ff > 0.0 ? 1.0 / std::sqrt(ff) : 0.0;
        nActive += hb.active[j];
    }
    hb.done = kRunning;
    hb.go = 1;
    CK(cudaMemsetAsync(R.U, 0, (size_t)m * n * sizeof(double), st));
    R.live = nActive > 0;
    if (!R.live) return XDCG_OK;
    CK(cudaMemcpyAsync(c->bs, c->h_bs, sizeof(BatchScalars), cudaMemcpyHostToDevice, st));
    // F~ = s_j L^-1 f_j; u~ = Z~ E^-1 Z~^T F~ (Algorithm 2); r = F~ - K~ u~; the
    // first directions p = r + Z~ E^-1 (Z~^T r - W~^T r)
    launch_fwd_scale_b<MB>(c->nNodes, m, L.dofStart64, L.dofStart32, L.F, R.F, n, c->bs, c->bF32,
                           c->bF32, st);
    CK(cudaMemsetAsync(c->bU32, 0, (size_t)n * MB * sizeof(float), st));
    launch_restrict_b<MB>(restrict_args(c, m, 2), st);
    launch_coarse_b<MB>(coarse_args(c, m, 0), st);
    launch_prolong_b<MB>(prolong_args(c, m, 1), st);
    launch_spmm<MB>(SpmmArgs{L.Ab, m, 1, c->bU32, c->bF32, c->bRA, c->partials, c->bs}, st);
    launch_restrict_b<MB>(restrict_args(c, m, 1), st);
    launch_coarse_b<MB>(coarse_args(c, m, 1), st);
    launch_prolong_b<MB>(prolong_args(c, m, 2), st);
    launch_batch_arm(c->bs, m, 1, st);
    c->launches += 10;
    R.spmm = SpmmArgs{L.Ab, m, 0, c->bP, nullptr, c->bQ, c->partials, c->bs};
    R.rst = restrict_args(c, m, 0);
    R.crs = coarse_args(c, m, 2);
    R.pro = prolong_args(c, m, 0);
    return XDCG_OK;
}

// replacement of the columns in mask M of one system
template <int MB>
void batch_replace(BatchRun &R, unsigned M, cudaStream_t st) {
    xdcg_ctx *c = R.c;
    Level32 &L = c->L32;
    const long long n = c->n;
    const int m = R.m;
    launch_batch_open(c->bs, c->bSlots, M, st);
    launch_bwd_accum_b<MB>(c->nNodes, m, L.dofStart64, L.dofStart32, L.F, c->bU32, c->bs, R.U, n,
                           st);
    int nr = 0;
    for (int j = 0; j < m; ++j)
        if ((M >> j) & 1u) {
            launch_spmv<double>(c->L64.A, R.U + j * n, c->bR64 + j * n, R.F + j * n, 1,
                                c->partials, c->bSlots + j, kFinStore, 0, st);
            ++nr;
        }
    launch_batch_judge(c->bs, c->bSlots, m, st);
    launch_fwd_scale_b<MB>(c->nNodes, m, L.dofStart64, L.dofStart32, L.F, c->bR64, n, c->bs,
                           c->bRA, c->bRB, st);
    launch_restrict_b<MB>(restrict_args(c, m, 1), st);
    launch_coarse_b<MB>(coarse_args(c, m, 3), st);
    launch_prolong_b<MB>(prolong_args(c, m, 3), st);
    launch_batch_arm(c->bs, m, 0, st);
    c->launches += 8 + nr;
}

// per-column results from the final scalars; the system's status
xdcg_status batch_results(const BatchRun &R, xdcg_result *res) {
    const BatchScalars &hb = *R.c->h_bs;
    bool bad = false, limit = false;
    for (int j = 0; j < R.m; ++j) {
        xdcg_result r{};
        r.bad_index = hb.outcome[j] == kColBad ? j : -1;
        r.iterations = hb.itsc[j];
        r.outer_cycles = hb.cycles[j];
        // the FP32 recursion's residual before the last replacement
        r.rel_res_recursive = std::sqrt(hb.cycles[j] ? hb.rrRep[j] : hb.rr[j]);
        r.rel_res_true = hb.outcome[j] == kColBad ? std::nan("")
                         : hb.ff[j] > 0.0        ? std::sqrt(hb.rn2[j] / hb.ff[j])
                                                 : 0.0;
        bad |= hb.outcome[j] == kColBad;
        limit |= hb.outcome[j] == kColLimit;
        if (res) res[j] = r;
    }
    return bad ? XDCG_BREAKDOWN : limit ? XDCG_NO_CONVERGENCE : XDCG_OK;
}

// Device tables of the live systems' iteration arguments for launches over
// several systems: one version per live set (a version is never rewritten
// while launches that read it may be queued).
struct SysTables {
    int nSys = 0, versions = 0, used = 0;
    size_t vbytes = 0;
    unsigned char *dev = nullptr, *host = nullptr;   // device / pinned staging
    cudaStream_t st = nullptr;
    ~SysTables() {
        if (dev) cudaFreeAsync(dev, st);
        if (host) {
            cudaStreamSynchronize(st);   // copies from the staging may still be queued
            cudaFreeHost(host);
        }
    }
};

xdcg_status sys_tables_init(SysTables &T, int nSys, cudaStream_t st) {
    T.st = st;
    T.nSys = nSys;
    T.versions = nSys + 1;
    T.vbytes = (size_t)nSys * (sizeof(SpmmArgs) + sizeof(RestrictBArgs) + sizeof(CoarseBArgs) +
                               sizeof(ProlongBArgs)) +
               4 * sizeof(int) * (size_t)(nSys + 1);
    T.vbytes = (T.vbytes + 255) & ~(size_t)255;
    CK(cudaMallocAsync(reinterpret_cast<void **>(&T.dev), T.vbytes * T.versions, st));
    CK(cudaMallocHost(reinterpret_cast<void **>(&T.host), T.vbytes * T.versions));
    return XDCG_OK;
}

xdcg_status sys_tables_build(SysTables &T, BatchRun *runs, int nSys, cudaStream_t st,
                             BatchSysTab *tab) {
    if (T.used >= T.versions) return XDCG_CUDA_ERROR;
    const size_t base = T.vbytes * T.used++;
    unsigned char *h = T.host + base, *d = T.dev + base;
    int nLive = 0;
    for (int s = 0; s < nSys; ++s) nLive += runs[s].live;
    auto *hs = reinterpret_cast<SpmmArgs *>(h);
    auto *hr = reinterpret_cast<RestrictBArgs *>(hs + nLive);
    auto *hc = reinterpret_cast<CoarseBArgs *>(hr + nLive);
    auto *hp = reinterpret_cast<ProlongBArgs *>(hc + nLive);
    int *ho = reinterpret_cast<int *>(hp + nLive);
    int *off[4];
    for (int q = 0; q < 4; ++q) {
        off[q] = ho + q * (nLive + 1);
        off[q][0] = 0;
    }
    int i = 0;
    for (int s = 0; s < nSys; ++s) {
        if (!runs[s].live) continue;
        const BatchRun &R = runs[s];
        hs[i] = R.spmm;
        hr[i] = R.rst;
        hc[i] = R.crs;
        hp[i] = R.pro;
        off[0][i + 1] = off[0][i] + R.spmm.A.grid;
        off[1][i + 1] = off[1][i] + R.rst.B.nUnits;
        off[2][i + 1] = off[2][i] + coarse_b_blocks(R.crs.k, R.c->bMB);
        off[3][i + 1] = off[3][i] + R.pro.B.nPUnits;
        ++i;
    }
    const size_t used = reinterpret_cast<unsigned char *>(ho + 4 * (nLive + 1)) - h;
    CK(cudaMemcpyAsync(d, h, used, cudaMemcpyHostToDevice, st));
    tab->nSys = nLive;
    tab->spmm = reinterpret_cast<const SpmmArgs *>(d);
    tab->rst = reinterpret_cast<const RestrictBArgs *>(d + ((unsigned char *)hr - h));
    tab->crs = reinterpret_cast<const CoarseBArgs *>(d + ((unsigned char *)hc - h));
    tab->pro = reinterpret_cast<const ProlongBArgs *>(d + ((unsigned char *)hp - h));
    for (int q = 0; q < 4; ++q) {
        tab->off[q] = reinterpret_cast<const int *>(d + ((unsigned char *)off[q] - h));
        tab->blocks[q] = off[q][nLive];
    }
    return XDCG_OK;
}

template <int MB>
xdcg_status solve_batches(BatchRun *runs, int nSys, cudaStream_t st, xdcg_status *status) {
    xdcg_ctx *c0 = runs[0].c;
    xdcg_status s;
    // ||f_j||^2 of every column of every system, one wait
    for (int q = 0; q < nSys; ++q) {
        xdcg_ctx *c = runs[q].c;
        const long long n = c->n;
        launch_batch_slots(c->bSlots, (1u << runs[q].m) - 1u, st);
        for (int j = 0; j < runs[q].m; ++j)
            launch_dot<double>(runs[q].F + j * n, runs[q].F + j * n, n, c->partials,
                               c->bSlots + j, kFinStore, 0, st);
        c->launches += 1 + runs[q].m;
        CK(cudaMemcpyAsync(c->h_slots, c->bSlots, sizeof(Scalars) * runs[q].m,
                           cudaMemcpyDeviceToHost, st));
    }
    CK(cudaStreamSynchronize(st));
    int nLive = 0;
    for (int q = 0; q < nSys; ++q) {
        if ((s = batch_start<MB>(runs[q], st)) != XDCG_OK) return s;
        nLive += runs[q].live;
    }
    const bool multi = nSys > 1;
    SysTables T;
    BatchSysTab tab{};
    if (multi && nLive > 0) {
        if ((s = sys_tables_init(T, nSys, st)) != XDCG_OK) return s;
        if ((s = sys_tables_build(T, runs, nSys, st, &tab)) != XDCG_OK) return s;
    }
    long long maxTicks = 16;
    for (int q = 0; q < nSys; ++q) {
        const xdcg_options &o = runs[q].c->opt;
        maxTicks = std::max(maxTicks, (long long)kMaxBatch *
                                          ((long long)o.max_iter / kTick + 2LL * o.max_outer + 2));
    }
    // Per system: iterating (its snapshot read each tick), replacing (over
    // several systems: held, its replacement on its own context's stream
    // while the others iterate; back when that stream's event has fired) or
    // done.
    enum { kSysRun, kSysRepl, kSysDone };
    std::vector<int> state(nSys), snapOk(nSys, 0);
    struct Events {
        std::vector<cudaEvent_t> v;
        ~Events() {
            for (auto e : v)
                if (e) cudaEventDestroy(e);
        }
    } evHold, evRepl;
    if (multi) {
        evHold.v.assign(nSys, nullptr);
        evRepl.v.assign(nSys, nullptr);
        for (int q = 0; q < nSys; ++q) {
            CK(cudaEventCreateWithFlags(&evHold.v[q], cudaEventDisableTiming));
            CK(cudaEventCreateWithFlags(&evRepl.v[q], cudaEventDisableTiming));
        }
    }
    for (int q = 0; q < nSys; ++q) state[q] = runs[q].live ? kSysRun : kSysDone;
    auto drain = [&]() {
        for (int q = 0; q < nSys; ++q) cudaStreamSynchronize(runs[q].c->st);
        cudaStreamSynchronize(st);
    };
    // a tick's iterations, enqueued on s
    auto enqueueTick = [&](cudaStream_t s) {
        for (int i = 0; i < kTick; ++i) {
            if (multi) {
                launch_iteration_sys<MB>(tab, s);
                c0->launches += 5;
            } else {
                launch_spmm<MB>(runs[0].spmm, s);
                launch_restrict_b<MB>(runs[0].rst, s);
                launch_coarse_b<MB>(runs[0].crs, s);
                launch_prolong_b<MB>(runs[0].pro, s);
                c0->launches += 4;
            }
        }
    };
    // opt.graph (of the first context): the tick as one recorded graph,
    // recorded again whenever the set of live systems (the table) changes
    struct TickGraph {
        LoopGraph g;
        ~TickGraph() {
            if (g.exec) cudaGraphExecDestroy(g.exec);
        }
    } tickG;
    const bool useGraph = c0->opt.graph != 0;
    xdcg_status status_all = XDCG_OK;
    bool snap = false;
    for (long long tick = 0; nLive > 0; ++tick) {
        if (tick > maxTicks) {
            status_all = XDCG_NO_CONVERGENCE;
            break;
        }
        int nRun = 0;
        for (int q = 0; q < nSys; ++q) nRun += state[q] == kSysRun;
        if (nRun > 0 && useGraph) {
            const LoopKey key{tab.spmm, tab.rst, tab.crs, tab.pro,
                              reinterpret_cast<const void *>((intptr_t)tab.nSys), runs[0].c,
                              reinterpret_cast<const void *>((intptr_t)runs[0].m), nullptr};
            if ((s = loop_graph(c0, tickG.g, key, enqueueTick)) != XDCG_OK) {
                if (multi) drain();
                return s;
            }
            CK(cudaGraphLaunch(tickG.g.exec, st));
            c0->launches += tickG.g.launches;
            c0->graphLaunches++;
        } else if (nRun > 0) {
            enqueueTick(st);
        }
        if (nRun == 0) {
            // every live system is replacing: wait for one
            for (int q = 0; q < nSys; ++q)
                if (state[q] == kSysRepl) {
                    CK(cudaEventSynchronize(evRepl.v[q]));
                    break;
                }
        } else if (snap) {
            CK(cudaEventSynchronize(c0->evb[(tick - 1) & 1]));
        }
        bool changed = false;
        for (int q = 0; q < nSys; ++q) {
            BatchRun &R = runs[q];
            if (state[q] == kSysRepl) {
                const cudaError_t e = cudaEventQuery(evRepl.v[q]);
                if (e == cudaSuccess) {
                    state[q] = kSysRun;
                    snapOk[q] = 0;
                } else if (e != cudaErrorNotReady) {
                    return XDCG_CUDA_ERROR;
                }
                continue;
            }
            if (state[q] != kSysRun || !snapOk[q]) continue;
            const BatchScalars &hb = *R.c->h_bs;
            if (hb.done == kFault || hb.fault) {
                drain();
                return XDCG_TIMEOUT;
            }
            unsigned M = 0;
            int nAct = 0;
            for (int j = 0; j < R.m; ++j)
                if (hb.active[j]) {
                    ++nAct;
                    if (hb.pend[j]) M |= 1u << j;
                }
            if (nAct == 0) {
                R.live = false;
                state[q] = kSysDone;
                changed = true;
                --nLive;
            } else if (M && multi) {
                cudaStream_t sq = R.c->st;
                launch_batch_hold(R.c->bs, st);
                CK(cudaEventRecord(evHold.v[q], st));
                CK(cudaStreamWaitEvent(sq, evHold.v[q], 0));
                batch_replace<MB>(R, M, sq);
                CK(cudaEventRecord(evRepl.v[q], sq));
                c0->launches += 1;
                state[q] = kSysRepl;
                snapOk[q] = 0;
            } else if (M) {
                batch_replace<MB>(R, M, st);
            }
        }
        if (nLive == 0) break;
        if (changed && multi)
            if ((s = sys_tables_build(T, runs, nSys, st, &tab)) != XDCG_OK) return s;
        for (int q = 0; q < nSys; ++q)
            if (state[q] == kSysRun) {
                CK(cudaMemcpyAsync(runs[q].c->h_bs, runs[q].c->bs, sizeof(BatchScalars),
                                   cudaMemcpyDeviceToHost, st));
                snapOk[q] = 1;
            }
        CK(cudaEventRecord(c0->evb[tick & 1], st));
        snap = true;
    }
    if (multi) drain();
    CK(cudaStreamSynchronize(st));
    CK(cudaGetLastError());
    for (int q = 0; q < nSys; ++q) status[q] = status_all;
    return XDCG_OK;
}

xdcg_status do_solve(xdcg_ctx *c, const double *f, double *u, double tol, bool guess,
                     xdcg_result *out) {
    NvtxRange range(c->opt.precision == XDCG_MIXED ? "xdcg solve (mixed)" : "xdcg solve (fp64)");
    xdcg_result res{};
    res.bad_index = -1;
    if (tol <= 0) tol = c->opt.tol;
    const long long l0 = c->launches, g0 = c->graphLaunches;
    CK(cudaEventRecord(c->ev0, c->st));
    xdcg_status s = (c->opt.precision == XDCG_MIXED) ? solve_mixed(c, f, u, tol, guess, &res)
                                                    : solve_fp64(c, f, u, tol, guess, &res);
    if (s == XDCG_CUDA_ERROR) return s;
    CK(cudaEventRecord(c->ev1, c->st));
    CK(cudaEventSynchronize(c->ev1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
    res.t_solve_ms = ms;
    res.n_launches = c->launches - l0;
    res.n_graph_launches = (int32_t)(c->graphLaunches - g0);
    if (out) *out = res;
    return s;
}

void free_ctx(xdcg_ctx *c) {
    if (!c) return;
    for (void *p : c->allocs) cudaFree(p);
    for (void *p : c->temps) cudaFree(p);
    if (c->h_sc) cudaFreeHost(c->h_sc);
    if (c->h_bs) cudaFreeHost(c->h_bs);
    if (c->h_slots) cudaFreeHost(c->h_slots);
    if (c->h_done) cudaFreeHost(c->h_done);
    if (c->h_poll) cudaFreeHost(c->h_poll);
    for (auto e : c->evS) cudaEventDestroy(e);
    for (auto e : c->evE) cudaEventDestroy(e);
    for (auto e : c->evP) cudaEventDestroy(e);
    if (c->ev0) cudaEventDestroy(c->ev0);
    if (c->ev1) cudaEventDestroy(c->ev1);
    for (auto e : c->evb)
        if (e) cudaEventDestroy(e);
    for (auto &g : c->loop32)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    if (c->loop64.exec) cudaGraphExecDestroy(c->loop64.exec);
    if (c->capSt) cudaStreamDestroy(c->capSt);
    delete c;
}


// ---- set-up -----------------------------------------------------------------

// In-place FP64 inversion of the SPD matrices dims[m] x dims[m] at A + offs[m]
// (blocked symmetric sweeps, dense_inv.cu); a failing pivot sets *d_bad to
// the matrix index (badByMatrix) or the pivot index.  Tables and scratch are
// set-up temporaries.
xdcg_status dense_inverse(xdcg_ctx *c, double *A, const std::vector<int> &dims,
                          const std::vector<long long> &offs, int *d_bad, int badByMatrix) {
    const int nMat = (int)dims.size();
    if (nMat == 0) return XDCG_OK;
    std::vector<int> tileOff(nMat + 1, 0), rowTileOff(nMat + 1, 0);
    std::vector<long long> cOff(nMat, 0);
    long long cTot = 0, nEnt = 0;
    int maxDim = 0;
    for (int m = 0; m < nMat; ++m) {
        const int T = dense_inv_tiles(dims[m]);
        if ((long long)tileOff[m] + (long long)T * (T + 1) / 2 > INT_MAX) return XDCG_INVALID_ARG;
        tileOff[m + 1] = tileOff[m] + T * (T + 1) / 2;
        rowTileOff[m + 1] = rowTileOff[m] + T;
        cOff[m] = cTot;
        cTot += (long long)dense_inv_panel_doubles(dims[m]);
        nEnt = std::max(nEnt, offs[m] + (long long)dims[m] * dims[m]);
        maxDim = std::max(maxDim, dims[m]);
    }
    DenseBatch B;
    B.nMat = nMat;
    B.nTiles = tileOff[nMat];
    B.nRowTiles = rowTileOff[nMat];
    B.dim = upload_tmp(c, dims);
    B.off = upload_tmp(c, offs);
    B.tileOff = upload_tmp(c, tileOff);
    B.rowTileOff = upload_tmp(c, rowTileOff);
    B.cOff = upload_tmp(c, cOff);
    B.A = A;
    B.D = dalloc_tmp<double>(c, (size_t)nMat * dense_inv_pivot_doubles());
    B.C = dalloc_tmp<double>(c, (size_t)cTot);
    B.thr = dalloc_tmp<double>(c, nMat);
    B.bad = d_bad;
    B.badByMatrix = badByMatrix;
    if (!B.dim || !B.off || !B.tileOff || !B.rowTileOff || !B.cOff || !B.D || !B.C || !B.thr)
        return XDCG_OOM;
    CK(launch_dense_inverse(B, maxDim, nEnt, 1e-14, c->st));
    return XDCG_OK;
}

xdcg_status setup_impl(xdcg_ctx *c, const xdcg_matrix *K, const xdcg_deflation *Zd,
                       const xdcg_blocks *blocks, int *bad, const xdcg_ctx *prev) {
    // wall time of each set-up phase (device work waited for at each mark)
    auto tPrev = std::chrono::steady_clock::now();
    auto mark = [&](int phase) -> bool {
        if (cudaStreamSynchronize(c->st) != cudaSuccess) return false;
        const auto now = std::chrono::steady_clock::now();
        c->info.t_setup_phase_ms[phase] +=
            std::chrono::duration<double, std::milli>(now - tPrev).count();
        tPrev = now;
        return true;
    };
    const int N = K->n_nodes;
    if (N <= 0 || !K->dof_ptr || !K->row_ptr) return XDCG_INVALID_ARG;
    if ((K->mem != XDCG_HOST && K->mem != XDCG_DEVICE) ||
        (Zd->mem != XDCG_HOST && Zd->mem != XDCG_DEVICE))
        return XDCG_INVALID_ARG;
    std::vector<int> dof, rowp, col;
    std::vector<long long> vptr;
    std::vector<double> val;
    if (!fetch(dof, K->dof_ptr, N + 1, K->mem) || !fetch(rowp, K->row_ptr, N + 1, K->mem))
        return XDCG_INVALID_ARG;
    if (dof[0] != 0 || rowp[0] != 0) return XDCG_INVALID_ARG;
    for (int I = 0; I < N; ++I) {
        const int b = dof[I + 1] - dof[I];
        if (b != 3 && b != 6 && b != 15) return XDCG_INVALID_ARG;
        if (rowp[I + 1] < rowp[I]) return XDCG_INVALID_ARG;
    }
    const long long nnzb = rowp[N];
    if (!fetch(col, K->col, nnzb, K->mem)) return XDCG_INVALID_ARG;
    std::vector<int64_t> vp64;
    if (!fetch(vp64, K->val_ptr, nnzb + 1, K->mem)) return XDCG_INVALID_ARG;
    vptr.assign(vp64.begin(), vp64.end());
    if (vptr[0] != 0) return XDCG_INVALID_ARG;
    std::atomic<bool> badInput{false};
    parallel_for(N, [&](long long i0, long long i1) {
        for (long long I = i0; I < i1 && !badInput; ++I) {
            bool diag = false;
            for (long long p = rowp[I]; p < rowp[I + 1]; ++p) {
                const int J = col[p];
                if (J < 0 || J >= N || (p > rowp[I] && col[p - 1] >= J) ||
                    vptr[p + 1] - vptr[p] !=
                        (long long)(dof[I + 1] - dof[I]) * (dof[J + 1] - dof[J])) {
                    badInput = true;
                    break;
                }
                if (J == I) diag = true;
            }
            if (!diag) badInput = true;
        }
    });
    if (badInput) return XDCG_INVALID_ARG;
    // values: read in place from host memory, fetched from device memory
    const long long nval = vptr[nnzb];
    const double *valp = nullptr;
    if (K->mem == XDCG_DEVICE) {
        if (!fetch(val, K->val, nval, K->mem)) return XDCG_INVALID_ARG;
        valp = val.data();
    } else {
        if (nval > 0 && !K->val) return XDCG_INVALID_ARG;
        valp = K->val;
    }
    std::vector<double> vmaxPart(16, 0.0);
    std::atomic<int> piece{0};
    parallel_for(nval, [&](long long i0, long long i1) {
        double m = 0.0;
        for (long long i = i0; i < i1; ++i) {
            const double v = valp[i];
            if (!std::isfinite(v)) {
                badInput = true;
                return;
            }
            m = std::max(m, std::fabs(v));
        }
        vmaxPart[piece++] = m;
    });
    if (badInput) return XDCG_INVALID_ARG;
    const double vmax = *std::max_element(vmaxPart.begin(), vmaxPart.end());
    // symmetry of pattern and values
    parallel_for(N, [&](long long i0, long long i1) {
        for (long long I = i0; I < i1 && !badInput; ++I) {
            const int bI = dof[I + 1] - dof[I];
            for (long long p = rowp[I]; p < rowp[I + 1]; ++p) {
                const int J = col[p];
                if (J < I) continue;
                const int bJ = dof[J + 1] - dof[J];
                const int *beg = &col[rowp[J]], *end = &col[0] + rowp[J + 1];
                const int *it = std::lower_bound(beg, end, (int)I);
                if (it == end || *it != I) {
                    badInput = true;
                    return;
                }
                const long long q = rowp[J] + (it - beg);
                for (int a = 0; a < bI; ++a)
                    for (int b2 = 0; b2 < bJ; ++b2)
                        if (std::fabs(valp[vptr[p] + a * bJ + b2] - valp[vptr[q] + b2 * bI + a]) >
                            1e-12 * vmax) {
                            badInput = true;
                            return;
                        }
            }
        }
    });
    if (badInput) return XDCG_INVALID_ARG;
    // deflation description
    const int S = Zd->n_sub;
    if (S <= 0) return XDCG_INVALID_ARG;
    std::vector<int> sub;
    std::vector<double> coords, centre;
    std::vector<int8_t> hs;
    // valued form: the caller's Z blocks per node (6 or 12 columns per box);
    // geometric form: coordinates, H signs and box centres
    const bool valued = Zd->values != nullptr;
    std::vector<int> subCols;
    std::vector<double> zval;
    std::vector<long long> zvOff(N + 1, 0);
    if (!fetch(sub, Zd->sub_of_node, N, Zd->mem)) return XDCG_INVALID_ARG;
    for (int I = 0; I < N; ++I)
        if (sub[I] < 0 || sub[I] >= S) return XDCG_INVALID_ARG;
    if (valued) {
        if (!fetch(subCols, Zd->sub_cols, S, Zd->mem)) return XDCG_INVALID_ARG;
        for (int s2 = 0; s2 < S; ++s2)
            if (subCols[s2] != 6 && subCols[s2] != 12) return XDCG_INVALID_ARG;
        for (int I = 0; I < N; ++I)
            zvOff[I + 1] = zvOff[I] + (long long)(dof[I + 1] - dof[I]) * subCols[sub[I]];
        if (!fetch(zval, Zd->values, (size_t)zvOff[N], Zd->mem)) return XDCG_INVALID_ARG;
        for (double v : zval)
            if (!std::isfinite(v)) return XDCG_INVALID_ARG;
        coords.assign(3 * (size_t)N, 0.0);
        hs.assign(N, 1);
        centre.assign(3 * (size_t)S, 0.0);
    } else {
        if (!fetch(coords, Zd->coords, 3 * (size_t)N, Zd->mem) || !fetch(hs, Zd->hsign, N, Zd->mem) ||
            !fetch(centre, Zd->centre, 3 * (size_t)S, Zd->mem))
            return XDCG_INVALID_ARG;
        for (int I = 0; I < N; ++I) {
            if (hs[I] != 1 && hs[I] != -1) return XDCG_INVALID_ARG;
            for (int e = 0; e < 3; ++e)
                if (!std::isfinite(coords[3 * I + e])) return XDCG_INVALID_ARG;
        }
    }

    c->nNodes = N;
    c->n = dof[N];
    c->nBox = S;
    const long long n = c->n;

    // caller blocks: contiguous dof ranges of whole nodes, each at most
    // XDCG_MAX_BLOCK_DOFS dofs
    std::vector<int> bptr, bNode0, bNode1, blockOfNode;
    if (blocks) {
        const int nb = blocks->n_blocks;
        if (nb < 1 || nb > N || (blocks->mem != XDCG_HOST && blocks->mem != XDCG_DEVICE) ||
            !fetch(bptr, blocks->dof_ptr, (size_t)nb + 1, blocks->mem))
            return XDCG_INVALID_ARG;
        if (bptr[0] != 0 || bptr[nb] != n) return XDCG_INVALID_ARG;
        bNode0.resize(nb);
        bNode1.resize(nb);
        blockOfNode.resize(N);
        for (int b = 0; b < nb; ++b) {
            const int d0 = bptr[b], d1 = bptr[b + 1];
            if (d1 <= d0 || d1 - d0 > XDCG_MAX_BLOCK_DOFS) return XDCG_INVALID_ARG;
            const auto i0 = std::lower_bound(dof.begin(), dof.end(), d0);
            const auto i1 = std::lower_bound(dof.begin(), dof.end(), d1);
            if (i0 == dof.end() || *i0 != d0 || i1 == dof.end() || *i1 != d1)
                return XDCG_INVALID_ARG;   // a boundary inside a node
            bNode0[b] = (int)(i0 - dof.begin());
            bNode1[b] = (int)(i1 - dof.begin());
            for (int I = bNode0[b]; I < bNode1[b]; ++I) blockOfNode[I] = b;
        }
    }

    if (!mark(0)) return XDCG_CUDA_ERROR;   // validation
    // ---- chunk rows: S (pure standard) and X (the rest)
    std::vector<int> kindb(N);
    for (int I = 0; I < N; ++I) kindb[I] = dof[I + 1] - dof[I];
    std::vector<int> sRows, xRows;
    std::vector<int> rowNode, rowPart;   // per chunk row: node and chunk within node
    const long long nChunks = n / 3;
    rowNode.resize(nChunks);
    rowPart.resize(nChunks);
    for (int I = 0; I < N; ++I)
        for (int ci = 0; ci < kindb[I] / 3; ++ci) {
            rowNode[dof[I] / 3 + ci] = I;
            rowPart[dof[I] / 3 + ci] = ci;
        }
    std::vector<char> pure(N, 0);
    for (int I = 0; I < N; ++I) {
        bool ok = kindb[I] == 3;
        for (long long p = rowp[I]; ok && p < rowp[I + 1]; ++p) ok = kindb[col[p]] == 3;
        pure[I] = ok;
    }
    std::vector<int> rowLen(nChunks, 0);
    parallel_for(nChunks, [&](long long r0, long long r1) {
        for (long long r = r0; r < r1; ++r) {
            const int I = rowNode[r];
            int len = 0;
            for (long long p = rowp[I]; p < rowp[I + 1]; ++p) len += kindb[col[p]] / 3;
            rowLen[r] = len;
        }
    });
    for (long long r = 0; r < nChunks; ++r) {
        const int I = rowNode[r];
        if (pure[I] && rowPart[r] == 0)
            sRows.push_back((int)r);
        else
            xRows.push_back((int)r);
    }
    // blocks of chunk row r in column order: (col chunk, pointer to 3x3 source)
    auto for_blocks = [&](long long r, auto &&fn) {
        const int I = rowNode[r], ci = rowPart[r];
        const int bI = kindb[I];
        int t = 0;
        for (long long p = rowp[I]; p < rowp[I + 1]; ++p) {
            const int J = col[p];
            const int bJ = kindb[J];
            for (int cj = 0; cj < bJ / 3; ++cj, ++t) {
                int blk[9];   // positions of the 3x3 block's entries in val
                for (int a = 0; a < 3; ++a)
                    for (int b2 = 0; b2 < 3; ++b2)
                        blk[a * 3 + b2] = (int)(vptr[p] + (3 * ci + a) * bJ + 3 * cj + b2);
                fn(t, dof[J] / 3 + cj, blk);
            }
        }
        (void)bI;
    };
    // sliced-ELL layouts: S rows in natural order, X rows sorted by length
    // X rows: bucketed by length (so a slice pads little), in natural order
    // within a bucket (so a slice's rows are spatial neighbours and the x
    // gathers of one step coalesce)
    std::stable_sort(xRows.begin(), xRows.end(), [&](int a, int b) {
        const int ba = rowLen[a] / kXBucket, bb = rowLen[b] / kXBucket;
        return ba != bb ? ba > bb : a < b;
    });
    struct SellHost {
        std::vector<int> row, len, col, src;
        std::vector<long long> slicePtr;
        int nSlices = 0;
    };
    // chunkMap (may be null) renumbers the chunk rows and columns written
    auto build_sell = [&](const std::vector<int> &rows, int tpr, SellHost &H,
                          const std::vector<int> *chunkMap) {
        const int rpw = 32 / tpr;
        const int nr = (int)rows.size();
        H.nSlices = (nr + rpw - 1) / rpw;
        H.row = rows;
        if (chunkMap)
            for (int &r : H.row) r = (*chunkMap)[r];
        H.len.resize(nr);
        H.slicePtr.assign(H.nSlices + 1, 0);
        for (int sl = 0; sl < H.nSlices; ++sl) {
            int mx = 0;
            for (int q = 0; q < rpw && sl * rpw + q < nr; ++q) mx = std::max(mx, rowLen[rows[sl * rpw + q]]);
            H.slicePtr[sl + 1] = H.slicePtr[sl] + 32LL * std::max(1, (mx + tpr - 1) / tpr);
        }
        const long long slots = std::max<long long>(H.slicePtr[H.nSlices], 1);
        H.col.resize(slots);
        H.src.resize(9 * (size_t)slots);
        // slices write disjoint ranges of col, src and len
        parallel_for(H.nSlices, [&](long long sl0, long long sl1) {
          for (long long sl = sl0; sl < sl1; ++sl) {
            const long long base = H.slicePtr[sl];
            std::fill(H.col.begin() + base, H.col.begin() + H.slicePtr[sl + 1], 0);
            std::fill(H.src.begin() + 9 * base, H.src.begin() + 9 * H.slicePtr[sl + 1], -1);
            const long long steps = (H.slicePtr[sl + 1] - base) / 32;
            auto cidx = [&](long long st2, int lane) { return base + st2 * 32 + lane; };
            auto vidx = [&](long long st2, int e, int lane) {
                return 9 * base + (st2 * 9 + e) * 32 + lane;
            };
            for (int q = 0; q < rpw && sl * rpw + q < nr; ++q) {
                const int r = rows[sl * rpw + q];
                H.len[sl * rpw + q] = rowLen[r];
                const int rOut = chunkMap ? (*chunkMap)[r] : r;
                for (long long st2 = 0; st2 < steps; ++st2)
                    for (int h = 0; h < tpr; ++h) H.col[cidx(st2, q + rpw * h)] = rOut;
                for_blocks(r, [&](int t, int cc, const int *blk) {
                    const long long st2 = t / tpr;
                    const int lane = q + rpw * (t % tpr);
                    H.col[cidx(st2, lane)] = chunkMap ? (*chunkMap)[cc] : cc;
                    for (int e = 0; e < 9; ++e) H.src[vidx(st2, e, lane)] = blk[e];
                });
            }
          }
        });
        if (H.nSlices == 0) {
            H.col[0] = 0;
            std::fill(H.src.begin(), H.src.end(), -1);
        }
    };
    SellHost HS, HX;
    build_sell(sRows, kTprS, HS, nullptr);
    build_sell(xRows, kTprX, HX, nullptr);
    const int nS = (int)sRows.size(), nX = (int)xRows.size();
    long long nnzb3 = 0;
    for (long long r = 0; r < nChunks; ++r) nnzb3 += rowLen[r];

    // ---- node lists and diagonal blocks
    std::vector<int> lists[3];
    for (int I = 0; I < N; ++I) lists[kindb[I] == 3 ? 0 : (kindb[I] == 6 ? 1 : 2)].push_back(I);
    const int Bsz[3] = {3, 6, 15};
    std::vector<double> Dsoa[3];
    // block Jacobi factors the node blocks; point Jacobi only their diagonals
    const bool pointJacobi = c->opt.jacobi == XDCG_POINT_JACOBI;
    for (int t = 0; t < 3; ++t) {
        const int B = Bsz[t], cnt = (int)lists[t].size();
        Dsoa[t].assign((size_t)B * B * std::max(cnt, 1), 0.0);
        for (int i = 0; i < cnt; ++i) {
            const int I = lists[t][i];
            long long pd = -1;
            for (long long p = rowp[I]; p < rowp[I + 1]; ++p)
                if (col[p] == I) pd = p;
            for (int e = 0; e < B * B; ++e)
                Dsoa[t][(size_t)e * cnt + i] =
                    (pointJacobi && e / B != e % B) ? 0.0 : valp[vptr[pd] + e];
        }
    }
    // each node's block as factored, for a later update of this context
    c->hostKind.assign(kindb.begin(), kindb.end());
    c->hostListPos.assign(N, 0);
    c->hostDiagOff.assign(N + 1, 0);
    for (int I = 0; I < N; ++I) c->hostDiagOff[I + 1] = c->hostDiagOff[I] + (long long)kindb[I] * kindb[I];
    c->hostDiag.resize((size_t)c->hostDiagOff[N]);
    for (int t = 0; t < 3; ++t) {
        const int B = Bsz[t], cnt = (int)lists[t].size();
        for (int i = 0; i < cnt; ++i) {
            const int I = lists[t][i];
            c->hostListPos[I] = i;
            for (int e = 0; e < B * B; ++e)
                c->hostDiag[c->hostDiagOff[I] + e] = Dsoa[t][(size_t)e * cnt + i];
        }
    }
    // an update reuses the factor of every node whose kind and block are
    // unchanged (bitwise) since the previous context
    const bool reuse = prev && prev->nNodes == N && prev->opt.jacobi == c->opt.jacobi &&
                       (int)prev->hostKind.size() == N;
    std::vector<int> fresh[3], freshPos[3], keepSrc[3], keepDst[3];
    for (int t = 0; t < 3; ++t) {
        const int B = Bsz[t];
        for (int i = 0; i < (int)lists[t].size(); ++i) {
            const int I = lists[t][i];
            const bool same =
                reuse && prev->hostKind[I] == B &&
                std::memcmp(&prev->hostDiag[prev->hostDiagOff[I]], &c->hostDiag[c->hostDiagOff[I]],
                            sizeof(double) * B * B) == 0;
            if (same) {
                keepSrc[t].push_back(prev->hostListPos[I]);
                keepDst[t].push_back(i);
            } else {
                fresh[t].push_back(I);
                freshPos[t].push_back(i);
            }
        }
        c->reusedFactors += (int)keepSrc[t].size();
    }

    // ---- boxes: own nodes, enriched-mode decision, coarse columns, W entries
    std::vector<int> ownPtr(S + 1, 0), ownNodes(N);
    for (int I = 0; I < N; ++I) ownPtr[sub[I] + 1]++;
    for (int s = 0; s < S; ++s) ownPtr[s + 1] += ownPtr[s];
    {
        std::vector<int> fill(ownPtr.begin(), ownPtr.end() - 1);
        for (int I = 0; I < N; ++I) ownNodes[fill[sub[I]]++] = I;
    }
    std::vector<int> menr(S, 0), col0(S + 1, 0);
    for (int s = 0; s < S; ++s) {
        if (valued) {
            menr[s] = subCols[s] == 12;
        } else if (Zd->enriched_modes) {
            std::vector<double> pts;
            for (int t = ownPtr[s]; t < ownPtr[s + 1]; ++t) {
                const int I = ownNodes[t];
                if (kindb[I] == 6)
                    for (int e = 0; e < 3; ++e) pts.push_back(coords[3 * I + e]);
            }
            menr[s] = pts.empty() ? 0 : (points_collinear(pts) ? 0 : 1);
        }
        col0[s + 1] = col0[s] + (menr[s] ? 12 : 6);
    }
    c->k = col0[S];
    const int k = c->k;
    // W entries: (box s, node I) for every node I coupled to a node of s;
    // ordered by box, then owner box of I, then I (segments of E)
    std::vector<std::vector<int>> extOf(S);
    {
        std::vector<int> mark(S, -1);
        for (int I = 0; I < N; ++I)
            for (long long p = rowp[I]; p < rowp[I + 1]; ++p) {
                const int s = sub[col[p]];
                if (mark[s] != I) { mark[s] = I; extOf[s].push_back(I); }
            }
    }
    std::vector<int> extPtr(S + 1, 0), extNode, extBox;
    std::vector<long long> wOff(1, 0);
    std::vector<int> segBox, segOwner, segBegin, segEnd;
    for (int s = 0; s < S; ++s) {
        auto &v = extOf[s];
        std::stable_sort(v.begin(), v.end(), [&](int a, int b) {
            return sub[a] != sub[b] ? sub[a] < sub[b] : a < b;
        });
        const int M = menr[s] ? 12 : 6;
        for (size_t i = 0; i < v.size(); ++i) {
            const int e = (int)extNode.size();
            if (i == 0 || sub[v[i]] != sub[v[i - 1]]) {
                segBox.push_back(s);
                segOwner.push_back(sub[v[i]]);
                segBegin.push_back(e);
                segEnd.push_back(e);
            }
            segEnd.back() = e + 1;
            extNode.push_back(v[i]);
            extBox.push_back(s);
            wOff.push_back(wOff.back() + (long long)kindb[v[i]] * M);
        }
        extPtr[s + 1] = (int)extNode.size();
    }
    const int nExt = (int)extNode.size();
    const long long nW = wOff.back();
    wOff.pop_back();

    if (!mark(1)) return XDCG_CUDA_ERROR;   // host layout
    // ---- upload and set-up kernels
    cudaStream_t st = c->st;
    c->mixed = c->opt.precision == XDCG_MIXED;
    const bool mixed = c->mixed;
    int *d_dof = upload(c, dof);
    int *d_sub = upload(c, sub);
    std::vector<signed char> hsc(hs.begin(), hs.end());
    signed char *d_hs = upload(c, hsc);
    int *d_col0 = upload(c, col0);
    int *d_menr = upload(c, menr);
    double *d_x64 = dalloc<double>(c, 3 * (size_t)N);
    if (!d_dof || !d_sub || !d_hs || !d_col0 || !d_menr || !d_x64) return XDCG_OOM;
    {
        double *d_coords = upload_tmp(c, coords), *d_centre = upload_tmp(c, centre);
        if (!d_coords || !d_centre) return XDCG_OOM;
        launch_xrel(N, d_coords, d_centre, d_sub, d_x64, nullptr, st);
    }
    KinDev kin;   // the input matrix on the device, for the set-up kernels
    kin.nNodes = N;
    kin.dofStart = d_dof;
    kin.rowPtr = upload_tmp(c, rowp);
    kin.col = upload_tmp(c, col);
    kin.valPtr = upload_tmp(c, vptr);
    double *d_val = dalloc_tmp<double>(c, (size_t)nval);
    if (d_val && nval > 0)
        CK(cudaMemcpyAsync(d_val, valp, (size_t)nval * sizeof(double), cudaMemcpyHostToDevice, st));
    kin.val = d_val;
    if (!kin.rowPtr || !kin.col || !kin.valPtr || !kin.val) return XDCG_OOM;
    // SpMV layouts: values gathered on the device through the index maps
    // structure of a SELL part; the values are gathered through *d_src
    auto upload_sell_structure = [&](const SellHost &H, auto &D, int **d_src) -> bool {
        D.nRows = (int)H.row.size();
        D.nSlices = H.nSlices;
        D.row = upload(c, H.row);
        D.len = upload(c, H.len);
        D.slicePtr = upload(c, H.slicePtr);
        D.col = upload(c, H.col);
        *d_src = upload_tmp(c, H.src);
        return D.row && D.len && D.slicePtr && D.col && *d_src;
    };
    auto upload_sell = [&](const SellHost &H, SellDev<double> &D, int **d_src) -> bool {
        if (!upload_sell_structure(H, D, d_src)) return false;
        double *v = dalloc<double>(c, H.src.size());
        D.val = v;
        if (!v) return false;
        launch_gather(*d_src, (long long)H.src.size(), d_val, v, nullptr, st);
        return true;
    };
    auto &A = c->L64.A;
    int *d_srcS = nullptr, *d_srcX = nullptr;
    if (!upload_sell(HS, A.S, &d_srcS) || !upload_sell(HX, A.X, &d_srcX)) return XDCG_OOM;
    // persistent SpMV grids and each warp's slice range, balanced by steps
    auto partition = [&](const SellHost &PS, const SellHost &PX, int grid) -> const int * {
        const int nW = grid * kSpmvWarps, nT = PS.nSlices + PX.nSlices;
        std::vector<long long> pre(nT + 1, 0);
        for (int i = 0; i < nT; ++i) {
            const SellHost &H = i < PS.nSlices ? PS : PX;
            const int sl = i < PS.nSlices ? i : i - PS.nSlices;
            pre[i + 1] = pre[i] + (H.slicePtr[sl + 1] - H.slicePtr[sl]) / 32;
        }
        std::vector<int> ws(nW + 1);
        int i = 0;
        for (int w = 0; w < nW; ++w) {
            const long long target = pre[nT] * w / nW;
            while (i < nT && pre[i + 1] <= target) ++i;
            if (i < nT && target - pre[i] > pre[i + 1] - target) ++i;
            ws[w] = i;
        }
        ws[nW] = nT;
        return upload(c, ws);
    };
    const unsigned long long waitNs = (unsigned long long)(c->opt.wait_s * 1e9);
    A.waitNs = waitNs;
    A.shape = kSpmvDefaultShapeF64;
    A.grid = spmv_persistent_grid<double>(HS.nSlices + HX.nSlices, A.shape);
    if (A.grid < 1) return XDCG_CUDA_ERROR;
    A.warpSlice = partition(HS, HX, A.grid);
    if (!A.warpSlice) return XDCG_OOM;
    c->info.spmv_shape_fp64 = A.shape;   // until autotuned or pinned below
    // The autotuner: every compiled pipeline shape of the SpMV (steps per
    // bulk-copy stage, stages per warp, blocks per SM; each with its own
    // persistent grid and step-balanced warp ranges) timed on this matrix,
    // the fastest kept.  Two warm-up launches and five timed ones (CUDA
    // events, median) per shape, x = 0 (the time does not depend on x).
    auto autotune = [&](auto &Ad, const SellHost &PS, const SellHost &PX, auto zero, double *usOut,
                        int32_t *pick) -> xdcg_status {
        using T = decltype(zero);
        const int nShapes = spmv_shape_count<T>();
        T *x = dalloc_tmp<T>(c, n), *y = dalloc_tmp<T>(c, n);
        double *parts = dalloc_tmp<double>(c, kMaxGrid);
        Scalars *scT = dalloc_tmp<Scalars>(c, 1);
        if (!x || !y || !parts || !scT) return XDCG_OOM;
        CK(cudaMemsetAsync(x, 0, n * sizeof(T), st));
        cudaEvent_t e0, e1;
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        double best = 1e300;
        SpmvDev<T> keep = Ad;
        for (int sh = 0; sh < nShapes && sh < 8; ++sh) {
            SpmvDev<T> cand = Ad;
            cand.shape = sh;
            cand.grid = spmv_persistent_grid<T>(PS.nSlices + PX.nSlices, sh);
            usOut[sh] = -1.0;
            if (cand.grid < 1 || cand.grid > kMaxGrid) continue;
            cand.warpSlice = sh == Ad.shape ? Ad.warpSlice : partition(PS, PX, cand.grid);
            if (!cand.warpSlice) return XDCG_OOM;
            std::vector<float> t;
            for (int rep = 0; rep < 7; ++rep) {
                init_scalars(c, scT, -1.0, nullptr, INT_MAX);
                CK(cudaEventRecord(e0, st));
                launch_spmv<T>(cand, x, y, nullptr, 0, parts, scT, kFinStore, 0, st);
                CK(cudaEventRecord(e1, st));
                CK(cudaEventSynchronize(e1));
                float ms = 0.f;
                CK(cudaEventElapsedTime(&ms, e0, e1));
                if (rep >= 2) t.push_back(ms);
            }
            std::sort(t.begin(), t.end());
            usOut[sh] = 1e3 * t[t.size() / 2];
            if (usOut[sh] < best) {
                best = usOut[sh];
                keep = cand;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        Ad = keep;
        *pick = keep.shape;
        return XDCG_OK;
    };
    // a shape pinned by the caller (options.spmv_shape_fp32 / _fp64 >= 0)
    // replaces the default or the autotuner's pick
    auto pin = [&](auto &Ad, const SellHost &PS, const SellHost &PX, auto zero, int sh,
                   int32_t *pick) -> xdcg_status {
        using T = decltype(zero);
        if (sh < 0 || sh == Ad.shape) return XDCG_OK;
        SpmvDev<T> cand = Ad;
        cand.shape = sh;
        cand.grid = spmv_persistent_grid<T>(PS.nSlices + PX.nSlices, sh);
        if (cand.grid < 1 || cand.grid > kMaxGrid) return XDCG_CUDA_ERROR;
        cand.warpSlice = partition(PS, PX, cand.grid);
        if (!cand.warpSlice) return XDCG_OOM;
        Ad = cand;
        *pick = sh;
        return XDCG_OK;
    };
    for (int sh = 0; sh < 8; ++sh) c->info.spmv_shape_us_fp64[sh] = c->info.spmv_shape_us_fp32[sh] = -1.0;
    if (c->opt.autotune) {
        xdcg_status ts = autotune(A, HS, HX, 0.0, c->info.spmv_shape_us_fp64,
                                  &c->info.spmv_shape_fp64);
        if (ts != XDCG_OK) return ts;
    }
    {
        xdcg_status ts = pin(A, HS, HX, 0.0, c->opt.spmv_shape_fp64, &c->info.spmv_shape_fp64);
        if (ts != XDCG_OK) return ts;
    }

    if (!mark(2)) return XDCG_CUDA_ERROR;   // uploads, SpMV values
    // node data and block factors (FP64)
    // failure slots: [0] node block (node), [1] coarse pivot, [2] caller block
    int *d_bad = dalloc<int>(c, 3);
    if (!d_bad) return XDCG_OOM;
    {
        std::vector<int> init = {INT_MAX, INT_MAX, INT_MAX};
        CK(cudaMemcpyAsync(d_bad, init.data(), 3 * sizeof(int), cudaMemcpyHostToDevice, st));
        CK(cudaStreamSynchronize(st));
    }
    auto &N64 = c->L64.N;
    N64.nNodes = N;
    N64.nStd = (int)lists[0].size();
    N64.nH = (int)lists[1].size();
    N64.nT = (int)lists[2].size();
    N64.dofStart = d_dof;
    N64.sub = d_sub;
    N64.xrel = d_x64;
    N64.hsign = d_hs;
    N64.col0 = d_col0;
    N64.menr = d_menr;
    const int *dl[3];
    double *L64[3];
    for (int t = 0; t < 3; ++t) {
        const int B = Bsz[t], cnt = (int)lists[t].size();
        dl[t] = upload(c, lists[t]);
        L64[t] = dalloc<double>(c, (size_t)B * (B + 1) / 2 * std::max(cnt, 1));
        if (!dl[t] || !L64[t]) return XDCG_OOM;
        if (reuse) {
            // carried-over factors, then only the changed nodes factored
            const int nf = (int)fresh[t].size(), nk = (int)keepSrc[t].size();
            const double *Lprev = t == 0 ? prev->L64.N.Lstd : (t == 1 ? prev->L64.N.Lh : prev->L64.N.Lt);
            const int prevCnt = t == 0 ? prev->L64.N.nStd : (t == 1 ? prev->L64.N.nH : prev->L64.N.nT);
            if (nk > 0) {
                int *d_src = upload_tmp(c, keepSrc[t]), *d_dst = upload_tmp(c, keepDst[t]);
                if (!d_src || !d_dst) return XDCG_OOM;
                launch_copy_factors(nk, B * (B + 1) / 2, d_src, d_dst, Lprev, prevCnt, L64[t], cnt,
                                    st);
            }
            if (nf > 0) {
                std::vector<double> Df((size_t)B * B * nf);
                for (int j = 0; j < nf; ++j)
                    for (int e = 0; e < B * B; ++e)
                        Df[(size_t)e * nf + j] = Dsoa[t][(size_t)e * cnt + freshPos[t][j]];
                int *d_nodes = upload_tmp(c, fresh[t]), *d_pos = upload_tmp(c, freshPos[t]);
                double *d_D = upload_tmp(c, Df);
                if (!d_nodes || !d_pos || !d_D) return XDCG_OOM;
                launch_block_cholesky(B, nf, d_nodes, d_D, L64[t], nullptr, d_bad, st, d_pos, cnt);
            }
            continue;
        }
        double *d_D = upload_tmp(c, Dsoa[t]);
        if (!d_D) return XDCG_OOM;
        launch_block_cholesky(B, cnt, dl[t], d_D, L64[t], nullptr, d_bad, st);
    }
    N64.stdNodes = dl[0]; N64.hNodes = dl[1]; N64.tNodes = dl[2];
    N64.Lstd = L64[0]; N64.Lh = L64[1]; N64.Lt = L64[2];

    // W = K Z and E = Z^T W
    int *d_extBox = upload_tmp(c, extBox), *d_extNode = upload(c, extNode);
    int *d_extPtr = upload(c, extPtr), *d_ownPtr = upload(c, ownPtr), *d_own = upload(c, ownNodes);
    long long *d_wOff = upload(c, wOff);
    double *d_W = dalloc<double>(c, nW);
    if (!d_extBox || !d_extNode || !d_extPtr || !d_ownPtr || !d_own || !d_wOff || !d_W)
        return XDCG_OOM;
    // Z by value: the caller's blocks for the set-up kernels (node order) and,
    // in box order, for the FP64 restriction and prolongation
    ZvalDev zv{nullptr, nullptr};
    double *d_zslot = nullptr;
    long long *d_zslotOff = nullptr;
    if (valued) {
        zv.v = upload_tmp(c, zval);
        zv.off = upload_tmp(c, zvOff);
        std::vector<double> zslot;
        std::vector<long long> zslotOff(N);
        zslot.reserve(zval.size());
        for (int t = 0; t < N; ++t) {
            const int I = ownNodes[t];
            zslotOff[t] = (long long)zslot.size();
            zslot.insert(zslot.end(), zval.begin() + zvOff[I], zval.begin() + zvOff[I + 1]);
        }
        d_zslot = upload(c, zslot);
        d_zslotOff = upload(c, zslotOff);
        if (!zv.v || !zv.off || !d_zslot || !d_zslotOff) return XDCG_OOM;
    }
    launch_build_W(kin, nExt, d_extBox, d_extNode, d_wOff, d_sub, d_x64, d_hs, d_menr, zv, d_W,
                   st);
    // node data in box order (slots) and per-entry dof data for the box kernels
    std::vector<int> ownDof(N), extDof(nExt);
    std::vector<unsigned char> ownB(N), extB(nExt);
    std::vector<signed char> ownH(N);
    std::vector<double> ownCoords(3 * (size_t)N);
    std::vector<int> ownSub(N);
    for (int t = 0; t < N; ++t) {
        const int I = ownNodes[t];
        ownDof[t] = dof[I];
        ownB[t] = (unsigned char)kindb[I];
        ownH[t] = (signed char)hs[I];
        ownSub[t] = sub[I];
        for (int e = 0; e < 3; ++e) ownCoords[3 * (size_t)t + e] = coords[3 * (size_t)I + e];
    }
    for (int e = 0; e < nExt; ++e) {
        extDof[e] = dof[extNode[e]];
        extB[e] = (unsigned char)kindb[extNode[e]];
    }
    int *d_ownDof = upload(c, ownDof), *d_extDof = upload(c, extDof);
    unsigned char *d_ownB = upload(c, ownB), *d_extB = upload(c, extB);
    signed char *d_ownH = upload(c, ownH);
    double *d_ownX = dalloc<double>(c, 3 * (size_t)N);
    {
        double *d_oc = upload_tmp(c, ownCoords), *d_centre2 = upload_tmp(c, centre);
        int *d_os = upload_tmp(c, ownSub);
        if (!d_oc || !d_centre2 || !d_os) return XDCG_OOM;
        if (d_ownX) launch_xrel(N, d_oc, d_centre2, d_os, d_ownX, nullptr, st);
    }
    if (!d_ownDof || !d_extDof || !d_ownB || !d_extB || !d_ownH || !d_ownX) return XDCG_OOM;
    auto &B64 = c->L64.B;
    B64.nBox = S;
    B64.col0 = d_col0;
    B64.menr = d_menr;
    B64.ownPtr = d_ownPtr;
    B64.ownDof = d_ownDof;
    B64.ownB = d_ownB;
    B64.ownH = d_ownH;
    B64.ownX = d_ownX;
    B64.ownZ = d_zslotOff;
    B64.Zt = d_zslot;
    B64.extPtr = d_extPtr;
    B64.extDof = d_extDof;
    B64.extB = d_extB;
    B64.wOff = d_wOff;
    B64.W = d_W;
    c->Einv = dalloc<double>(c, (size_t)k * k);
    c->E = dalloc<double>(c, (size_t)k * k);
    int *sb = upload_tmp(c, segBox), *so = upload_tmp(c, segOwner),
        *sbg = upload_tmp(c, segBegin), *se = upload_tmp(c, segEnd);
    if (!c->Einv || !c->E || !sb || !so || !sbg || !se) return XDCG_OOM;
    CK(cudaMemsetAsync(c->Einv, 0, (size_t)k * k * sizeof(double), st));
    launch_build_E((int)segBox.size(), sb, so, sbg, se, d_extNode, d_wOff, d_W, d_dof, d_x64,
                   d_hs, d_col0, d_menr, zv, k, c->Einv, st);
    launch_symmetrize(c->Einv, k, st);
    CK(cudaMemcpyAsync(c->E, c->Einv, (size_t)k * k * sizeof(double), cudaMemcpyDeviceToDevice,
                       st));
    if (!mark(3)) return XDCG_CUDA_ERROR;   // node factors, W, E
    // E^-1 in place (pivots relative to E's largest diagonal entry); an update
    // whose E is unchanged (bitwise) takes the previous context's inverse
    {
        bool same = false;
        if (prev && prev->k == k && prev->E) {
            int *d_differ = dalloc_tmp<int>(c, 1);
            if (!d_differ) return XDCG_OOM;
            CK(cudaMemsetAsync(d_differ, 0, sizeof(int), st));
            launch_differ(c->E, prev->E, (long long)k * k, d_differ, st);
            int h = 1;
            CK(cudaMemcpyAsync(&h, d_differ, sizeof(int), cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            same = h == 0;
        }
        if (same) {
            CK(cudaMemcpyAsync(c->Einv, prev->Einv, (size_t)k * k * sizeof(double),
                               cudaMemcpyDeviceToDevice, st));
            c->reusedCoarse = 1;
        } else {
            xdcg_status es = dense_inverse(c, c->Einv, {k}, {0LL}, d_bad + 1, 0);
            if (es != XDCG_OK) return es;
        }
    }
    if (!mark(4)) return XDCG_CUDA_ERROR;   // E^-1

    // block-scaled FP32 level of the mixed path: K~ = L^-1 K L^-T, Z~ = L^T Z, W~ = L^-1 W
    if (mixed) {
        c->Einv32 = dalloc<float>(c, (size_t)k * k);
        if (!c->Einv32) return XDCG_OOM;
        launch_cast_f32(c->Einv, c->Einv32, (long long)k * k, st);
        std::vector<int> nodeList(N), nodeIdx(N);
        for (int t = 0; t < 3; ++t)
            for (size_t i = 0; i < lists[t].size(); ++i) {
                nodeList[lists[t][i]] = t;
                nodeIdx[lists[t][i]] = (int)i;
            }
        FacDev F;
        for (int t = 0; t < 3; ++t) {
            F.L[t] = L64[t];
            F.cnt[t] = (int)lists[t].size();
        }
        F.nodeList = upload(c, nodeList);
        F.nodeIdx = upload(c, nodeIdx);
        std::vector<int> blockRow(nnzb);
        for (int I = 0; I < N; ++I)
            for (long long p = rowp[I]; p < rowp[I + 1]; ++p) blockRow[p] = I;
        int *d_brow = upload_tmp(c, blockRow);
        double *d_Kt = dalloc_tmp<double>(c, (size_t)nval);
        std::vector<long long> zOff(N + 1, 0);   // explicit Z~ blocks in slot order
        for (int t = 0; t < N; ++t)
            zOff[t + 1] = zOff[t] + (long long)ownB[t] * (menr[ownSub[t]] ? 12 : 6);
        long long *d_zOff = upload_tmp(c, zOff);
        float *d_Zt = dalloc_tmp<float>(c, zOff[N]);
        float *d_Wt = dalloc_tmp<float>(c, nW);
        // The FP32 system is numbered box by box: node slots in box order,
        // each node's dofs together, so box s owns the contiguous dof range
        // [ownRowPtr[s], ownRowPtr[s + 1]) and own row r is dof r.
        std::vector<int> dof32(N + 1, 0);
        {
            int off = 0;
            for (int t = 0; t < N; ++t) {
                dof32[ownNodes[t]] = off;
                off += kindb[ownNodes[t]];
            }
            dof32[N] = off;
        }
        std::vector<int> chunkMap(nChunks);
        for (long long r = 0; r < nChunks; ++r) chunkMap[r] = dof32[rowNode[r]] / 3 + rowPart[r];
        std::vector<int> sRows32(sRows), xRows32(xRows);
        std::stable_sort(sRows32.begin(), sRows32.end(),
                         [&](int a, int b) { return chunkMap[a] < chunkMap[b]; });
        std::stable_sort(xRows32.begin(), xRows32.end(), [&](int a, int b) {
            const int ba = rowLen[a] / kXBucket, bb = rowLen[b] / kXBucket;
            return ba != bb ? ba > bb : chunkMap[a] < chunkMap[b];
        });
        SellHost HS32, HX32;
        build_sell(sRows32, kTprS, HS32, &chunkMap);
        build_sell(xRows32, kTprX, HX32, &chunkMap);
        auto &A2 = c->L32.A;
        int *d_src32S = nullptr, *d_src32X = nullptr;
        if (!upload_sell_structure(HS32, A2.S, &d_src32S) ||
            !upload_sell_structure(HX32, A2.X, &d_src32X))
            return XDCG_OOM;
        float *v32S = dalloc<float>(c, HS32.src.size()), *v32X = dalloc<float>(c, HX32.src.size());
        const int *d_dof32 = upload(c, dof32);
        if (!F.nodeList || !F.nodeIdx || !d_brow || !d_Kt || !d_zOff || !d_Zt || !d_Wt || !v32S ||
            !v32X || !d_dof32)
            return XDCG_OOM;
        A2.S.val = v32S;
        A2.X.val = v32X;
        c->L32.F = F;
        CK(cudaMemcpyAsync(d_Kt, d_val, (size_t)nval * sizeof(double), cudaMemcpyDeviceToDevice,
                           st));
        launch_scale_blocks(kin, d_brow, nnzb, F, d_Kt, st);
        launch_gather(d_src32S, (long long)HS32.src.size(), d_Kt, nullptr, v32S, st);
        launch_gather(d_src32X, (long long)HX32.src.size(), d_Kt, nullptr, v32X, st);
        A2.waitNs = waitNs;
        A2.shape = kSpmvDefaultShapeF32;
        A2.grid = spmv_persistent_grid<float>(HS32.nSlices + HX32.nSlices, A2.shape);
        if (A2.grid < 1) return XDCG_CUDA_ERROR;
        A2.warpSlice = partition(HS32, HX32, A2.grid);
        if (!A2.warpSlice) return XDCG_OOM;
        c->info.spmv_shape_fp32 = A2.shape;   // until autotuned or pinned below
        if (c->opt.autotune) {
            xdcg_status ts = autotune(A2, HS32, HX32, 0.0f, c->info.spmv_shape_us_fp32,
                                      &c->info.spmv_shape_fp32);
            if (ts != XDCG_OK) return ts;
        }
        {
            xdcg_status ts = pin(A2, HS32, HX32, 0.0f, c->opt.spmv_shape_fp32,
                                 &c->info.spmv_shape_fp32);
            if (ts != XDCG_OK) return ts;
        }
        if (c->opt.max_batch > 0) {
            // the batched product's own persistent grid (its registers and
            // stages set its blocks per SM) and step-balanced warp ranges
            auto &Ab = c->L32.Ab;
            Ab = A2;
            Ab.grid = spmm_persistent_grid(c->opt.max_batch <= 4 ? 4 : 8,
                                           HS32.nSlices + HX32.nSlices);
            if (Ab.grid < 1) return XDCG_CUDA_ERROR;
            Ab.warpSlice = partition(HS32, HX32, Ab.grid);
            if (!Ab.warpSlice) return XDCG_OOM;
        }
        launch_build_Zt(N, d_own, d_dof, d_sub, d_x64, d_hs, d_menr, zv, F, d_zOff, d_Zt, st);
        launch_scale_W(nExt, d_extBox, d_extNode, d_wOff, d_menr, d_dof, F, d_W, d_Wt, st);
        // row-parallel layouts: own rows (Z~) and coupled rows (W~) of each box,
        // column-major per box
        std::vector<int> ownRowPtr(S + 1, 0), ownRowStart(N);
        std::vector<long long> zBase(S + 1, 0);
        for (int sb2 = 0; sb2 < S; ++sb2) {
            for (int t = ownPtr[sb2]; t < ownPtr[sb2 + 1]; ++t) ownRowStart[t] = dof32[ownNodes[t]];
            ownRowPtr[sb2 + 1] = ownPtr[sb2 + 1] < N ? dof32[ownNodes[ownPtr[sb2 + 1]]] : dof32[N];
            zBase[sb2 + 1] = zBase[sb2] + (long long)(menr[sb2] ? 12 : 6) *
                                              (ownRowPtr[sb2 + 1] - ownRowPtr[sb2]);
        }
        std::vector<int> extRowPtr(S + 1, 0), extRowStart(nExt), extRowDof;
        std::vector<long long> wBase(S + 1, 0);
        for (int sb2 = 0; sb2 < S; ++sb2) {
            for (int e = extPtr[sb2]; e < extPtr[sb2 + 1]; ++e) {
                extRowStart[e] = (int)extRowDof.size();
                for (int i = 0; i < extB[e]; ++i) extRowDof.push_back(dof32[extNode[e]] + i);
            }
            extRowPtr[sb2 + 1] = (int)extRowDof.size();
            wBase[sb2 + 1] = wBase[sb2] + (long long)(menr[sb2] ? 12 : 6) *
                                              (extRowPtr[sb2 + 1] - extRowPtr[sb2]);
        }
        c->extRows32 = extRowPtr[S];
        c->zEnt32 = zBase[S];
        c->wEnt32 = wBase[S];
        RowBoxDev &R = c->L32.R;
        c->g32 = dalloc<float>(c, std::max(k, 1));
        if (!c->g32) return XDCG_OOM;
        R.g32 = c->g32;
        R.nBox = S;
        R.col0 = d_col0;
        R.menr = d_menr;
        R.ownRowPtr = upload(c, ownRowPtr);
        R.zBase = upload(c, zBase);
        R.extRowPtr = upload(c, extRowPtr);
        R.extRowDof = upload(c, extRowDof);
        R.wBase = upload(c, wBase);
        float *Zcm = dalloc<float>(c, zBase[S]), *Wcm = dalloc<float>(c, wBase[S]);
        int *d_ownSub = upload_tmp(c, ownSub), *d_ors = upload_tmp(c, ownRowStart),
            *d_ers = upload_tmp(c, extRowStart);
        if (!R.ownRowPtr || !R.zBase || !R.extRowPtr || !R.extRowDof ||
            !R.wBase || !Zcm || !Wcm || !d_ownSub || !d_ors || !d_ers)
            return XDCG_OOM;
        // balanced restriction units: each box's own rows followed by its coupled
        // rows, cut into nearly equal pieces of at most unitRows rows (with
        // halve12, half as many for a box with 12 columns, whose rows cost
        // about twice as much: the batched kernels, whose units are a box
        // each); prolongation units: each box's own rows in pieces of at most
        // pRows
        auto build_units = [&](RowBoxDev &T, int unitRows, int pRows, bool halve12) -> bool {
            std::vector<int> unitBox, uOb, uOe, uEb, uEe, boxUnit(S + 1, 0);
            for (int sb2 = 0; sb2 < S; ++sb2) {
                boxUnit[sb2] = (int)unitBox.size();
                const long long nOwn = ownRowPtr[sb2 + 1] - ownRowPtr[sb2];
                const long long nCpl = extRowPtr[sb2 + 1] - extRowPtr[sb2];
                const long long Tr = nOwn + nCpl;
                const long long ur = halve12 && menr[sb2] ? std::max(1, unitRows / 2) : unitRows;
                const long long nu = std::max<long long>(1, (Tr + ur - 1) / ur);
                for (long long j = 0; j < nu; ++j) {
                    const long long a0 = Tr * j / nu, a1 = Tr * (j + 1) / nu;   // [a0, a1)
                    unitBox.push_back(sb2);
                    uOb.push_back(ownRowPtr[sb2] + (int)std::min(a0, nOwn));
                    uOe.push_back(ownRowPtr[sb2] + (int)std::min(a1, nOwn));
                    uEb.push_back(extRowPtr[sb2] + (int)(std::max(a0, nOwn) - nOwn));
                    uEe.push_back(extRowPtr[sb2] + (int)(std::max(a1, nOwn) - nOwn));
                }
            }
            boxUnit[S] = (int)unitBox.size();
            T.nUnits = (int)unitBox.size();
            T.unitBox = upload(c, unitBox);
            T.unitOwnBegin = upload(c, uOb);
            T.unitOwnEnd = upload(c, uOe);
            T.unitExtBegin = upload(c, uEb);
            T.unitExtEnd = upload(c, uEe);
            T.boxUnit = upload(c, boxUnit);
            std::vector<int> pBox, pBegin, pEnd;
            for (int sb2 = 0; sb2 < S; ++sb2)
                for (int rb = ownRowPtr[sb2]; rb < ownRowPtr[sb2 + 1]; rb += pRows) {
                    pBox.push_back(sb2);
                    pBegin.push_back(rb);
                    pEnd.push_back(std::min(ownRowPtr[sb2 + 1], rb + pRows));
                }
            T.nPUnits = (int)pBox.size();
            T.pUnitBox = upload(c, pBox);
            T.pUnitBegin = upload(c, pBegin);
            T.pUnitEnd = upload(c, pEnd);
            return T.unitBox && T.unitOwnBegin && T.unitOwnEnd && T.unitExtBegin &&
                   T.unitExtEnd && T.boxUnit && T.pUnitBox && T.pUnitBegin && T.pUnitEnd &&
                   T.nPUnits > 0 && T.nUnits <= kMaxGrid;
        };
        if (!build_units(R, kUnitRows, kProlongRows, false)) return XDCG_OOM;
        R.unitPart = dalloc<double>(c, 24 * (size_t)R.nUnits);
        R.boxTicket = dalloc<unsigned int>(c, S);
        if (!R.unitPart || !R.boxTicket) return XDCG_OOM;
        CK(cudaMemsetAsync(R.boxTicket, 0, S * sizeof(unsigned int), st));
        launch_to_colmajor(N, d_ownSub, d_ors, d_ownB, d_zOff, R.ownRowPtr, R.zBase, d_menr, d_Zt,
                           Zcm, st);
        launch_to_colmajor(nExt, d_extBox, d_ers, d_extB, d_wOff, R.extRowPtr, R.wBase, d_menr,
                           d_Wt, Wcm, st);
        R.Z = Zcm;
        R.W = Wcm;
        if (c->opt.max_batch > 0) {
            // the batched kernels give each row MB threads: smaller units keep as
            // many rows in flight per block as the single-column kernels have
            c->L32.Rb = R;
            if (!build_units(c->L32.Rb, kUnitRowsBatch, kProlongRowsBatch, true)) return XDCG_OOM;
        }
        c->L32.dofStart64 = d_dof;
        c->L32.dofStart32 = d_dof32;
    }
    if (!mark(5)) return XDCG_CUDA_ERROR;   // FP32 level
    // ---- caller blocks: K's diagonal blocks gathered densely and inverted in
    // FP64; for MIXED also L_b^T (K_bb)^-1 L_b in FP32 (the blocks of the
    // block-scaled system's M~^-1)
    if (blocks) {
        const int nb = blocks->n_blocks;
        std::vector<int> bStart(nb), bDim(nb), rowBlock(n), blockRow(nnzb);
        std::vector<long long> aOff(nb);
        long long tot = 0;
        for (int b = 0; b < nb; ++b) {
            bStart[b] = bptr[b];
            bDim[b] = bptr[b + 1] - bptr[b];
            aOff[b] = tot;
            tot += (long long)bDim[b] * bDim[b];
            for (int d = bptr[b]; d < bptr[b + 1]; ++d) rowBlock[d] = b;
        }
        c->blkEntries = tot;
        for (int I = 0; I < N; ++I)
            for (long long p = rowp[I]; p < rowp[I + 1]; ++p) blockRow[p] = I;
        std::vector<int> unitBlk, unitR0, unitR1;
        for (int b = 0; b < nb; ++b)
            for (int r = 0; r < bDim[b]; r += kBlkUnitRows) {
                unitBlk.push_back(b);
                unitR0.push_back(r);
                unitR1.push_back(std::min(bDim[b], r + kBlkUnitRows));
            }
        if (unitBlk.size() > (size_t)kMaxGrid) return XDCG_INVALID_ARG;
        std::vector<int> idx64(n);
        for (long long d = 0; d < n; ++d) idx64[d] = (int)d;
        double *A64 = dalloc<double>(c, (size_t)tot);
        int *d_bStart = upload_tmp(c, bStart), *d_bDim = upload_tmp(c, bDim);
        int *d_bon = upload_tmp(c, blockOfNode), *d_brow = upload_tmp(c, blockRow);
        long long *d_aOff = upload(c, aOff);
        int *d_bPos = upload(c, bptr), *d_idx64 = upload(c, idx64);
        int *d_ub = upload(c, unitBlk), *d_u0 = upload(c, unitR0), *d_u1 = upload(c, unitR1);
        if (!A64 || !d_bStart || !d_bDim || !d_bon || !d_brow || !d_aOff || !d_bPos || !d_idx64 ||
            !d_ub || !d_u0 || !d_u1)
            return XDCG_OOM;
        CK(cudaMemsetAsync(A64, 0, (size_t)tot * sizeof(double), st));
        launch_gather_blocks(kin, nnzb, d_brow, d_bon, d_bStart, d_bDim, d_aOff, A64, st);
        xdcg_status es = dense_inverse(c, A64, bDim, aOff, d_bad + 2, 1);
        if (es != XDCG_OK) return es;
        BlkDev<double> &J = c->L64.J;
        J.nBlk = nb;
        J.nUnits = (int)unitBlk.size();
        J.aOff = d_aOff;
        J.bPos = d_bPos;
        J.idx = d_idx64;
        J.A = A64;
        J.unitBlk = d_ub;
        J.unitRow0 = d_u0;
        J.unitRow1 = d_u1;
        if (mixed) {
            // positions in the box-major FP32 numbering
            std::vector<int> dof32(N + 1, 0);
            {
                int off = 0;
                for (int t = 0; t < N; ++t) {
                    dof32[ownNodes[t]] = off;
                    off += kindb[ownNodes[t]];
                }
            }
            std::vector<int> idx32(n);
            for (int I = 0; I < N; ++I)
                for (int i = 0; i < kindb[I]; ++i) idx32[dof[I] + i] = dof32[I] + i;
            float *A32 = dalloc<float>(c, (size_t)tot);
            double *Y = dalloc_tmp<double>(c, (size_t)tot);
            int *d_rowBlock = upload_tmp(c, rowBlock), *d_n0 = upload_tmp(c, bNode0),
                *d_n1 = upload_tmp(c, bNode1);
            int *d_idx32 = upload(c, idx32);
            if (!A32 || !Y || !d_rowBlock || !d_n0 || !d_n1 || !d_idx32) return XDCG_OOM;
            launch_scale_block_inverse((int)n, d_rowBlock, d_bStart, d_bDim, d_n0, d_n1, d_aOff,
                                       d_dof, c->L32.F, A64, Y, A32, st);
            BlkDev<float> &J32 = c->L32.J;
            J32.nBlk = nb;
            J32.nUnits = J.nUnits;
            J32.aOff = d_aOff;
            J32.bPos = d_bPos;
            J32.idx = d_idx32;
            J32.A = A32;
            J32.unitBlk = d_ub;
            J32.unitRow0 = d_u0;
            J32.unitRow1 = d_u1;
        }
        c->userBlocks = true;
    }

    if (!mark(6)) return XDCG_CUDA_ERROR;   // caller blocks
    int hbad[3];
    CK(cudaMemcpyAsync(hbad, d_bad, 3 * sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    CK(cudaGetLastError());
    for (void *p : c->temps) cudaFree(p);
    c->temps.clear();
    if (hbad[0] != INT_MAX) { *bad = hbad[0]; return XDCG_NOT_SPD_BLOCK; }
    if (hbad[2] != INT_MAX) { *bad = hbad[2]; return XDCG_NOT_SPD_BLOCK; }
    if (hbad[1] != INT_MAX) { *bad = hbad[1]; return XDCG_COARSE_NOT_SPD; }

    // ---- work vectors and scalar blocks
    c->u64 = dalloc<double>(c, n); c->r64 = dalloc<double>(c, n); c->p64 = dalloc<double>(c, n);
    c->q64 = dalloc<double>(c, n); c->y64 = dalloc<double>(c, n);
    c->f64 = dalloc<double>(c, n); c->uh64 = dalloc<double>(c, n);
    if (mixed) {
        c->f32 = dalloc<float>(c, n); c->u32 = dalloc<float>(c, n); c->r32 = dalloc<float>(c, n);
        c->p32 = dalloc<float>(c, n); c->q32 = dalloc<float>(c, n); c->y32 = dalloc<float>(c, n);
        if (!c->f32 || !c->u32 || !c->r32 || !c->p32 || !c->q32 || !c->y32) return XDCG_OOM;
    }
    c->g = dalloc<double>(c, k); c->zr = dalloc<double>(c, k); c->nu = dalloc<double>(c, k);
    c->nu32 = dalloc<float>(c, k);
    c->partials = dalloc<double>(c, 4 * (size_t)kMaxGrid);
    c->sc = dalloc<Scalars>(c, 1); c->sc32 = dalloc<Scalars>(c, 1); c->aux = dalloc<Scalars>(c, 1);
    if (c->opt.record_history) {
        c->hist = dalloc<double>(c, (size_t)c->opt.max_iter + 1);
        if (!c->hist) return XDCG_OOM;
    }
    if (mixed && c->opt.max_batch > 0) {
        const int MB = c->opt.max_batch <= 4 ? 4 : 8;
        c->bMB = MB;
        const size_t nv = (size_t)n * MB, kv = (size_t)std::max(k, 1) * MB;
        c->bF32 = dalloc<float>(c, nv); c->bU32 = dalloc<float>(c, nv);
        c->bRA = dalloc<float>(c, nv); c->bRB = dalloc<float>(c, nv);
        c->bP = dalloc<float>(c, nv); c->bQ = dalloc<float>(c, nv);
        c->bG32 = dalloc<float>(c, (size_t)g_ld(c) * MB); c->bNU32 = dalloc<float>(c, kv);
        c->bG = dalloc<double>(c, kv); c->bZR = dalloc<double>(c, kv); c->bNU = dalloc<double>(c, kv);
        c->bUnitPart = dalloc<double>(c, (size_t)c->L32.Rb.nUnits * MB * 24);
        c->bR64 = dalloc<double>(c, (size_t)n * MB);
        c->bs = dalloc<BatchScalars>(c, 1);
        c->bSlots = dalloc<Scalars>(c, kMaxBatch);
        if (!c->bF32 || !c->bU32 || !c->bRA || !c->bRB || !c->bP || !c->bQ || !c->bG32 ||
            !c->bNU32 || !c->bG || !c->bZR || !c->bNU || !c->bUnitPart || !c->bR64 || !c->bs ||
            !c->bSlots)
            return XDCG_OOM;
        CK(cudaMemsetAsync(c->bG32, 0, (size_t)g_ld(c) * MB * sizeof(float), st));
        if (cudaMallocHost(&c->h_bs, sizeof(BatchScalars)) != cudaSuccess) return XDCG_OOM;
        if (cudaMallocHost(&c->h_slots, sizeof(Scalars) * kMaxBatch) != cudaSuccess)
            return XDCG_OOM;
        if (!spmm_prepare()) return XDCG_CUDA_ERROR;
    }
    if (!c->u64 || !c->r64 || !c->p64 || !c->q64 || !c->y64 || !c->f64 || !c->uh64 || !c->g ||
        !c->zr || !c->nu || !c->nu32 || !c->partials || !c->sc || !c->sc32 || !c->aux)
        return XDCG_OOM;
    CK(cudaMemsetAsync(c->sc, 0, sizeof(Scalars), st));
    CK(cudaMemsetAsync(c->sc32, 0, sizeof(Scalars), st));
    CK(cudaMemsetAsync(c->aux, 0, sizeof(Scalars), st));
    if (cudaMallocHost(&c->h_sc, sizeof(Scalars)) != cudaSuccess) return XDCG_OOM;
    if (cudaMallocHost(&c->h_done, 2 * sizeof(int)) != cudaSuccess) return XDCG_OOM;
    if (cudaMallocHost(&c->h_poll, 2 * sizeof(Scalars)) != cudaSuccess) return XDCG_OOM;
    CK(cudaEventCreate(&c->ev0));
    CK(cudaEventCreate(&c->ev1));
    CK(cudaEventCreateWithFlags(&c->evb[0], cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&c->evb[1], cudaEventDisableTiming));
    CK(cudaStreamSynchronize(st));
    if (c->L64.A.grid > kMaxGrid || (mixed && c->L32.A.grid > kMaxGrid)) return XDCG_INVALID_ARG;

    // ---- algorithmic byte counts (see the roofline notes of the design)
    long long nStdN = (long long)lists[0].size(), nHN = (long long)lists[1].size(),
              nTN = (long long)lists[2].size();
    auto spmv_bytes = [&](int s) {
        return 9LL * nnzb3 * s + 4LL * nnzb3 + 8LL * (nS + nX) + 8LL * (HS.nSlices + HX.nSlices)
               + 2LL * n * s;
    };
    const long long fac = 6 * nStdN + 21 * nHN + 120 * nTN;
    // FP64 path: SpMV; update (u, p, r, q read, u, r, y written, factors);
    // restriction (r, y, W, box lists); coarse GEMV (E^-1 and k-vectors);
    // prolongation (y, p read, p written, node geometry)
    const long long iter64 = spmv_bytes(8) + 7LL * n * 8 + fac * 8 + 4LL * N
                             + 2LL * n * 8 + nW * 8 + 12LL * nExt + 16LL * k
                             + 8LL * k * k + 24LL * k + 3LL * n * 8 + 33LL * N;
    // FP32 scaled path (identity block preconditioner), per kernel:
    // restriction + update: own rows read map, r, q, p, u and write r', u,
    // plus Z~; coupled rows read map, r, q, plus W~; g and Z~^T r written;
    // coarse: E^-1 in FP32 and the k-vectors; prolongation: own rows read
    // map, r', p and write p, plus Z~ and nu
    const long long restrict32 = mixed ? 28LL * n + 4LL * c->zEnt32 + 12LL * c->extRows32 +
                                             4LL * c->wEnt32 + 16LL * k
                                       : 0;
    const long long coarse32 = mixed ? (c->opt.coarse_fp64 ? 8LL : 4LL) * k * k + 28LL * k : 0;
    const long long prolong32 = mixed ? 16LL * n + 4LL * c->zEnt32 + 4LL * k : 0;
    // caller blocks: the inverses, r gathered and y written once (per precision)
    const long long blk64 = c->userBlocks ? 8LL * c->blkEntries + 20LL * n : 0;
    const long long blk32 = c->userBlocks ? 4LL * c->blkEntries + 12LL * n : 0;
    const long long iter32 = mixed ? spmv_bytes(4) + restrict32 + coarse32 + prolong32 + blk32 : 0;
    c->info.n = n;
    c->info.n_nodes = N;
    c->info.k = k;
    c->info.nnz = 9 * nnzb3;
    c->info.nnzb3 = nnzb3;
    c->info.spmv_bytes_fp64 = spmv_bytes(8);
    c->info.spmv_bytes_fp32 = spmv_bytes(4);
    c->info.iter_bytes_fp64 = iter64 + blk64;
    c->info.iter_bytes_fp32 = iter32;
    c->info.restrict_bytes_fp32 = restrict32;
    c->info.coarse_bytes_fp32 = coarse32;
    c->info.prolong_bytes_fp32 = prolong32;
    c->info.nnzb = nnzb;
    auto spmv_alg = [&](int s) {
        return (long long)s * 9LL * nnzb3 + 4LL * nnzb + 4LL * (N + 1) + 2LL * s * n;
    };
    c->info.spmv_alg_bytes_fp64 = spmv_alg(8);
    c->info.spmv_alg_bytes_fp32 = spmv_alg(4);
    c->info.block_entries = c->blkEntries;
    if (!mark(7)) return XDCG_CUDA_ERROR;   // work vectors, scalar blocks
    return XDCG_OK;
}

}  // namespace

extern "C" {

xdcg_status xdcg_default_options(xdcg_options *opt) {
    if (!opt) return XDCG_INVALID_ARG;
    opt->tol = 1e-8;
    opt->max_iter = 10000;
    opt->precision = XDCG_FP64;
    opt->inner_tol = 1e-3;
    opt->max_outer = 30;
    opt->time_spmv = 0;
    opt->jacobi = XDCG_BLOCK_JACOBI;
    opt->record_history = 0;
    opt->max_batch = 0;
    opt->coarse_fp64 = 0;
    opt->wait_s = 2.0;
    opt->autotune = 0;
    opt->graph = 0;
    opt->spmv_shape_fp32 = -1;
    opt->spmv_shape_fp64 = -1;
    return XDCG_OK;
}

static xdcg_status setup_common(xdcg_ctx **out, const xdcg_ctx *prev, const xdcg_matrix *K,
                         const xdcg_deflation *Z, const xdcg_blocks *blocks,
                         const xdcg_options *opt, void *stream, int32_t *bad_index) {
    NvtxRange range(prev ? "xdcg setup update" : "xdcg setup");
    if (bad_index) *bad_index = -1;
    if (!out) return XDCG_INVALID_ARG;
    *out = nullptr;
    if (!K || !Z) return XDCG_INVALID_ARG;
    xdcg_ctx *c = new (std::nothrow) xdcg_ctx();
    if (!c) return XDCG_OOM;
    if (opt)
        c->opt = *opt;
    else
        xdcg_default_options(&c->opt);
    if (!(c->opt.tol > 0) || c->opt.max_iter < 0 || c->opt.max_outer < 1 ||
        (c->opt.precision != XDCG_FP64 && c->opt.precision != XDCG_MIXED) ||
        c->opt.time_spmv < 0 || c->opt.time_spmv > 2 ||
        (c->opt.jacobi != XDCG_BLOCK_JACOBI && c->opt.jacobi != XDCG_POINT_JACOBI) ||
        c->opt.max_batch < 0 || c->opt.max_batch > kMaxBatch ||
        (c->opt.coarse_fp64 != 0 && c->opt.coarse_fp64 != 1) ||
        (c->opt.autotune != 0 && c->opt.autotune != 1) ||
        (c->opt.graph != 0 && c->opt.graph != 1) ||
        c->opt.spmv_shape_fp32 < -1 || c->opt.spmv_shape_fp32 >= spmv_shape_count<float>() ||
        c->opt.spmv_shape_fp64 < -1 || c->opt.spmv_shape_fp64 >= spmv_shape_count<double>() ||
        !(c->opt.wait_s >= 0.0 && c->opt.wait_s <= 60.0) ||
        !(c->opt.inner_tol > 0 && c->opt.inner_tol < 1) ||
        (blocks && (c->opt.jacobi != XDCG_BLOCK_JACOBI || c->opt.max_batch > 0))) {
        delete c;
        return XDCG_INVALID_ARG;
    }
    c->st = (cudaStream_t)stream;
    if (cudaGetDevice(&c->device) != cudaSuccess) { delete c; return XDCG_CUDA_ERROR; }
    const auto t0 = std::chrono::steady_clock::now();
    int bad = -1;
    xdcg_status s = setup_impl(c, K, Z, blocks, &bad, prev);
    if (bad_index) *bad_index = bad;
    if (s != XDCG_OK) {
        cudaStreamSynchronize(c->st);
        free_ctx(c);
        return s;
    }
    c->info.t_setup_ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    c->info.reused_node_factors = c->reusedFactors;
    c->info.reused_coarse_inverse = c->reusedCoarse;
    *out = c;
    return XDCG_OK;
}

xdcg_status xdcg_setup(xdcg_ctx **out, const xdcg_matrix *K, const xdcg_deflation *Z,
                       const xdcg_blocks *blocks, const xdcg_options *opt, void *stream,
                       int32_t *bad_index) {
    return setup_common(out, nullptr, K, Z, blocks, opt, stream, bad_index);
}

xdcg_status xdcg_setup_update(xdcg_ctx **out, const xdcg_ctx *prev, const xdcg_matrix *K,
                              const xdcg_deflation *Z, const xdcg_blocks *blocks,
                              const xdcg_options *opt, void *stream, int32_t *bad_index) {
    if (!prev) {
        if (bad_index) *bad_index = -1;
        if (out) *out = nullptr;
        return XDCG_INVALID_ARG;
    }
    // the previous context's device arrays are read on this call's stream
    if (cudaStreamSynchronize(prev->st) != cudaSuccess) return XDCG_CUDA_ERROR;
    return setup_common(out, prev, K, Z, blocks, opt, stream, bad_index);
}

xdcg_status xdcg_solve(xdcg_ctx *c, const double *f, double *u, double tol, xdcg_result *res) {
    if (!c || !f || !u || f == u) return XDCG_INVALID_ARG;
    return do_solve(c, f, u, tol, false, res);
}

xdcg_status xdcg_solve_x0(xdcg_ctx *c, const double *f, double *u, double tol, xdcg_result *res) {
    if (!c || !f || !u || f == u) return XDCG_INVALID_ARG;
    return do_solve(c, f, u, tol, true, res);
}

xdcg_status xdcg_solve_batch(xdcg_ctx *c, const double *F, double *U, int32_t m, double tol,
                             xdcg_result *res) {
    NvtxRange range("xdcg solve_batch");
    if (!c || !F || !U || F == U || m < 1) return XDCG_INVALID_ARG;
    if (tol <= 0) tol = c->opt.tol;
    if (c->bMB == 0) {
        // no batched run on this context: the columns one after another
        xdcg_status worst = XDCG_OK;
        for (int j = 0; j < m; ++j) {
            xdcg_result r1{};
            xdcg_status s = do_solve(c, F + (size_t)j * c->n, U + (size_t)j * c->n, tol, false, &r1);
            if (s == XDCG_CUDA_ERROR || s == XDCG_TIMEOUT) return s;
            if (s != XDCG_OK) worst = s;
            if (res) res[j] = r1;
        }
        return worst;
    }
    if (m > c->opt.max_batch) return XDCG_INVALID_ARG;
    xdcg_ctx *one[1] = {c};
    const double *Fs[1] = {F};
    double *Us[1] = {U};
    const int32_t ms[1] = {m};
    xdcg_status st1 = XDCG_OK;
    xdcg_status s = xdcg_solve_systems(one, 1, Fs, Us, ms, tol, res, &st1);
    return s == XDCG_OK ? st1 : s;
}

xdcg_status xdcg_solve_systems(xdcg_ctx *const *ctxs, int32_t n_sys, const double *const *F,
                               double *const *U, const int32_t *m, double tol,
                               xdcg_result *res, xdcg_status *status) {
    NvtxRange range("xdcg solve_systems");
    if (!ctxs || n_sys < 1 || !F || !U || !m) return XDCG_INVALID_ARG;
    std::vector<BatchRun> runs(n_sys);
    for (int q = 0; q < n_sys; ++q) {
        xdcg_ctx *c = ctxs[q];
        if (!c || !c->mixed || c->bMB == 0 || c->bMB != ctxs[0]->bMB ||
            c->device != ctxs[0]->device)
            return XDCG_INVALID_ARG;
        if (!F[q] || !U[q] || (const double *)U[q] == F[q] || m[q] < 1 ||
            m[q] > c->opt.max_batch)
            return XDCG_INVALID_ARG;
        for (int r = 0; r < q; ++r)
            if (ctxs[r] == c) return XDCG_INVALID_ARG;   // one set of scalars per context
        runs[q].c = c;
        runs[q].F = F[q];
        runs[q].U = U[q];
        runs[q].m = m[q];
        runs[q].tol = tol > 0 ? tol : c->opt.tol;
    }
    xdcg_ctx *c0 = ctxs[0];
    int prev = -1;
    CK(cudaGetDevice(&prev));
    CK(cudaSetDevice(c0->device));
    cudaStream_t st = c0->st;
    // every system's work runs on the first context's stream, ordered after
    // and before the work queued on the others' streams
    std::vector<cudaEvent_t> evs;
    auto order = [&](cudaStream_t from, cudaStream_t to) -> xdcg_status {
        if (from == to) return XDCG_OK;
        cudaEvent_t e;
        CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        evs.push_back(e);
        CK(cudaEventRecord(e, from));
        CK(cudaStreamWaitEvent(to, e, 0));
        return XDCG_OK;
    };
    xdcg_status s = XDCG_OK;
    for (int q = 1; q < n_sys && s == XDCG_OK; ++q) s = order(ctxs[q]->st, st);
    std::vector<xdcg_status> sst(n_sys, XDCG_OK);
    std::vector<long long> l0(n_sys);
    for (int q = 0; q < n_sys; ++q) l0[q] = ctxs[q]->launches;
    const long long g0 = c0->graphLaunches;
    float ms = 0.f;
    if (s == XDCG_OK) {
        CK(cudaEventRecord(c0->ev0, st));
        s = c0->bMB == 4 ? solve_batches<4>(runs.data(), n_sys, st, sst.data())
                         : solve_batches<8>(runs.data(), n_sys, st, sst.data());
        if (s == XDCG_OK) {
            CK(cudaEventRecord(c0->ev1, st));
            CK(cudaEventSynchronize(c0->ev1));
            CK(cudaEventElapsedTime(&ms, c0->ev0, c0->ev1));
        }
    }
    for (int q = 1; q < n_sys; ++q) {
        xdcg_status s2 = order(st, ctxs[q]->st);
        if (s == XDCG_OK) s = s2;
    }
    for (auto e : evs) cudaEventDestroy(e);
    cudaSetDevice(prev);
    if (s != XDCG_OK) return s;
    xdcg_status worst = XDCG_OK;
    long long off = 0;
    for (int q = 0; q < n_sys; ++q) {
        xdcg_result local[kMaxBatch];
        xdcg_status sq = batch_results(runs[q], local);
        if (sst[q] != XDCG_OK) sq = sst[q];
        for (int j = 0; j < m[q]; ++j) {
            local[j].t_solve_ms = ms;
            local[j].n_launches = ctxs[q]->launches - l0[q];
            local[j].n_graph_launches = (int32_t)(c0->graphLaunches - g0);   // shared by all
            if (res) res[off + j] = local[j];
        }
        off += m[q];
        if (status) status[q] = sq;
        if (sq == XDCG_BREAKDOWN || (sq == XDCG_NO_CONVERGENCE && worst == XDCG_OK)) worst = sq;
    }
    return worst;
}

xdcg_status xdcg_solve_host(xdcg_ctx *c, const double *f_host, double *u_host, double tol,
                            xdcg_result *res) {
    if (!c || !f_host || !u_host) return XDCG_INVALID_ARG;
    CK(cudaMemcpyAsync(c->f64, f_host, c->n * sizeof(double), cudaMemcpyHostToDevice, c->st));
    xdcg_status s = do_solve(c, c->f64, c->uh64, tol, false, res);
    if (s == XDCG_CUDA_ERROR) return s;
    CK(cudaMemcpyAsync(u_host, c->uh64, c->n * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    return s;
}

xdcg_status xdcg_get_history(xdcg_ctx *c, double *out, int32_t cap, int32_t *count) {
    if (!c || !count || cap < 0 || (cap > 0 && !out)) return XDCG_INVALID_ARG;
    if (!c->hist) return XDCG_INVALID_ARG;
    const int m = std::min(cap, c->histLen);
    *count = c->histLen;
    if (m == 0) return XDCG_OK;
    std::vector<double> rr(m);
    CK(cudaMemcpyAsync(rr.data(), c->hist, m * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    for (int i = 0; i < m; ++i) out[i] = c->histFF > 0 ? std::sqrt(rr[i] / c->histFF) : 0.0;
    return XDCG_OK;
}

xdcg_status xdcg_get_info(const xdcg_ctx *c, xdcg_info_t *info) {
    if (!c || !info) return XDCG_INVALID_ARG;
    *info = c->info;
    return XDCG_OK;
}

// y = K~ x for caller-ordered x, y: the FP32 operator works in the box-major
// numbering, so x is renumbered into p32 and the product back out of q32
void spmv32_caller_order(xdcg_ctx *c, const float *x, float *y, double *partials, Scalars *sc) {
    const int *nat = c->L32.dofStart64, *box = c->L32.dofStart32;
    launch_renumber(c->nNodes, nat, nat, box, x, c->p32, c->st);
    launch_spmv<float>(c->L32.A, c->p32, c->q32, nullptr, 0, partials, sc, kFinStore, 2, c->st);
    launch_renumber(c->nNodes, nat, box, nat, c->q32, y, c->st);
    c->launches += 3;
}

xdcg_status xdcg_spmv(xdcg_ctx *c, int32_t precision, const void *x, void *y, double *xty) {
    if (!c || !x || !y || x == y) return XDCG_INVALID_ARG;
    if (precision == XDCG_MIXED && !c->mixed) return XDCG_INVALID_ARG;
    init_scalars(c, c->aux, -1.0, nullptr, INT_MAX);
    if (precision == XDCG_FP64) {
        launch_spmv<double>(c->L64.A, (const double *)x, (double *)y, nullptr, 0, c->partials,
                            c->aux, kFinStore, 2, c->st);
        c->launches++;
    } else if (precision == XDCG_MIXED) {
        spmv32_caller_order(c, (const float *)x, (float *)y, c->partials, c->aux);
    } else {
        return XDCG_INVALID_ARG;
    }
    CK(cudaGetLastError());
    double v[3];
    xdcg_status s = read_aux(c, v, 3);
    if (s != XDCG_OK) return s;
    if (xty) *xty = v[2];
    return XDCG_OK;
}

xdcg_status xdcg_element_sensitivity(xdcg_ctx *c, int64_t n_el, const int64_t *elem_dof_ptr,
                                     const int32_t *elem_dofs, const int64_t *elem_mat_off,
                                     const double *elem_mat, int64_t mat_len, const double *u,
                                     const double *lam, double *out) {
    if (!c || n_el < 0) return XDCG_INVALID_ARG;
    if (n_el == 0) return XDCG_OK;
    if (!elem_dof_ptr || !elem_dofs || !elem_mat_off || !elem_mat || mat_len < 0 || !u || !lam ||
        !out)
        return XDCG_INVALID_ARG;
    // the fault word of the scalar block flags bad element data
    init_scalars(c, c->aux, -1.0, nullptr, INT_MAX);
    launch_element_sensitivity(n_el, c->n, elem_dof_ptr, elem_dofs, elem_mat_off, mat_len,
                               elem_mat, u, lam, out, &c->aux->fault, c->st);
    c->launches++;
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(c->h_sc, c->aux, sizeof(Scalars), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    return c->h_sc->fault ? XDCG_INVALID_ARG : XDCG_OK;
}

xdcg_status xdcg_stiffness_gradient(xdcg_ctx *c, const xdcg_matrix *K, const double *lam,
                                    const double *u, double *out) {
    if (!c || !K || !lam || !u || !out || K->mem != XDCG_DEVICE || !K->dof_ptr ||
        !K->row_ptr || !K->col || !K->val_ptr || K->n_nodes != c->nNodes)
        return XDCG_INVALID_ARG;
    // the pattern's sizes (two entries each, read back)
    int32_t nnzb32 = 0;
    int64_t nval = 0;
    CK(cudaMemcpyAsync(&nnzb32, K->row_ptr + K->n_nodes, sizeof(int32_t), cudaMemcpyDeviceToHost,
                       c->st));
    CK(cudaStreamSynchronize(c->st));
    if (nnzb32 < 0) return XDCG_INVALID_ARG;
    CK(cudaMemcpyAsync(&nval, K->val_ptr + nnzb32, sizeof(int64_t), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    if (nval < 0) return XDCG_INVALID_ARG;
    // the fault word of the scalar block flags bad structure
    init_scalars(c, c->aux, -1.0, nullptr, INT_MAX);
    launch_stiffness_gradient(c->nNodes, nnzb32, c->n, nval, K->dof_ptr, K->row_ptr, K->col,
                              K->val_ptr, lam, u, out, &c->aux->fault, c->st);
    c->launches++;
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(c->h_sc, c->aux, sizeof(Scalars), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    return c->h_sc->fault ? XDCG_INVALID_ARG : XDCG_OK;
}

// ---- no-allocation SpMV: reduction scratch in one static device array ------

namespace {

// [Scalars block | XDCG_NOALLOC_MAX_BLOCKS partial sums]; zero at load time
constexpr int kNoallocScalarsDoubles = (int)((sizeof(Scalars) + 255) / 256 * 256 / sizeof(double));
static __device__ __align__(256) double
    g_noalloc_scratch[kNoallocScalarsDoubles + XDCG_NOALLOC_MAX_BLOCKS];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
double *g_noalloc_ptr[kMaxDevices] = {nullptr};

__global__ void k_noalloc_result(const Scalars *sc, int slot, double *out) {
    if (threadIdx.x == 0 && blockIdx.x == 0)
        *out = sc->done == kFault ? __longlong_as_double(0x7ff8000000000000ll) : sc->scratch[slot];
}

}  // namespace

xdcg_status xdcg_spmv_noalloc(xdcg_ctx *c, int32_t precision, const void *x, void *y,
                              double *xty_dev) {
    if (!c || !x || !y || x == y) return XDCG_INVALID_ARG;
    if (precision != XDCG_FP64 && precision != XDCG_MIXED) return XDCG_INVALID_ARG;
    if (precision == XDCG_MIXED && !c->mixed) return XDCG_INVALID_ARG;
    const int grid = precision == XDCG_FP64 ? c->L64.A.grid : c->L32.A.grid;
    if (grid > XDCG_NOALLOC_MAX_BLOCKS) return XDCG_TOO_LARGE;
    // the context's stream and buffers belong to the device that was current
    // at set-up; the scratch must be that device's copy of the array
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (dev != c->device || dev < 0 || dev >= kMaxDevices) return XDCG_INVALID_ARG;
    double *base = nullptr;
    {
        // first call on this device: resolve the array's device address
        // (the host-side name is only a stand-in, not a device pointer)
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        if (!g_noalloc_ptr[dev]) {
            void *p = nullptr;
            CK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
            g_noalloc_ptr[dev] = (double *)p;
        }
        base = g_noalloc_ptr[dev];
    }
    Scalars *sc = reinterpret_cast<Scalars *>(base);
    double *partials = base + kNoallocScalarsDoubles;
    // clear the scalar block (done flag, tickets) left by the previous call
    init_scalars(c, sc, -1.0, nullptr, INT_MAX);
    if (precision == XDCG_FP64) {
        launch_spmv<double>(c->L64.A, (const double *)x, (double *)y, nullptr, 0, partials, sc,
                            kFinStore, 2, c->st);
        c->launches++;
    } else {
        spmv32_caller_order(c, (const float *)x, (float *)y, partials, sc);
    }
    if (xty_dev) {
        k_noalloc_result<<<1, 32, 0, c->st>>>(sc, 2, xty_dev);
        c->launches++;
    }
    CK(cudaGetLastError());
    return XDCG_OK;
}

xdcg_status xdcg_precond(xdcg_ctx *c, const double *r, double *z) {
    if (!c || !r || !z || r == z) return XDCG_INVALID_ARG;
    cudaStream_t st = c->st;
    init_scalars(c, c->aux, -1.0, nullptr, INT_MAX);
    CK(cudaMemcpyAsync(c->r64, r, c->n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    PlainPath{c, c->L64, c->st}.update(nullptr, c->r64, nullptr, nullptr, c->y64, 1, c->aux);
    launch_restrict(c->L64.B, c->r64, c->y64, 1, c->g, c->zr, c->aux, st);
    launch_coarse(c->Einv, c->k, c->g, c->zr, c->nu, nullptr, 0, c->partials, c->aux, st);
    launch_prolong(c->L64.B, c->nu, c->y64, z, 2, c->aux, st);
    c->launches += 4;
    CK(cudaStreamSynchronize(st));
    CK(cudaGetLastError());
    return XDCG_OK;
}

xdcg_status xdcg_coarse_matrix(xdcg_ctx *c, double *E_host) {
    if (!c || !E_host) return XDCG_INVALID_ARG;
    CK(cudaMemcpyAsync(E_host, c->E, (size_t)c->k * c->k * sizeof(double),
                       cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    return XDCG_OK;
}

xdcg_status xdcg_destroy(xdcg_ctx *c) {
    if (!c) return XDCG_INVALID_ARG;
    cudaStreamSynchronize(c->st);
    free_ctx(c);
    return XDCG_OK;
}

const char *xdcg_status_string(xdcg_status s) {
    switch (s) {
        case XDCG_OK: return "ok";
        case XDCG_INVALID_ARG: return "invalid argument";
        case XDCG_NOT_SPD_BLOCK: return "node block not SPD";
        case XDCG_COARSE_NOT_SPD: return "coarse matrix E not SPD";
        case XDCG_BREAKDOWN: return "CG breakdown (p^T K p <= 0 or not finite)";
        case XDCG_NO_CONVERGENCE: return "no convergence within max_iter";
        case XDCG_CUDA_ERROR: return "CUDA error";
        case XDCG_OOM: return "out of device memory";
        case XDCG_TOO_LARGE:
            return "problem exceeds the fixed scratch of xdcg_spmv_noalloc (XDCG_NOALLOC_MAX_BLOCKS)";
        case XDCG_TIMEOUT: return "a bounded device-side wait ran out (results invalid)";
    }
    return "unknown status";
}

}  // extern "C"
