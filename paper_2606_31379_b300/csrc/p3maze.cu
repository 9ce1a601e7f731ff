// C ABI of the P3MaZe CUDA library: context set-up, the per-step pipeline
// and the observables.  See include/p3maze.h for the contract of each call.
#include "p3maze.h"

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "common.cuh"
#include "mesh.cuh"
#include "particles.cuh"

using namespace p3;

namespace {

thread_local std::string g_init_error = "no error";

constexpr int kReduceBlocks = 296;  // 2 x 148 SMs
constexpr int kLevelMin = 16;       // levels are halved while even and larger than this
constexpr int kMaxGraphs = 4;       // pointer phases of the phi (2) and y (4) rings
constexpr int kMaxStepGraphs = 2 * kMaxGraphs + 1;  // whole steps, tails (per phase) and one head

// Device scalar slots.
enum { S_QSUM = 0, S_ESR, S_EVDW, S_VLR, S_MV2, S_EBOND, S_EXCL, S_WSR, S_NSCAL };

struct Level {
    int n = 0;
    int64_t pts = 0;
    void* e = nullptr;
    void* b = nullptr;
    void* r = nullptr;
    // levels with n <= kCoarseMax can be the coarse level: Hartley table H
    // (n x n), scaled pseudo-inverse eigenvalues D (n^3), transform work array
    void* H = nullptr;
    void* D = nullptr;
    void* t = nullptr;
    // mixed precision, n = 32 or 64: the coarse solve by FFT (D stored
    // bit-reversed and scaled for those kernels), twiddles exp(-2 pi i k / n)
    void* tw = nullptr;
    // FP32 levels with N % 4 == 0 that sweep: the other buffer of the
    // out-of-place full sweeps (level 0: the smoothing ping-pong buffer, free
    // during the solve), and the buffer (e or e2) that holds the level's
    // correction when its V-cycle ends (set when the V-cycle is launched)
    void* e2 = nullptr;
    void* fin = nullptr;
};

// Largest level whose red-black sweeps run as one launch each (sweep_fuse).
constexpr int kSweepFuseMaxN = 64;

// One captured MD step for a given pointer phase of the field rings.
enum { PART_ALL = 0, PART_HEAD = 1, PART_TAIL = 2 };  // what a step graph records

struct StepGraph {
    bool valid = false;
    int part = PART_ALL;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t x = nullptr;
    int icur = 0;
    double* yh[4] = {nullptr, nullptr, nullptr, nullptr};
    int64_t launches[P3MAZE_NSTAGES] = {};
    bool timed[P3MAZE_NSTAGES] = {};
};

inline unsigned nblk(int64_t m) { return (unsigned)((m + P3_THREADS - 1) / P3_THREADS); }

// In mixed precision the 8-byte constraint arrays (phi, Psi, z history, s,
// final residual) hold 64-bit fixed-point values (x 2^40, potential units).
inline fix_t* fx(double* p) { return reinterpret_cast<fix_t*>(p); }
inline dim3 g3(int n) { return dim3((n + P3_BX - 1) / P3_BX, (n + P3_BY - 1) / P3_BY, n); }
inline dim3 g3h(int n) { return dim3((n / 2 + P3_BX - 1) / P3_BX, (n + P3_BY - 1) / P3_BY, n); }
// z-marching stencils: ZC planes per thread.
inline dim3 gz(int n, int zc) { return dim3((n + P3_BX - 1) / P3_BX, (n + P3_BY - 1) / P3_BY, (n + zc - 1) / zc); }
inline unsigned gz_blocks(int n, int zc) { const dim3 g = gz(n, zc); return g.x * g.y * g.z; }
// Fine residual: each block walks every 16th z plane (about a thousand blocks at 128^3).
inline dim3 resid_grid(int n) { return dim3((n + P3_BX - 1) / P3_BX, (n + P3_BY - 1) / P3_BY, std::min(n, 16)); }
const dim3 kB3(P3_BX, P3_BY, 1);

}  // namespace

// Library-internal: set the message of p3maze_last_error(NULL).
__attribute__((visibility("hidden"))) void p3_set_global_error(const char* msg) { g_init_error = msg; }

struct p3maze_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;       // internal work stream (highest priority)
    cudaStream_t user_stream = nullptr;  // the caller's stream; every call is fenced against it
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cudaStream_t body_stream = nullptr;  // capture of the while-node body
    cudaStream_t pair_stream = nullptr;  // short-range forces, concurrent with the mesh pipeline
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // positions are final once the drift of a step has run: recorded there (a
    // node of the step graphs) so that p3maze_step_host copies them out on
    // copy_stream while the step's forces are formed
    cudaEvent_t ev_drift = nullptr, ev_copied = nullptr;
    cudaStream_t copy_stream = nullptr;
    // parameters
    int np = 0, N = 0, nc = 0, ncell = 0, prec = 0, pred = 3, itmax = 50, nu1 = 2, nu2 = 2, K = 0;
    int nmol = 0, nlev = 0, method = 0;
    int zc = 8;                          // z planes per thread in the diffusion step (tunable)
    int pair_fork = 0;                   // pair kernel forked after: 0 smoothing, 1 the cell list (tunable)
    int pair_blocks = 0;                 // pair grid: 0 one block per home box, else a persistent grid (tunable)
    int lr_force = 0;                    // P3MAZE_LR_FORCE_FD (the paper's) or P3MAZE_LR_FORCE_ANALYTIC
    int sr_shift = 0;                    // P3MAZE_SR_TRUNCATE or P3MAZE_SR_SHIFT_FORCE
    int nsm = 148;                       // SMs of the device
    bool pdl = true;                     // chained mesh kernels overlap their predecessor's tail (P3MAZE_PDL=0: off)
    int fuse = 1;                        // mixed mode: diffusion steps per launch, 1 to 4, or 5: all in one
                                         // cluster launch (16 <= N <= 64) (tunable)
    ClusterMesh* cltab = nullptr;        // this mesh's entry for the cluster smoothing kernel
    bool cluster_ok = false;             // the device runs this mesh's clusters of the smoothing kernel
    int cl_ctas = 0;                     // CTAs per cluster of mode 5 (0: automatic)
    void* Ssm = nullptr;                 // mode 6: (1 + c lambda_k)^K / N^3 in the Hartley basis (FP32, N <= 64
                                         // or N = 128)
    void* fht_tw = nullptr;              // mode 6 by FFT (N = 32, 64, 128): exp(-2 pi i k / N), k < N / 2
    int sweep_fuse = 1;                  // FP32 quad levels: a full red-black sweep per launch
    // rollback (p3maze_set_rollback): a device copy of the state taken at the
    // first step call after the last wait, restored when that call's steps fail
    bool rollback = false;
    void* snap = nullptr;
    size_t snap_bytes = 0;
    bool snap_taken = false;
    int64_t snap_steps = 0;
    int snap_nhist = 0;
    int64_t settings_gen = 0;            // bumped whenever a setting recorded in graphs changes
    double res_scale = 1.0;              // residual in the method's units: 1 (MaZe) or 4pi/h (P3M)
    double res_unit = 1.0;               // device residual per charge unit: 1 (FP64) or 4pi/h (mixed, fixed point)
    int64_t P = 0;
    double L = 0, h = 0, inv_h = 0, alpha = 0, sigma = 0, rc = 0, c = 0, tol = 0, dt = 0, ke = 0;
    double inv_cell = 0, lcell = 0, v_self = 0;
    double ke_pair = 0;                  // Coulomb constant of the erfc pair term (0 for PMaZe)
    SRTable tab{};
    double kb = 0, r0 = 0, ka = 0, th0 = 0;
    // particle arrays (original order)
    double *r = nullptr, *v = nullptr, *F = nullptr, *Fsr = nullptr, *Flr = nullptr, *Fb = nullptr;
    double *hdt_acc = nullptr, *mass = nullptr, *Q = nullptr;
    int *type = nullptr, *mol = nullptr, *tri = nullptr;
    // cell list and cell-ordered copies
    int *cell = nullptr, *count = nullptr, *start = nullptr, *fill = nullptr, *order = nullptr;
    int *ts = nullptr, *ms = nullptr, *cs = nullptr;
    PQ* xq = nullptr;
    PQ* xl64 = nullptr;
    float4* xl32 = nullptr;
    MeshPt* mp = nullptr;                 // mixed mode: mesh coordinates in cell order
    double *Fs = nullptr, *ecs = nullptr, *evs = nullptr, *wsr = nullptr, *eb = nullptr, *ex = nullptr;
    // mesh
    void *q = nullptr, *qs = nullptr;
    double* phi[2] = {nullptr, nullptr};
    double* psi[2] = {nullptr, nullptr};  // (h/4pi) M phi, same ring as phi
    int icur = 0;                         // [icur] = step k, [1-icur] = step k-1
    double* yh[4] = {nullptr, nullptr, nullptr, nullptr};  // [0] work, [1..3] y^k, y^{k-1}, y^{k-2}
    int nhist = 0;
    double* sig = nullptr;
    double* rfin = nullptr;
    float* phi32 = nullptr;               // mixed mode: FP32 copy of phi^k for the interpolation
    std::vector<Level> lev;
    int lc = 0;                           // coarse level in use (solved exactly)
    int cmax = 64;                        // coarse level: first with n <= cmax (tunable)
    // reductions and solver state
    double* partial = nullptr;
    double* dscal = nullptr;
    double* bmax = nullptr;          // block maxima of the fine residual
    MGState* dmg = nullptr;
    double* hscal = nullptr;
    MGState* hmg = nullptr;
    p3maze_stats st{};
    // graphs
    bool use_graphs = true;
    bool capturing = false;
    bool in_body = false;
    StepGraph graphs[kMaxStepGraphs];
    int64_t body_launches = 0;       // kernels per V-cycle iteration of the while body
    int64_t eager_iters = 0;         // V-cycles launched outside graphs since the last reset
    int64_t graph_iters_seen = 0;    // graph V-cycles already folded into the launch count
    // timing and launch accounting
    bool timing = false;
    cudaEvent_t ev[P3MAZE_NSTAGES][2] = {};
    bool pending[P3MAZE_NSTAGES] = {};
    double stage_ms[P3MAZE_NSTAGES] = {};
    int64_t launches[P3MAZE_NSTAGES] = {};
    int64_t timed_steps = 0;
    std::vector<void*> allocs;
    size_t dev_bytes = 0;                // device memory this context allocated
    std::string err = "no error";
};

namespace {

int fail(p3maze_ctx* c, int code, const std::string& msg) {
    if (c) c->err = msg;
    else g_init_error = msg;
    return code;
}

// A failed runtime call also leaves the thread's last error set: it is
// cleared, so that a later launch check does not report it again.
#define CK(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) {                                                              \
            cudaGetLastError();                                                               \
            return fail(ctx, P3MAZE_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
        }                                                                                     \
    } while (0)

#define CKL()                                                                                 \
    do {                                                                                      \
        cudaError_t e_ = cudaGetLastError();                                                  \
        if (e_ != cudaSuccess)                                                                \
            return fail(ctx, P3MAZE_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e_)); \
    } while (0)

template <typename P>
int dalloc(p3maze_ctx* ctx, P** p, size_t bytes) {
    void* d = nullptr;
    cudaError_t e = cudaMalloc(&d, bytes ? bytes : 16);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, P3MAZE_ERR_OOM, std::string("cudaMalloc(") + std::to_string(bytes) + "): " +
                                             cudaGetErrorString(e));
    }
    ctx->allocs.push_back(d);
    ctx->dev_bytes += bytes ? bytes : 16;
    *p = (P*)d;
    return P3MAZE_OK;
}

#define ALLOC(ptr, bytes)                                  \
    do {                                                   \
        int rc_ = dalloc(ctx, &(ptr), (size_t)(bytes));    \
        if (rc_) return rc_;                               \
    } while (0)

// Host array -> device array on the context's stream, complete on return (the
// source may be a temporary).  A plain cudaMemcpy runs on the legacy default
// stream, which the context's non-blocking streams are not ordered after.
#define UPLOAD(dst, src, bytes)                                                                  \
    do {                                                                                         \
        CK(cudaMemcpyAsync((dst), (src), (size_t)(bytes), cudaMemcpyHostToDevice, ctx->stream)); \
        CK(cudaStreamSynchronize(ctx->stream));                                                  \
    } while (0)

// Count `k` kernel launches of stage `st` (into the while-body tally while
// capturing the body).
inline void count(p3maze_ctx* ctx, int st, int k = 1) {
    if (ctx->in_body) ctx->body_launches += k;
    else ctx->launches[st] += k;
}

// Stage events; while capturing they must be external records so that the
// graph gets event-record nodes (a plain record only orders the capture).
void record(p3maze_ctx* ctx, cudaEvent_t ev) {
    if (ctx->capturing) cudaEventRecordWithFlags(ev, ctx->stream, cudaEventRecordExternal);
    else cudaEventRecord(ev, ctx->stream);
}

void stage_begin(p3maze_ctx* ctx, int st) {
    if (ctx->timing) record(ctx, ctx->ev[st][0]);
}

void stage_end(p3maze_ctx* ctx, int st) {
    if (ctx->timing) {
        record(ctx, ctx->ev[st][1]);
        ctx->pending[st] = true;
    }
}

// Fold the elapsed time of every stage recorded this step into the totals.
int collect_timing(p3maze_ctx* ctx) {
    if (!ctx->timing) return P3MAZE_OK;
    for (int st = 0; st < P3MAZE_NSTAGES; ++st) {
        if (!ctx->pending[st]) continue;
        CK(cudaEventSynchronize(ctx->ev[st][1]));
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, ctx->ev[st][0], ctx->ev[st][1]));
        ctx->stage_ms[st] += t;
        ctx->pending[st] = false;
    }
    ctx->timed_steps += 1;
    return P3MAZE_OK;
}

// Order the work stream after everything queued on the caller's stream so far.
int enter(p3maze_ctx* ctx) {
    CK(cudaEventRecord(ctx->ev_in, ctx->user_stream));
    CK(cudaStreamWaitEvent(ctx->stream, ctx->ev_in, 0));
    return P3MAZE_OK;
}

// Order the caller's stream after everything queued on the work stream.
int leave(p3maze_ctx* ctx) {
    CK(cudaEventRecord(ctx->ev_out, ctx->stream));
    CK(cudaStreamWaitEvent(ctx->user_stream, ctx->ev_out, 0));
    return P3MAZE_OK;
}


// ------------------------------------------------------------------ pipeline
// Launch with programmatic stream serialisation when pdl is set: the grid may
// be scheduled while its predecessor in the stream is still running, and
// its blocks wait in pdl_wait() until the predecessor has completed and its
// writes are visible.  Only kernels that call pdl_wait() before their first
// memory access may be launched this way.
template <typename... KArgs, typename... Args>
cudaError_t launch_maybe_pdl(bool pdl, void (*k)(KArgs...), dim3 g, dim3 b, size_t smem, cudaStream_t s,
                             Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = g;
    cfg.blockDim = b;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k, static_cast<KArgs>(args)...);
}

// Systems of at most 2048 particles (two per thread) build the cell list in
// one block with shared-memory counts; larger ones use the multi-kernel path
// (one SM walking 32768 particles takes about 90 us, three times longer).
constexpr int kCellBlockMaxCells = 12288, kCellBlockMaxParticles = 2048;
inline bool cells_in_one_block(int np, int ncell) {
    return ncell <= kCellBlockMaxCells && np <= kCellBlockMaxParticles;
}
inline size_t cells_block_smem(int ncell) { return 2 * sizeof(int) * (size_t)ncell; }

int build_cells(p3maze_ctx* ctx, bool counted) {
    cudaStream_t s = ctx->stream;
    stage_begin(ctx, P3MAZE_ST_CELLS);
    int launches = 0;
    // every launch may overlap its predecessor's tail (programmatic dependent
    // launch); the per-cell counts are zero on entry (cleared at setup and by
    // k_cell_sort once the scan has used them), or already formed by the
    // drift (counted)
    const bool pdl = ctx->pdl;
    if (cells_in_one_block(ctx->np, ctx->ncell)) {
        CK(launch_maybe_pdl(pdl, k_cells_block, dim3(1), dim3(kCellBlockThreads), cells_block_smem(ctx->ncell), s,
                            ctx->np, ctx->r, ctx->inv_cell, ctx->nc, ctx->ncell, ctx->cell, ctx->start, ctx->order));
        launches += 1;
    } else {
        if (!counted) {
            CK(launch_maybe_pdl(pdl, k_cell_count, dim3(nblk(ctx->np)), dim3(P3_THREADS), 0, s, ctx->np, ctx->r,
                                ctx->inv_cell, ctx->nc, ctx->cell, ctx->count));
            launches += 1;
        }
        CK(launch_maybe_pdl(pdl, k_scan_cells, dim3(1), dim3(kScanThreads), 0, s, ctx->ncell, ctx->count, ctx->start,
                            ctx->fill));
        CK(launch_maybe_pdl(pdl, k_cell_scatter, dim3(nblk(ctx->np)), dim3(P3_THREADS), 0, s, ctx->np, ctx->cell,
                            ctx->start, ctx->fill, ctx->order));
        CK(launch_maybe_pdl(pdl, k_cell_sort, dim3(nblk(ctx->ncell)), dim3(P3_THREADS), 0, s, ctx->ncell, ctx->start,
                            ctx->order, ctx->count));
        launches += 3;
    }
    CK(launch_maybe_pdl(pdl, k_gather_sorted, dim3(nblk(ctx->np)), dim3(P3_THREADS), 0, s, ctx->np, ctx->order,
                        ctx->r, ctx->Q, ctx->type, ctx->mol, ctx->cell, ctx->nc, ctx->lcell, ctx->xq, ctx->xl64,
                        ctx->xl32, ctx->ts, ctx->ms, ctx->cs, ctx->mp, ctx->N, ctx->inv_h));
    launches += 1;
    CKL();
    count(ctx, P3MAZE_ST_CELLS, launches);
    stage_end(ctx, P3MAZE_ST_CELLS);
    return P3MAZE_OK;
}

// Temporally blocked diffusion: tile 32 x 16 columns, S steps per launch.
constexpr int kTbX = 32, kTbY = 16;
inline dim3 tb_grid(int n, int zc) { return dim3((n + kTbX - 1) / kTbX, (n + kTbY - 1) / kTbY, (n + zc - 1) / zc); }
inline unsigned tb_blocks(int n, int zc) { const dim3 g = tb_grid(n, zc); return g.x * g.y * g.z; }
// Entries of the partial-sum buffer.
inline unsigned partial_slots(int n) { return std::max<unsigned>(std::max<unsigned>(1024, gz_blocks(n, 1)), tb_blocks(n, 1)); }
// FP64 field update: grid-stride over at most 1024 blocks (their sums are
// added by the last block; more blocks would queue on its arrival counter).
inline unsigned update_blocks(int n) { return std::min(nblk((int64_t)n * n * n), 1024u); }

template <typename T, int S>
void launch_tb_s(p3maze_ctx* ctx, bool last, const T* src, T* dst) {
    const dim3 blk(kTbX + 2 * S, kTbY + 2 * S, 1);
    const size_t smem = 2 * S * (size_t)blk.x * blk.y * sizeof(T);
    if (last)
        k_diffuse_tb<T, S, kTbX, kTbY, true><<<tb_grid(ctx->N, ctx->zc), blk, smem, ctx->stream>>>(
            ctx->N, ctx->zc, src, dst, (T)ctx->c, ctx->partial);
    else
        k_diffuse_tb<T, S, kTbX, kTbY, false><<<tb_grid(ctx->N, ctx->zc), blk, smem, ctx->stream>>>(
            ctx->N, ctx->zc, src, dst, (T)ctx->c, nullptr);
}

template <typename T>
void launch_diffuse_tb(p3maze_ctx* ctx, int S, bool last, const T* src, T* dst) {
    switch (S) {
        case 1: launch_tb_s<T, 1>(ctx, last, src, dst); break;
        case 2: launch_tb_s<T, 2>(ctx, last, src, dst); break;
        case 3: launch_tb_s<T, 3>(ctx, last, src, dst); break;
        default: launch_tb_s<T, 4>(ctx, last, src, dst); break;
    }
}

// Planes per thread of k_diffuse4 for a tuning value zc (1, 2, 4 or 8).
inline int diffuse4_planes(int zc) { return zc <= 1 ? 1 : zc <= 2 ? 2 : zc <= 4 ? 4 : 8; }


// FP32 quads (N % 4 == 0): the asynchronous-copy temporal blocking, a
// 56 x (32 - 2S) output tile per block.
template <int S>
dim3 tq_grid(int n, int zc) {
    return dim3((n + kTqTX - 1) / kTqTX, (n + tq_tile_y<S>() - 1) / tq_tile_y<S>(), (n + zc - 1) / zc);
}
inline unsigned tq_blocks(int n, int zc, int S) {
    const dim3 g = S == 1 ? tq_grid<1>(n, zc) : S == 2 ? tq_grid<2>(n, zc) : S == 3 ? tq_grid<3>(n, zc)
                                                                                   : tq_grid<4>(n, zc);
    return g.x * g.y * g.z;
}
template <int S>
cudaError_t launch_tq_s(p3maze_ctx* ctx, bool last, bool pdl, const float* src, float* dst) {
    const dim3 g = tq_grid<S>(ctx->N, ctx->zc);
    if (last)
        return launch_maybe_pdl(pdl, k_diffuse_tq<S, true>, g, dim3(kTqThreads), tq_smem_bytes<S>(), ctx->stream,
                                ctx->N, ctx->zc, src, dst, (float)ctx->c, ctx->partial);
    return launch_maybe_pdl(pdl, k_diffuse_tq<S, false>, g, dim3(kTqThreads), tq_smem_bytes<S>(), ctx->stream,
                            ctx->N, ctx->zc, src, dst, (float)ctx->c, (double*)nullptr);
}
cudaError_t launch_diffuse_tq(p3maze_ctx* ctx, int S, bool last, bool pdl, const float* src, float* dst) {
    switch (S) {
        case 1: return launch_tq_s<1>(ctx, last, pdl, src, dst);
        case 2: return launch_tq_s<2>(ctx, last, pdl, src, dst);
        case 3: return launch_tq_s<3>(ctx, last, pdl, src, dst);
        default: return launch_tq_s<4>(ctx, last, pdl, src, dst);
    }
}

// y = H3 (table o (H3 x)) by FFT (n = 32, 64, 128; the table bit-reversed
// and scaled for the kernels): the x-y transforms of x into tmp, the z
// transforms and scaling in place (n = 64, 128: tiles of 32 x columns over
// all SMs; n = 32: one block per ky slice), the x-y transforms into y.  With
// partial given, the last launch also forms the sum of y into *sum_out
// (arrive: its block counter, zero between uses).  pdl_first: the first
// launch may overlap its predecessor.
template <int R>
cudaError_t launch_fht_r(bool pdl_first, bool pdl, cudaStream_t s, const float* x, float* tmp, float* y,
                         const float2* tw, const float* table, double* partial, unsigned* arrive,
                         double* sum_out) {
    constexpr int n = 32 * R;
    const dim3 g(n), b(fht_threads<R>());
    const size_t sm = fht_smem_bytes(n);
    cudaError_t e = launch_maybe_pdl(pdl_first, k_fht_xy<R, false>, g, b, sm, s, x, tmp, tw, (double*)nullptr,
                                     (unsigned*)nullptr, (double*)nullptr);
    if (e == cudaSuccess) {
        if constexpr (R >= 2)
            e = launch_maybe_pdl(pdl, k_fht_cols<R, 1, false>, dim3(n / 32, n), dim3(kFhtColThreads),
                                 fht_cols_smem_bytes(n, 1), s, tmp, (int64_t)n * n, (int64_t)n, tw, table);
        else
            e = launch_maybe_pdl(pdl, k_fht_z<R>, g, b, fht_z_smem_bytes(n), s, tmp, tw, table);
    }
    if (e == cudaSuccess)
        e = launch_maybe_pdl(pdl, k_fht_xy<R, true>, g, b, sm, s, (const float*)tmp, y, tw, partial, arrive, sum_out);
    return e;
}
cudaError_t launch_fht(int n, bool pdl_first, bool pdl, cudaStream_t s, const float* x, float* tmp, float* y,
                       const float2* tw, const float* table, double* partial, unsigned* arrive, double* sum_out) {
    switch (n) {
        case 32: return launch_fht_r<1>(pdl_first, pdl, s, x, tmp, y, tw, table, partial, arrive, sum_out);
        case 64: return launch_fht_r<2>(pdl_first, pdl, s, x, tmp, y, tw, table, partial, arrive, sum_out);
        default: return launch_fht_r<4>(pdl_first, pdl, s, x, tmp, y, tw, table, partial, arrive, sum_out);
    }
}

// n = 32 R >= 192 (192, 256, 320, 384): forward x (q into the ping-pong
// mesh t), forward y, forward z + scaling + inverse z, inverse y (all in
// place in t), inverse x (t into q^s, with the neutrality sum by its last
// block); five launches.  The block counter is the FP64 field update's
// (never in the same context: mixed only).
template <int R>
cudaError_t launch_fht_passes(p3maze_ctx* ctx) {
    const int64_t n = 32 * R;
    const bool pdl = ctx->pdl;
    cudaStream_t s = ctx->stream;
    float* t = (float*)ctx->lev[0].e;
    const float2* tw = (const float2*)ctx->fht_tw;
    const dim3 gr((unsigned)(n * n / 2 / kFhtRowPairs / kFhtRowWarps)), br(32 * kFhtRowWarps);
    const dim3 gc((unsigned)(n / 32), (unsigned)n), bc(kFhtColThreads);
    const size_t s0 = fht_cols_smem_bytes((int)n, 0), s1 = fht_cols_smem_bytes((int)n, 1);
    cudaError_t e = launch_maybe_pdl(pdl, k_fht_rows<R, false>, gr, br, 0, s, (const float*)ctx->q, t, tw,
                                     (double*)nullptr, (unsigned*)nullptr, (double*)nullptr);
    if (e == cudaSuccess)
        e = launch_maybe_pdl(pdl, k_fht_cols<R, 0, false>, gc, bc, s0, s, t, n, n * n, tw, (const float*)nullptr);
    if (e == cudaSuccess)
        e = launch_maybe_pdl(pdl, k_fht_cols<R, 1, false>, gc, bc, s1, s, t, n * n, n, tw, (const float*)ctx->Ssm);
    if (e == cudaSuccess)
        e = launch_maybe_pdl(pdl, k_fht_cols<R, 0, true>, gc, bc, s0, s, t, n, n * n, tw, (const float*)nullptr);
    if (e == cudaSuccess)
        e = launch_maybe_pdl(pdl, k_fht_rows<R, true>, gr, br, 0, s, (const float*)t, (float*)ctx->qs, tw,
                             ctx->partial, &ctx->dmg->arrive_sum, ctx->dscal + S_QSUM);
    return e;
}

// Spectral smoothing by FFT: q into q^s through the smoothing ping-pong
// mesh; the last launch's last block forms the neutrality sum from the
// per-plane (or per-block) sums.  The block counter is the FP64 field
// update's (mixed only, so never used by both in one context).
cudaError_t launch_fht_smoothing(p3maze_ctx* ctx) {
    switch (ctx->N) {
        case 192: return launch_fht_passes<6>(ctx);
        case 256: return launch_fht_passes<8>(ctx);
        case 320: return launch_fht_passes<10>(ctx);
        case 384: return launch_fht_passes<12>(ctx);
        default: break;
    }
    return launch_fht(ctx->N, ctx->pdl, ctx->pdl, ctx->stream, (const float*)ctx->q, (float*)ctx->lev[0].e,
                      (float*)ctx->qs, (const float2*)ctx->fht_tw, (const float*)ctx->Ssm, ctx->partial,
                      &ctx->dmg->arrive_sum, ctx->dscal + S_QSUM);
}
inline int fht_smoothing_launches(int n) { return fht_passes(n) ? 5 : 3; }

// Position of each frequency 0..n-1 in the forward transforms' output:
// n = Q m (m a power of two), frequency f = k + Q r at rev_m(r) + m k
// (Q = 1: plain bit reversal).
std::vector<int> fht_positions(int n) {
    const int Q = fht_q(n), m = n / Q;
    int bits = 0;
    while ((1 << bits) < m) ++bits;
    std::vector<int> pos(n);
    for (int f = 0; f < n; ++f) {
        const int k = f % Q, r0 = f / Q;
        int r = 0;
        for (int b = 0; b < bits; ++b) r |= ((r0 >> b) & 1) << (bits - 1 - b);
        pos[f] = r + m * k;
    }
    return pos;
}

// Twiddles exp(-2 pi i k / n), k < n / 2, then for a mixed-radix length the
// Q roots exp(-2 pi i j / Q); from FP64.
std::vector<float2> fht_twiddle_table(int n) {
    const int Q = fht_q(n);
    std::vector<float2> tw(n / 2 + (Q > 1 ? Q : 0));
    for (int k = 0; k < n / 2; ++k)
        tw[k] = make_float2((float)std::cos(2.0 * kPi * k / n), (float)-std::sin(2.0 * kPi * k / n));
    if (Q > 1)
        for (int j = 0; j < Q; ++j)
            tw[n / 2 + j] = make_float2((float)std::cos(2.0 * kPi * j / Q), (float)-std::sin(2.0 * kPi * j / Q));
    return tw;
}
inline size_t fht_twiddle_count(int n) { return (size_t)(n / 2 + (fht_q(n) > 1 ? fht_q(n) : 0)); }

// Raise the shared-memory limit of the FFT kernels for n points per axis.
// The limit is an attribute of the kernel, shared by every context in the
// process: only ever raise it.
cudaError_t fht_raise_smem(int n) {
    auto raise = [](const void* fn, size_t sm) {
        cudaFuncAttributes fa{};
        cudaError_t e = cudaFuncGetAttributes(&fa, fn);
        if (e == cudaSuccess && (size_t)fa.maxDynamicSharedSizeBytes < sm)
            e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        return e;
    };
    if (fht_passes(n)) {
        const void* k0[4] = {(const void*)k_fht_cols<6, 0, false>, (const void*)k_fht_cols<8, 0, false>,
                             (const void*)k_fht_cols<10, 0, false>, (const void*)k_fht_cols<12, 0, false>};
        const void* k0i[4] = {(const void*)k_fht_cols<6, 0, true>, (const void*)k_fht_cols<8, 0, true>,
                              (const void*)k_fht_cols<10, 0, true>, (const void*)k_fht_cols<12, 0, true>};
        const void* k1[4] = {(const void*)k_fht_cols<6, 1, false>, (const void*)k_fht_cols<8, 1, false>,
                             (const void*)k_fht_cols<10, 1, false>, (const void*)k_fht_cols<12, 1, false>};
        const int i = n == 192 ? 0 : n == 256 ? 1 : n == 320 ? 2 : 3;
        cudaError_t e = raise(k0[i], fht_cols_smem_bytes(n, 0));
        if (e == cudaSuccess) e = raise(k0i[i], fht_cols_smem_bytes(n, 0));
        if (e == cudaSuccess) e = raise(k1[i], fht_cols_smem_bytes(n, 1));
        return e;
    }
    const size_t sxy = fht_smem_bytes(n), sz = fht_z_smem_bytes(n), sc = fht_cols_smem_bytes(n, 1);
    const void* k[3];
    size_t szk = sz;
    if (n == 32) {
        k[0] = (const void*)k_fht_xy<1, false>;
        k[1] = (const void*)k_fht_xy<1, true>;
        k[2] = (const void*)k_fht_z<1>;
    } else if (n == 64) {
        k[0] = (const void*)k_fht_xy<2, false>;
        k[1] = (const void*)k_fht_xy<2, true>;
        k[2] = (const void*)k_fht_cols<2, 1, false>;
        szk = sc;
    } else {
        k[0] = (const void*)k_fht_xy<4, false>;
        k[1] = (const void*)k_fht_xy<4, true>;
        k[2] = (const void*)k_fht_cols<4, 1, false>;
        szk = sc;
    }
    cudaError_t e = raise(k[0], sxy);
    if (e == cudaSuccess) e = raise(k[1], sxy);
    if (e == cudaSuccess) e = raise(k[2], szk);
    return e;
}

// All diffusion steps of `members` meshes (table on the device, N <= nmax,
// all with cluster size cs) in one launch, one cluster of cs CTAs per mesh.
cudaError_t launch_cluster_smoothing(const ClusterMesh* tab, int members, int cs, int nmax, cudaStream_t s,
                                     bool pdl) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cs * members);
    cfg.blockDim = dim3(kClThreads);
    cfg.dynamicSmemBytes = cluster_smem_bytes(nmax, cs);
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 2 : 1;
    return cudaLaunchKernelEx(&cfg, k_diffuse_cluster, tab);
}

// Whether the device co-schedules clusters of cs CTAs of the smoothing
// kernel with its largest shared-memory need (asked once per size and
// process).
bool cluster_smoothing_supported(int cs) {
    static int cached[kClMaxCTAs + 1] = {-1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1};
    if (cs < 1 || cs > kClMaxCTAs) return false;
    if (cached[cs] >= 0) return cached[cs] == 1;
    const size_t smem = kClSmemBudget + 16;
    cudaError_t e = cudaFuncSetAttribute(k_diffuse_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_diffuse_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int nclusters = 0;
    if (e == cudaSuccess) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(cs);
        cfg.blockDim = dim3(kClThreads);
        cfg.dynamicSmemBytes = smem;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = cs;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        e = cudaOccupancyMaxActiveClusters(&nclusters, k_diffuse_cluster, &cfg);
    }
    if (e != cudaSuccess) cudaGetLastError();  // not available: the per-step kernels are used
    cached[cs] = (e == cudaSuccess && nclusters >= 1) ? 1 : 0;
    return cached[cs] == 1;
}

template <int Z>
cudaError_t diffuse4_z(bool sum, bool pdl, dim3 g, cudaStream_t s, int n, const float* src, float* dst, float c,
                       double* partial) {
    if (sum) return launch_maybe_pdl(pdl, k_diffuse4<Z, true>, g, kB3, 0, s, n, src, dst, c, partial);
    return launch_maybe_pdl(pdl, k_diffuse4<Z, false>, g, kB3, 0, s, n, src, dst, c, (double*)nullptr);
}

cudaError_t launch_diffuse4(int zc4, bool sum, bool pdl, dim3 g, cudaStream_t s, int n, const float* src,
                            float* dst, float c, double* partial) {
    switch (zc4) {
        case 1: return diffuse4_z<1>(sum, pdl, g, s, n, src, dst, c, partial);
        case 2: return diffuse4_z<2>(sum, pdl, g, s, n, src, dst, c, partial);
        case 4: return diffuse4_z<4>(sum, pdl, g, s, n, src, dst, c, partial);
        default: return diffuse4_z<8>(sum, pdl, g, s, n, src, dst, c, partial);
    }
}

template <int Z>
cudaError_t diffuse4x2_z(bool sum, bool pdl, dim3 g, cudaStream_t s, int n, const float* src, float* dst,
                         const float a[4], double* partial) {
    if (sum)
        return launch_maybe_pdl(pdl, k_diffuse4x2<Z, true>, g, kB3, 0, s, n, src, dst, a[0], a[1], a[2], a[3], partial);
    return launch_maybe_pdl(pdl, k_diffuse4x2<Z, false>, g, kB3, 0, s, n, src, dst, a[0], a[1], a[2], a[3],
                            (double*)nullptr);
}

cudaError_t launch_diffuse4x2(int zc4, bool sum, bool pdl, dim3 g, cudaStream_t s, int n, const float* src,
                              float* dst, const float a[4], double* partial) {
    switch (zc4) {
        case 1: return diffuse4x2_z<1>(sum, pdl, g, s, n, src, dst, a, partial);
        case 2: return diffuse4x2_z<2>(sum, pdl, g, s, n, src, dst, a, partial);
        case 4: return diffuse4x2_z<4>(sum, pdl, g, s, n, src, dst, a, partial);
        default: return diffuse4x2_z<8>(sum, pdl, g, s, n, src, dst, a, partial);
    }
}

template <typename T>
int spread_assign(p3maze_ctx* ctx) {
    cudaStream_t s = ctx->stream;
    stage_begin(ctx, P3MAZE_ST_SPREAD);
    // deterministic tiled assignment: every mesh point written once
    if constexpr (sizeof(T) == 4) {
        if (ctx->N % 4 == 0)
            CK(launch_maybe_pdl(ctx->pdl, k_spread_tile<float, MeshPt, true>, spread_grid(ctx->N), dim3(kSpThreads),
                                spread_smem_bytes<float>(), s, ctx->N, ctx->nc, (const int*)ctx->start,
                                (const MeshPt*)ctx->mp, ctx->inv_h, (float*)ctx->q));
        else
            CK(launch_maybe_pdl(ctx->pdl, k_spread_tile<float, MeshPt, false>, spread_grid(ctx->N), dim3(kSpThreads),
                                spread_smem_bytes<float>(), s, ctx->N, ctx->nc, (const int*)ctx->start,
                                (const MeshPt*)ctx->mp, ctx->inv_h, (float*)ctx->q));
    } else {
        CK(launch_maybe_pdl(ctx->pdl, k_spread_tile<double, PQ, false>, spread_grid(ctx->N), dim3(kSpThreads),
                            spread_smem_bytes<double>(), s, ctx->N, ctx->nc, (const int*)ctx->start,
                            (const PQ*)ctx->xq, ctx->inv_h, (double*)ctx->q));
    }
    count(ctx, P3MAZE_ST_SPREAD);
    stage_end(ctx, P3MAZE_ST_SPREAD);
    CKL();
    return P3MAZE_OK;
}

// K diffusion steps q -> q^s and the neutrality sum (Sec. 2; reading A2).
template <typename T>
int smooth(p3maze_ctx* ctx) {
    cudaStream_t s = ctx->stream;
    stage_begin(ctx, P3MAZE_ST_SMOOTH);
    if (ctx->K == 0) {
        CK(cudaMemcpyAsync(ctx->qs, ctx->q, sizeof(T) * ctx->P, cudaMemcpyDeviceToDevice, s));
        k_sum_partial<T><<<kReduceBlocks, P3_THREADS, 0, s>>>(ctx->P, (const T*)ctx->qs, ctx->partial);
        k_sum_final<<<1, P3_THREADS, 0, s>>>(kReduceBlocks, ctx->partial, ctx->dscal + S_QSUM);
        count(ctx, P3MAZE_ST_SMOOTH, 2);
    } else if constexpr (sizeof(T) == 4) {
        T* tmp[2] = {(T*)ctx->lev[0].e, (T*)ctx->lev[0].r};
        const T* src = (const T*)ctx->q;
        if (ctx->fuse == 6 && ctx->fht_tw) {
            // all K steps at once in the Hartley basis, each 1D transform by FFT
            CK(launch_fht_smoothing(ctx));
            count(ctx, P3MAZE_ST_SMOOTH, fht_smoothing_launches(ctx->N));
        } else if (ctx->fuse == 6) {
            // all K steps at once in the Hartley basis (N <= 64): forward
            // transform, scale by (1 + c lambda_k)^K / N^3, inverse transform
            const Level& L0 = ctx->lev[0];
            const size_t sm = coarse_smem_bytes(ctx->N, sizeof(float));
            const dim3 gc(ctx->N), bc(kCoarseThreads);
            k_coarse_xy<float><<<gc, bc, sm, s>>>(ctx->N, (const float*)ctx->q, (float*)L0.t, (const float*)L0.H);
            k_coarse_z<float><<<gc, bc, sm, s>>>(ctx->N, (float*)L0.t, (const float*)L0.H, (const float*)ctx->Ssm);
            k_coarse_xy<float><<<gc, bc, sm, s>>>(ctx->N, (const float*)L0.t, (float*)ctx->qs, (const float*)L0.H);
            k_sum_partial<float><<<kReduceBlocks, P3_THREADS, 0, s>>>(ctx->P, (const float*)ctx->qs, ctx->partial);
            k_sum_final<<<1, P3_THREADS, 0, s>>>(kReduceBlocks, ctx->partial, ctx->dscal + S_QSUM);
            count(ctx, P3MAZE_ST_SMOOTH, 5);
        } else if (ctx->fuse == 5) {
            // every step in one launch, the mesh resident in a cluster's shared memory
            const int cs = ctx->cl_ctas ? ctx->cl_ctas : cluster_size_for(ctx->N, 1, ctx->nsm);
            CK(launch_cluster_smoothing(ctx->cltab, 1, cs, ctx->N, s, false));
            count(ctx, P3MAZE_ST_SMOOTH, 1);
        } else if (ctx->fuse > 2) {
            // S = fuse steps per launch (temporal blocking), the remainder first
            const bool quads = ctx->N % 4 == 0;
            int done = 0, launches = 0, last_S = 1;
            while (done < ctx->K) {
                const int rem = (ctx->K - done) % ctx->fuse;
                const int S = (done == 0 && rem) ? rem : std::min(ctx->fuse, ctx->K - done);
                const bool last = done + S == ctx->K;
                T* dst = last ? (T*)ctx->qs : tmp[launches & 1];
                if (quads)
                    CK(launch_diffuse_tq(ctx, S, last, ctx->pdl && launches > 0, (const float*)src, (float*)dst));
                else
                    launch_diffuse_tb<T>(ctx, S, last, src, dst);
                src = dst;
                done += S;
                last_S = S;
                ++launches;
            }
            const int nb = quads ? (int)tq_blocks(ctx->N, ctx->zc, last_S) : (int)tb_blocks(ctx->N, ctx->zc);
            k_sum_final<<<1, 1024, 0, s>>>(nb, ctx->partial, ctx->dscal + S_QSUM);
            count(ctx, P3MAZE_ST_SMOOTH, launches + 1);
        } else if (ctx->N % 4 == 0) {
            // four points per thread, zc4 planes per thread; fuse 2: two steps
            // per launch as one 25-point stencil (a single step first if K is odd)
            const int zc4 = diffuse4_planes(ctx->zc);
            const dim3 g((ctx->N / 4 + P3_BX - 1) / P3_BX, (ctx->N + P3_BY - 1) / P3_BY, (ctx->N + zc4 - 1) / zc4);
            const double c = ctx->c;
            const float a[4] = {(float)(1.0 - 12.0 * c + 42.0 * c * c), (float)(2.0 * c - 12.0 * c * c),
                                (float)(c * c), (float)(2.0 * c * c)};
            int done = 0, launches = 0;
            while (done < ctx->K) {
                const int S = (ctx->fuse == 2 && (ctx->K - done) % 2 == 0) ? 2 : 1;
                const bool last = done + S == ctx->K;
                T* dst = last ? (T*)ctx->qs : tmp[launches & 1];
                const bool pdl = ctx->pdl && launches > 0;  // overlap with the previous diffusion launch
                if (S == 2)
                    CK(launch_diffuse4x2(zc4, last, pdl, g, s, ctx->N, (const float*)src, (float*)dst, a,
                                         last ? ctx->partial : nullptr));
                else
                    CK(launch_diffuse4(zc4, last, pdl, g, s, ctx->N, (const float*)src, (float*)dst, (float)ctx->c,
                                       last ? ctx->partial : nullptr));
                src = dst;
                done += S;
                ++launches;
            }
            CK(launch_maybe_pdl(ctx->pdl, k_sum_final, dim3(1), dim3(1024), 0, s, (int)(g.x * g.y * g.z),
                                ctx->partial, ctx->dscal + S_QSUM));
            count(ctx, P3MAZE_ST_SMOOTH, launches + 1);
        } else {
            for (int k = 0; k < ctx->K; ++k) {
                const bool last = k == ctx->K - 1;
                T* dst = last ? (T*)ctx->qs : tmp[k & 1];
                if (last)
                    k_diffuse<T, true><<<gz(ctx->N, ctx->zc), kB3, 0, s>>>(ctx->N, ctx->zc, src, dst, (T)ctx->c,
                                                                          ctx->partial);
                else
                    k_diffuse<T, false><<<gz(ctx->N, ctx->zc), kB3, 0, s>>>(ctx->N, ctx->zc, src, dst, (T)ctx->c,
                                                                           nullptr);
                src = dst;
            }
            k_sum_final<<<1, 1024, 0, s>>>((int)gz_blocks(ctx->N, ctx->zc), ctx->partial, ctx->dscal + S_QSUM);
            count(ctx, P3MAZE_ST_SMOOTH, ctx->K + 1);
        }
    } else {
        T* tmp[2] = {(T*)ctx->lev[0].e, (T*)ctx->lev[0].r};
        const T* src = (const T*)ctx->q;
        for (int k = 0; k < ctx->K; ++k) {
            const bool last = k == ctx->K - 1;
            T* dst = last ? (T*)ctx->qs : tmp[k & 1];
            if (last)
                k_diffuse<T, true><<<gz(ctx->N, ctx->zc), kB3, 0, s>>>(ctx->N, ctx->zc, src, dst, (T)ctx->c, ctx->partial);
            else
                k_diffuse<T, false><<<gz(ctx->N, ctx->zc), kB3, 0, s>>>(ctx->N, ctx->zc, src, dst, (T)ctx->c, nullptr);
            src = dst;
        }
        // neutrality: the last step's block sums (FP64) give mean(q^s)
        k_sum_final<<<1, 1024, 0, s>>>((int)gz_blocks(ctx->N, ctx->zc), ctx->partial, ctx->dscal + S_QSUM);
        count(ctx, P3MAZE_ST_SMOOTH, ctx->K + 1);
    }
    CKL();
    stage_end(ctx, P3MAZE_ST_SMOOTH);
    return P3MAZE_OK;
}

template <typename T>
int spread_smooth(p3maze_ctx* ctx) {
    int rc = spread_assign<T>(ctx);
    return rc ? rc : smooth<T>(ctx);
}

// One V-cycle on M e_l = b_l: levels above the coarse level by grid kernels
// (red-black Gauss-Seidel, fused residual + restriction, trilinear
// prolongation); the coarse level solved exactly by separable Hartley
// transforms (three launches).
template <typename T>
int vcycle(p3maze_ctx* ctx, int l, bool pdl_first) {
    cudaStream_t s = ctx->stream;
    Level& L = ctx->lev[l];
    T* e = (T*)L.e;
    T* b = (T*)L.b;
    // every launch but the first follows a kernel of this V-cycle and may
    // overlap its tail (programmatic dependent launch)
    bool pdl = ctx->pdl && pdl_first;
    auto go = [&](auto kernel, dim3 g, dim3 blk, size_t smem, auto... args) {
        const cudaError_t err = launch_maybe_pdl(pdl, kernel, g, blk, smem, s, args...);
        pdl = ctx->pdl;
        return err;
    };
    if (l == ctx->lc && L.tw) {
        CK(launch_fht(L.n, pdl, ctx->pdl, s, (const float*)b, (float*)L.t, (float*)e, (const float2*)L.tw,
                      (const float*)L.D, nullptr, nullptr, nullptr));
        count(ctx, P3MAZE_ST_SOLVE, 3);
        L.fin = e;
        return P3MAZE_OK;
    }
    if (l == ctx->lc) {
        const size_t sm = coarse_smem_bytes(L.n, sizeof(T));
        const dim3 gc(L.n), bc(kCoarseThreads);
        CK(go(k_coarse_xy<T>, gc, bc, sm, L.n, (const T*)b, (T*)L.t, (const T*)L.H));
        CK(go(k_coarse_z<T>, gc, bc, sm, L.n, (T*)L.t, (const T*)L.H, (const T*)L.D));
        CK(go(k_coarse_xy<T>, gc, bc, sm, L.n, (const T*)L.t, e, (const T*)L.H));
        count(ctx, P3MAZE_ST_SOLVE, 3);
        L.fin = e;
        return P3MAZE_OK;
    }
    Level& C = ctx->lev[l + 1];
    if (ctx->nu1 == 0) {
        CK(cudaMemsetAsync(e, 0, sizeof(T) * L.pts, s));
        pdl = false;  // the next launch follows a memset
    }
    // FP32 levels with N % 4 == 0 take the four-points-per-thread kernels
    const bool quads = sizeof(T) == 4 && L.n % 4 == 0;
    int launches = 0;
    // cur: the buffer holding the level's correction.  `count` full red-black
    // sweeps, colour pa first: on FP32 quad levels of at most 64^3 one
    // out-of-place launch per sweep (cur -> the other buffer), else two
    // in-place half sweeps.  Measured: the one-launch sweep takes 5.9 us at
    // 64^3 against 2 x 3.9 us, but 20 us at 128^3 against 2 x 7.6 us and
    // 164 us at 320^3 against 2 x 73 us (it forms the first colour on three
    // rows per thread).
    T* cur = e;
    auto sweeps = [&](int count, int pa) -> int {
        const bool pairs = quads && ctx->sweep_fuse && L.e2 && L.n <= kSweepFuseMaxN;
        for (int k = 0; k < count; ++k) {
            if (!pairs) {
                CK(go(k_rbgs<T>, g3h(L.n), kB3, 0, L.n, cur, (const T*)b, pa, 0));
                CK(go(k_rbgs<T>, g3h(L.n), kB3, 0, L.n, cur, (const T*)b, 1 - pa, 0));
                launches += 2;
                continue;
            }
            if constexpr (sizeof(T) == 4) {
                const int zc = L.n >= 128 ? 4 : 2;
                const dim3 g((L.n / 4 + P3_BX - 3) / (P3_BX - 2), (L.n + P3_BY - 1) / P3_BY, (L.n + zc - 1) / zc);
                const float* src = (const float*)cur;
                float* dst = (float*)(cur == e ? (T*)L.e2 : e);
                if (pa == 0 && zc == 4) CK(go(k_rbgs_pair4<0, 4>, g, kB3, 0, L.n, src, dst, (const float*)b));
                else if (pa == 0) CK(go(k_rbgs_pair4<0, 2>, g, kB3, 0, L.n, src, dst, (const float*)b));
                else if (zc == 4) CK(go(k_rbgs_pair4<1, 4>, g, kB3, 0, L.n, src, dst, (const float*)b));
                else CK(go(k_rbgs_pair4<1, 2>, g, kB3, 0, L.n, src, dst, (const float*)b));
                cur = (T*)dst;
                launches += 1;
            }
        }
        return P3MAZE_OK;
    };
    for (int it = 0; it < ctx->nu1; ++it) {
        if (it == 0) {
            // both colours from e = 0
            if constexpr (sizeof(T) == 4) {
                if (quads) {
                    const int zc = L.n >= 256 ? 4 : 2;
                    const dim3 g((L.n / 4 + P3_BX - 1) / P3_BX, (L.n + P3_BY - 1) / P3_BY, (L.n + zc - 1) / zc);
                    if (zc == 4) CK(go(k_rbgs_first4<4>, g, kB3, 0, L.n, (float*)e, (const float*)b));
                    else CK(go(k_rbgs_first4<2>, g, kB3, 0, L.n, (float*)e, (const float*)b));
                } else {
                    CK(go(k_rbgs_first<T>, g3(L.n), kB3, 0, L.n, e, (const T*)b));
                }
            } else {
                CK(go(k_rbgs_first<T>, g3(L.n), kB3, 0, L.n, e, (const T*)b));
            }
            launches += 1;
        } else {
            // the remaining pre-sweeps at once
            int rc = sweeps(ctx->nu1 - 1, 0);
            if (rc) return rc;
            break;
        }
    }
    if (C.n >= 128)
        CK(go(k_resid_restrict_z<T, 4>, gz(C.n, 4), kB3, 0, C.n, (const T*)cur, (const T*)b, (T*)C.b));
    else
        CK(go(k_resid_restrict_z<T, 2>, gz(C.n, 2), kB3, 0, C.n, (const T*)cur, (const T*)b, (T*)C.b));
    count(ctx, P3MAZE_ST_SOLVE, launches + 1);
    launches = 0;
    int rc = vcycle<T>(ctx, l + 1, true);
    if (rc) return rc;
    const T* ec = (const T*)C.fin;  // the coarse correction, wherever its V-cycle left it
    if constexpr (sizeof(T) == 4) {
        if (quads) {
            const dim3 g((L.n / 4 + P3_BX - 1) / P3_BX, (L.n + P3_BY - 1) / P3_BY, L.n / 2);
            CK(go(k_prolong_add4, g, kB3, 0, L.n, (const float*)ec, (float*)cur));
        } else {
            CK(go(k_prolong_add<T>, g3(L.n), kB3, 0, L.n, ec, cur));
        }
    } else {
        CK(go(k_prolong_add<T>, g3(L.n), kB3, 0, L.n, ec, cur));
    }
    rc = sweeps(ctx->nu2, 1);
    if (rc) return rc;
    count(ctx, P3MAZE_ST_SOLVE, 1 + launches);
    L.fin = cur;
    return P3MAZE_OK;
}

// Arguments of the check fused into the mixed-precision residual kernels.
// P3M: max|M phi + (4pi/h) q^s| = (4pi/h) max|M y - sigma_p| for phi = phi_p - (4pi/h) y.
CheckArgs check_args(p3maze_ctx* ctx, cudaGraphConditionalHandle h, int use_handle, double* sum_out = nullptr) {
    return CheckArgs{ctx->bmax, ctx->tol * ctx->res_unit / ctx->res_scale, ctx->itmax, ctx->dmg, h, use_handle,
                     reinterpret_cast<long long*>(ctx->partial), reinterpret_cast<long long*>(sum_out)};
}

// FP64: residual of the current y, then the check kernel.
template <typename T>
void launch_resid_check(p3maze_ctx* ctx, cudaGraphConditionalHandle h, int use_handle) {
    cudaStream_t s = ctx->stream;
    const dim3 gr = resid_grid(ctx->N);
    k_resid_fine<T><<<gr, kB3, 0, s>>>(ctx->N, ctx->yh[0], ctx->sig, (T*)ctx->lev[0].b, ctx->rfin, ctx->bmax);
    const CheckArgs ck = check_args(ctx, h, use_handle);
    k_mg_check<<<1, 1024, 0, s>>>(ck.bmax, (int)(gr.x * gr.y * gr.z), ck.tol, ck.itmax, ck.st, h, use_handle);
    count(ctx, P3MAZE_ST_SOLVE, 2);
}

// One correction iteration: V-cycle, then y += e with the new residual and
// the check (mixed: one fused kernel; FP64: three kernels).
template <typename T>
int launch_iteration(p3maze_ctx* ctx, cudaGraphConditionalHandle h, int use_handle) {
    int rc = vcycle<T>(ctx, 0, false);
    if (rc) return rc;
    if (ctx->prec == P3MAZE_MIXED) {
        // the increments' sum goes to slot P of the correction (gauge mode)
        CK(launch_maybe_pdl(ctx->pdl, k_resid_update_fix, resid_grid(ctx->N), kB3, 0, ctx->stream, ctx->N,
                            fx(ctx->yh[0]), (const float*)ctx->lev[0].fin, fx(ctx->rfin), (float*)ctx->lev[0].b,
                            check_args(ctx, h, use_handle, ctx->yh[0] + ctx->P)));
        count(ctx, P3MAZE_ST_SOLVE);
    } else {
        k_add_correction<T><<<nblk(ctx->P), P3_THREADS, 0, ctx->stream>>>(ctx->P, ctx->yh[0],
                                                                          (const T*)ctx->lev[0].fin);
        count(ctx, P3MAZE_ST_SOLVE);
        launch_resid_check<T>(ctx, h, use_handle);
    }
    return P3MAZE_OK;
}

// Read the check's decision on the host (eager steps).
int host_decision(p3maze_ctx* ctx, bool* cont) {
    CK(cudaMemcpyAsync(ctx->hmg, ctx->dmg, sizeof(MGState), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    *cont = !ctx->hmg->status && ctx->hmg->cont;
    return P3MAZE_OK;
}

// Correction solve to tol (Eqs. 16, 20) after the initial residual and check
// have been launched.  Eagerly: the host reads the decision after every
// check.  While capturing: a while node whose body is one iteration and
// whose condition the check sets, so a step needs no host round trip.
template <typename T>
int solve_loop(p3maze_ctx* ctx, cudaGraphConditionalHandle h) {
    cudaStream_t s = ctx->stream;
    if (!ctx->capturing) {
        for (;;) {
            CKL();
            bool cont = false;
            int rc = host_decision(ctx, &cont);
            if (rc) return rc;
            if (!cont) break;
            rc = launch_iteration<T>(ctx, 0, 0);
            if (rc) return rc;
            ctx->eager_iters += 1;
        }
        return P3MAZE_OK;
    }
    cudaStreamCaptureStatus cs;
    cudaGraph_t g;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    CK(cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &nd));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    CK(cudaGraphAddNode(&node, g, deps, nullptr, nd, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    CK(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    // populate the body on the second stream
    CK(cudaStreamBeginCaptureToGraph(ctx->body_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    ctx->stream = ctx->body_stream;
    ctx->in_body = true;
    ctx->body_launches = 0;
    int brc = launch_iteration<T>(ctx, h, 1);
    ctx->in_body = false;
    ctx->stream = s;
    if (brc) {
        cudaGraph_t junk = nullptr;
        cudaStreamEndCapture(ctx->body_stream, &junk);
        return brc;
    }
    cudaError_t le = cudaGetLastError();
    cudaGraph_t out = nullptr;
    CK(cudaStreamEndCapture(ctx->body_stream, &out));
    if (le != cudaSuccess) return fail(ctx, P3MAZE_ERR_CUDA, std::string("body launch: ") + cudaGetErrorString(le));
    return P3MAZE_OK;
}

// Verlet prediction, constraint residual, correction solve and field update
// (Eqs. 16-17, 20; supporting information Sec. 1).
template <typename T>
int solve_field(p3maze_ctx* ctx, int pred_order) {
    cudaStream_t s = ctx->stream;
    const int ik = ctx->icur, ikm1 = 1 - ctx->icur;
    const bool fixp = ctx->prec == P3MAZE_MIXED;
    // the while node's condition handle exists before the first check
    cudaGraphConditionalHandle h = 0;
    if (ctx->capturing) {
        cudaStreamCaptureStatus cs;
        cudaGraph_t g;
        CK(cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, nullptr, nullptr, nullptr));
        CK(cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault));
    }
    const int use_handle = ctx->capturing ? 1 : 0;
    stage_begin(ctx, P3MAZE_ST_PREDICT);
    if (fixp) {
#define P3_PREDICT(ORD)                                                                                           \
    CK(launch_maybe_pdl(ctx->pdl, k_predict_resid_fix<ORD>, resid_grid(ctx->N), kB3, 0, s, ctx->N,                \
                        fx(ctx->psi[ik]), fx(ctx->psi[ikm1]), (const float*)ctx->qs, ctx->dscal + S_QSUM,         \
                        1.0 / (double)ctx->P, (float)(4.0 * kPi / ctx->h), fx(ctx->yh[1]), fx(ctx->yh[2]),       \
                        fx(ctx->yh[3]), fx(ctx->yh[0]), fx(ctx->rfin), (float*)ctx->lev[0].b,                    \
                        check_args(ctx, h, use_handle)))
        switch (pred_order) {
            case 0: P3_PREDICT(0); break;
            case 1: P3_PREDICT(1); break;
            case 2: P3_PREDICT(2); break;
            default: P3_PREDICT(3); break;
        }
#undef P3_PREDICT
    } else
        k_predict<T><<<nblk(ctx->P), P3_THREADS, 0, s>>>(ctx->P, ctx->psi[ik], ctx->psi[ikm1], (const T*)ctx->qs,
                                                         ctx->dscal + S_QSUM, 1.0 / (double)ctx->P, ctx->yh[1],
                                                         ctx->yh[2], ctx->yh[3], pred_order, ctx->sig, ctx->yh[0]);
    CKL();
    count(ctx, P3MAZE_ST_PREDICT, 1);
    stage_end(ctx, P3MAZE_ST_PREDICT);
    stage_begin(ctx, P3MAZE_ST_SOLVE);
    if (!fixp) launch_resid_check<T>(ctx, h, use_handle);
    int rc = solve_loop<T>(ctx, h);
    if (rc) return rc;
    stage_end(ctx, P3MAZE_ST_SOLVE);
    stage_begin(ctx, P3MAZE_ST_UPDATE);
    if (fixp)
        CK(launch_maybe_pdl(ctx->pdl, k_update_fix, dim3(nblk(ctx->P)), dim3(P3_THREADS), 0, s, ctx->P,
                            fx(ctx->phi[ik]), fx(ctx->phi[ikm1]), fx(ctx->psi[ikm1]), fx(ctx->yh[0]), fx(ctx->rfin),
                            (const float*)ctx->qs, ctx->dscal + S_QSUM, 1.0 / (double)ctx->P,
                            (float)(4.0 * kPi / ctx->h), ctx->phi32));
    else
        k_update<T><<<update_blocks(ctx->N), P3_THREADS, 0, s>>>(
            ctx->P, ctx->phi[ik], ctx->phi[ikm1], ctx->psi[ikm1], ctx->yh[0], ctx->rfin, (const T*)ctx->qs,
            ctx->dscal + S_QSUM, 1.0 / (double)ctx->P, 4.0 * kPi / ctx->h, ctx->phi32, ctx->partial,
            &ctx->dmg->arrive_sum);
    count(ctx, P3MAZE_ST_UPDATE);
    stage_end(ctx, P3MAZE_ST_UPDATE);
    CKL();
    ctx->icur = ikm1;
    return P3MAZE_OK;
}

// Short-range pair forces on the pair stream (forked from the main stream
// after the cell list; joined before the interpolation).
int pair_forces(p3maze_ctx* ctx) {
    const double rc2 = ctx->rc * ctx->rc;
    const double halfL2 = 0.25 * ctx->L * ctx->L;
    const bool mixed = ctx->prec == P3MAZE_MIXED;
    cudaStream_t main = ctx->stream;
    CK(cudaEventRecord(ctx->ev_fork, main));
    CK(cudaStreamWaitEvent(ctx->pair_stream, ctx->ev_fork, 0));
    // the positions of this step are final (drift done): p3maze_step_host's
    // copy-out may start.  Recorded here, beside the fork's own event node,
    // so that no chain of dependent launches is cut by one more node (an
    // external record when capturing: an event node of the step graph)
    CK(ctx->capturing ? cudaEventRecordWithFlags(ctx->ev_drift, main, cudaEventRecordExternal)
                      : cudaEventRecord(ctx->ev_drift, main));
    ctx->stream = ctx->pair_stream;
    cudaStream_t s = ctx->stream;
    stage_begin(ctx, P3MAZE_ST_PAIR);
    const int nbox = (ctx->nc + 1) / 2;
    const unsigned nboxes = (unsigned)nbox * nbox * nbox;
    const unsigned pb = ctx->pair_blocks > 0 ? std::min(nboxes, (unsigned)ctx->pair_blocks) : nboxes;
#define PAIR3(KIND, MOL, SH)                                                                            \
    do {                                                                                                \
        if (mixed)                                                                                      \
            k_pair<KIND, float, 768, MOL, SH><<<pb, P3_THREADS, 0, s>>>(ctx->np, ctx->xl32, ctx->ts,    \
                ctx->ms, ctx->start, ctx->nc, nbox, ctx->lcell, rc2, halfL2, ctx->alpha, ctx->ke_pair,  \
                ctx->tab, ctx->Fs, ctx->ecs, ctx->evs, ctx->wsr);                                       \
        else                                                                                            \
            k_pair<KIND, double, 512, MOL, SH><<<pb, P3_THREADS, 0, s>>>(ctx->np, ctx->xl64, ctx->ts,   \
                ctx->ms, ctx->start, ctx->nc, nbox, ctx->lcell, rc2, halfL2, ctx->alpha, ctx->ke_pair,  \
                ctx->tab, ctx->Fs, ctx->ecs, ctx->evs, ctx->wsr);                                       \
    } while (0)
#define PAIR(KIND, MOL)                       \
    do {                                      \
        if (shift) PAIR3(KIND, MOL, true);    \
        else PAIR3(KIND, MOL, false);         \
    } while (0)
    const bool mol = ctx->nmol > 0;
    const bool shift = ctx->sr_shift == P3MAZE_SR_SHIFT_FORCE;
    if (ctx->tab.kind == 1) {
        if (mol) PAIR(1, true);
        else PAIR(1, false);
    } else if (ctx->tab.kind == 2) {
        if (mol) PAIR(2, true);
        else PAIR(2, false);
    } else {
        if (mol) PAIR(0, true);
        else PAIR(0, false);
    }
#undef PAIR
#undef PAIR3
    count(ctx, P3MAZE_ST_PAIR);
    stage_end(ctx, P3MAZE_ST_PAIR);
    ctx->stream = main;
    CKL();
    CK(cudaEventRecord(ctx->ev_join, ctx->pair_stream));
    return P3MAZE_OK;
}

// Join the pair branch, then interpolate the mesh force and add the bonded
// terms.  kick: the step's closing half kick follows; the mixed
// finite-difference interpolation does it itself when nothing else is added
// to F (no molecules), and *kicked says so.
int gather_forces(p3maze_ctx* ctx, bool kick, bool* kicked) {
    cudaStream_t s = ctx->stream;
    const bool mixed = ctx->prec == P3MAZE_MIXED;
    *kicked = false;
    CK(cudaStreamWaitEvent(s, ctx->ev_join, 0));
    stage_begin(ctx, P3MAZE_ST_GATHER);
    if (ctx->lr_force == P3MAZE_LR_FORCE_ANALYTIC) {
        if (mixed)
            k_gather_grad_mp<<<nblk(ctx->np), P3_THREADS, 0, s>>>(ctx->np, ctx->mp, ctx->order, ctx->N, ctx->inv_h,
                                                                  ctx->ke, ctx->phi32, ctx->Fs, ctx->F, ctx->Flr,
                                                                  ctx->Fsr);
        else
            k_gather_grad64<<<nblk(ctx->np), P3_THREADS, 0, s>>>(ctx->np, ctx->xq, ctx->order, ctx->N, ctx->inv_h,
                                                                 ctx->ke, ctx->phi[ctx->icur], ctx->Fs, ctx->F,
                                                                 ctx->Flr, ctx->Fsr);
    } else if (mixed) {
        *kicked = kick && ctx->nmol == 0;
        CK(launch_maybe_pdl(ctx->pdl, k_gather_mp, dim3(nblk(ctx->np)), dim3(P3_THREADS), 0, s, ctx->np, ctx->mp,
                            ctx->order, ctx->N, ctx->inv_h, ctx->ke, (const float*)ctx->phi32, (const double*)ctx->Fs,
                            ctx->F, ctx->Flr, ctx->Fsr, *kicked ? (const double*)ctx->hdt_acc : (const double*)nullptr,
                            *kicked ? ctx->v : (double*)nullptr));
    } else {
        CK(launch_maybe_pdl(ctx->pdl, k_gather<double>, dim3(nblk(ctx->np)), dim3(P3_THREADS), 0, s, ctx->np,
                            (const PQ*)ctx->xq, (const int*)ctx->order, ctx->N, ctx->inv_h, ctx->ke,
                            (const double*)ctx->phi[ctx->icur], (const double*)ctx->Fs, ctx->F, ctx->Flr, ctx->Fsr));
    }
    count(ctx, P3MAZE_ST_GATHER);
    if (ctx->nmol) {
        k_water<<<nblk(ctx->nmol), P3_THREADS, 0, s>>>(ctx->nmol, ctx->tri, ctx->r, ctx->Q, ctx->L, ctx->alpha, ctx->ke,
                                                      ctx->kb, ctx->r0, ctx->ka, ctx->th0, ctx->F, ctx->Fb, ctx->eb,
                                                      ctx->ex);
        count(ctx, P3MAZE_ST_GATHER);
    }
    CKL();
    return P3MAZE_OK;
}

// Assignment and smoothing use the whole GPU; the pair branch is forked
// after them so that it fills the SMs the latency-bound solve leaves idle.
template <typename T>
int mesh_pipeline(p3maze_ctx* ctx, int pred_order) {
    int rc = 0;
    if (ctx->pair_fork == 1 && (rc = pair_forces(ctx))) return rc;
    if ((rc = spread_smooth<T>(ctx))) return rc;
    if (ctx->pair_fork == 0 && (rc = pair_forces(ctx))) return rc;
    return solve_field<T>(ctx, pred_order);
}

// Cell list, mesh pipeline and forces at the current positions.  The gather
// stage stays open: the caller closes it (after the final half kick, which
// the interpolation may have done: *kicked).
int field_and_forces(p3maze_ctx* ctx, int pred_order, bool counted, bool kick, bool* kicked) {
    int rc = build_cells(ctx, counted);
    if (rc) return rc;
    rc = ctx->prec == P3MAZE_MIXED ? mesh_pipeline<float>(ctx, pred_order)
                                   : mesh_pipeline<double>(ctx, pred_order);
    if (rc) return rc;
    return gather_forces(ctx, kick, kicked);
}

// Copy the solver state to the host and turn a recorded failure into an error.
int read_solver_state(p3maze_ctx* ctx) {
    CK(cudaMemcpyAsync(ctx->hmg, ctx->dmg, sizeof(MGState), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    const MGState& m = *ctx->hmg;
    ctx->st.last_iters = m.last_iters;
    ctx->st.last_residual = m.last_res * ctx->res_scale / ctx->res_unit;
    ctx->st.total_iters = m.total_iters;
    // V-cycles run inside graphs: add their body launches to the tally
    const int64_t graph_iters = m.total_iters - ctx->eager_iters;
    if (graph_iters > ctx->graph_iters_seen) {
        ctx->launches[P3MAZE_ST_SOLVE] += (graph_iters - ctx->graph_iters_seen) * ctx->body_launches;
        ctx->graph_iters_seen = graph_iters;
    }
    if (m.status == P3MAZE_ERR_INVALID)
        return fail(ctx, P3MAZE_ERR_INVALID, "non-finite position or velocity copied in from the host");
    if (m.status == P3MAZE_ERR_NONFINITE) return fail(ctx, P3MAZE_ERR_NONFINITE, "non-finite constraint residual");
    if (m.status == P3MAZE_ERR_NOT_CONVERGED) {
        char buf[160];
        std::snprintf(buf, sizeof buf, "multigrid did not reach tol %.3g in %d V-cycles (residual %.3g)", ctx->tol,
                      ctx->itmax, m.last_res * ctx->res_scale / ctx->res_unit);
        return fail(ctx, P3MAZE_ERR_NOT_CONVERGED, buf);
    }
    return P3MAZE_OK;
}

// Full solve from phi = 0 at the current positions (phi^{-1} = phi^0, empty
// multiplier history) and the forces there.
int initialise_field(p3maze_ctx* ctx) {
    cudaStream_t s = ctx->stream;
    const size_t mb = sizeof(double) * ctx->P;
    for (int k = 0; k < 2; ++k) {
        CK(cudaMemsetAsync(ctx->phi[k], 0, mb, s));
        CK(cudaMemsetAsync(ctx->psi[k], 0, mb, s));
    }
    for (int k = 0; k < 4; ++k) CK(cudaMemsetAsync(ctx->yh[k], 0, mb + 8, s));  // with the sum slot
    CK(cudaMemsetAsync(ctx->dmg, 0, sizeof(MGState), s));
    ctx->nhist = 0;
    const bool was_timing = ctx->timing;
    ctx->timing = false;
    bool kicked = false;
    int rc = field_and_forces(ctx, 0, false, false, &kicked);
    ctx->timing = was_timing;
    if (rc) return rc;
    rc = read_solver_state(ctx);
    ctx->st.init_iters = ctx->hmg->last_iters;
    if (rc) return rc;
    CK(cudaMemcpyAsync(ctx->phi[1 - ctx->icur], ctx->phi[ctx->icur], mb, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(ctx->psi[1 - ctx->icur], ctx->psi[ctx->icur], mb, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemsetAsync(ctx->yh[0], 0, mb + 8, s));
    // the initial solve is not part of the step statistics
    CK(cudaMemsetAsync(ctx->dmg, 0, sizeof(MGState), s));
    CK(cudaStreamSynchronize(s));
    ctx->eager_iters = 0;
    ctx->graph_iters_seen = 0;
    ctx->st.total_iters = 0;
    return P3MAZE_OK;
}

// Half kick and drift.  On the multi-kernel cell-list path the same launch
// also forms each particle's cell and the per-cell counts (*counted: the
// cell-list build then skips its count kernel).
int kick_drift(p3maze_ctx* ctx, bool* counted) {
    cudaStream_t s = ctx->stream;
    stage_begin(ctx, P3MAZE_ST_INTEGRATE);
    *counted = !cells_in_one_block(ctx->np, ctx->ncell);
    if (*counted)
        CK(launch_maybe_pdl(ctx->pdl, k_kick_drift_count, dim3(nblk(ctx->np)), dim3(P3_THREADS), 0, s, ctx->np,
                            ctx->r, ctx->v, (const double*)ctx->F, (const double*)ctx->hdt_acc, ctx->dt, ctx->L,
                            ctx->inv_cell, ctx->nc, ctx->cell, ctx->count));
    else
        k_kick_drift<<<nblk(ctx->np), P3_THREADS, 0, s>>>(ctx->np, ctx->r, ctx->v, ctx->F, ctx->hdt_acc, ctx->dt,
                                                          ctx->L);
    count(ctx, P3MAZE_ST_INTEGRATE);
    stage_end(ctx, P3MAZE_ST_INTEGRATE);
    CKL();
    return P3MAZE_OK;
}

// The launches of one MD step (eager, or recorded into a graph): kick/drift,
// field and forces, closing kick.
int step_body(p3maze_ctx* ctx, int order) {
    cudaStream_t s = ctx->stream;
    bool counted = false;
    int rc = kick_drift(ctx, &counted);
    if (rc) return rc;
    bool kicked = false;
    rc = field_and_forces(ctx, order, counted, true, &kicked);
    if (rc) return rc;
    if (!kicked) {
        CK(launch_maybe_pdl(ctx->pdl, k_kick, dim3(nblk(ctx->np)), dim3(P3_THREADS), 0, s, ctx->np, ctx->v,
                            (const double*)ctx->F, (const double*)ctx->hdt_acc));
        count(ctx, P3MAZE_ST_GATHER);
    }
    stage_end(ctx, P3MAZE_ST_GATHER);
    CKL();
    // the converged correction becomes y^{k+1}; the oldest history buffer is reused
    double* oldest = ctx->yh[3];
    ctx->yh[3] = ctx->yh[2];
    ctx->yh[2] = ctx->yh[1];
    ctx->yh[1] = ctx->yh[0];
    ctx->yh[0] = oldest;
    return P3MAZE_OK;
}

// A mixed-precision step split at the smoothing, for batches whose members'
// smoothing runs as one cluster launch over all of them: the head is the
// kick/drift, the cell list and the assignment (no pointer-phase dependence);
// the tail forks the short-range branch and runs the solve, interpolation,
// kick and pointer rotation.  head + cluster smoothing + tail = step_body.
int step_head(p3maze_ctx* ctx) {
    bool counted = false;
    int rc = kick_drift(ctx, &counted);
    if (rc) return rc;
    rc = build_cells(ctx, counted);
    return rc ? rc : spread_assign<float>(ctx);
}

int step_tail(p3maze_ctx* ctx, int order) {
    int rc = pair_forces(ctx);
    if (!rc) rc = solve_field<float>(ctx, order);
    bool kicked = false;
    if (!rc) rc = gather_forces(ctx, true, &kicked);
    if (rc) return rc;
    cudaStream_t s = ctx->stream;
    if (!kicked) {
        CK(launch_maybe_pdl(ctx->pdl, k_kick, dim3(nblk(ctx->np)), dim3(P3_THREADS), 0, s, ctx->np, ctx->v,
                            (const double*)ctx->F, (const double*)ctx->hdt_acc));
        count(ctx, P3MAZE_ST_GATHER);
    }
    stage_end(ctx, P3MAZE_ST_GATHER);
    CKL();
    double* oldest = ctx->yh[3];
    ctx->yh[3] = ctx->yh[2];
    ctx->yh[2] = ctx->yh[1];
    ctx->yh[1] = ctx->yh[0];
    ctx->yh[0] = oldest;
    return P3MAZE_OK;
}

void destroy_graphs(p3maze_ctx* ctx) {
    for (StepGraph& G : ctx->graphs) {
        if (G.x) cudaGraphExecDestroy(G.x);
        if (G.g) cudaGraphDestroy(G.g);
        G = StepGraph();
    }
}

// Record one steady-state step (full predictor history) for the current
// pointer phase.  The pointer state is restored afterwards.
int capture_graph(p3maze_ctx* ctx, StepGraph& G, int part) {
    cudaStream_t s = ctx->stream;
    int64_t saved[P3MAZE_NSTAGES];
    bool saved_pending[P3MAZE_NSTAGES];
    for (int st = 0; st < P3MAZE_NSTAGES; ++st) {
        saved[st] = ctx->launches[st];
        saved_pending[st] = ctx->pending[st];
        ctx->launches[st] = 0;
        ctx->pending[st] = false;
    }
    const int icur = ctx->icur;
    double* yh[4];
    std::memcpy(yh, ctx->yh, sizeof yh);
    CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    ctx->capturing = true;
    int rc = part == PART_HEAD ? step_head(ctx) : part == PART_TAIL ? step_tail(ctx, ctx->pred) : step_body(ctx, ctx->pred);
    ctx->capturing = false;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(s, &g);
    ctx->icur = icur;
    std::memcpy(ctx->yh, yh, sizeof yh);
    for (int st = 0; st < P3MAZE_NSTAGES; ++st) {
        G.launches[st] = ctx->launches[st];
        G.timed[st] = ctx->pending[st];
        ctx->launches[st] = saved[st];
        ctx->pending[st] = saved_pending[st];
    }
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return fail(ctx, P3MAZE_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    }
    cudaError_t ie = cudaGraphInstantiate(&G.x, g, 0);
    if (ie != cudaSuccess) {
        cudaGraphDestroy(g);
        return fail(ctx, P3MAZE_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ie));
    }
    G.g = g;
    G.icur = icur;
    G.part = part;
    std::memcpy(G.yh, yh, sizeof yh);
    G.valid = true;
    return P3MAZE_OK;
}

// Replay (recording it first if needed) the graph of a whole step or of a
// step's head or tail for the current pointer phase (the head has none).
int step_graph(p3maze_ctx* ctx, int part = PART_ALL) {
    StepGraph* G = nullptr;
    for (StepGraph& sg : ctx->graphs)
        if (sg.valid && sg.part == part &&
            (part == PART_HEAD || (sg.icur == ctx->icur && std::memcmp(sg.yh, ctx->yh, sizeof sg.yh) == 0)))
            G = &sg;
    if (!G) {
        for (StepGraph& sg : ctx->graphs)
            if (!sg.valid) {
                G = &sg;
                break;
            }
        if (!G) {
            destroy_graphs(ctx);
            G = &ctx->graphs[0];
        }
        int rc = capture_graph(ctx, *G, part);
        if (rc) return rc;
    }
    CK(cudaGraphLaunch(G->x, ctx->stream));
    for (int st = 0; st < P3MAZE_NSTAGES; ++st) {
        ctx->launches[st] += G->launches[st];
        if (G->timed[st]) ctx->pending[st] = true;
    }
    if (part == PART_HEAD) return P3MAZE_OK;
    // pointer rotation identical to step_body
    ctx->icur = 1 - ctx->icur;
    double* oldest = ctx->yh[3];
    ctx->yh[3] = ctx->yh[2];
    ctx->yh[2] = ctx->yh[1];
    ctx->yh[1] = ctx->yh[0];
    ctx->yh[0] = oldest;
    return P3MAZE_OK;
}

int step_once(p3maze_ctx* ctx) {
    int rc;
    if (ctx->use_graphs && ctx->nhist >= ctx->pred) {
        rc = step_graph(ctx);
    } else {
        rc = step_body(ctx, std::min(ctx->pred, ctx->nhist));
    }
    if (rc) return rc;
    ctx->nhist = std::min(ctx->nhist + 1, 3);
    ctx->st.steps += 1;
    return collect_timing(ctx);
}

// Levels N, N/2, ... halved while even and larger than kLevelMin; the
// deepest must be small enough for the exact coarse solve (<= kCoarseMax).
int validate_mesh(int N, int* nlev, int* ncoarse) {
    if (N < 4) return 0;
    int n = N, l = 1;
    while (n > kLevelMin && (n % 2) == 0) {
        n /= 2;
        ++l;
    }
    if (n > kCoarseMax) return 0;
    *nlev = l;
    *ncoarse = n;
    return 1;
}

// Coarse level for a limit cmax: the first level with n <= cmax, else the deepest.
int coarse_level(const p3maze_ctx* ctx, int cmax) {
    for (int l = 0; l < ctx->nlev; ++l)
        if (ctx->lev[l].n <= cmax) return l;
    return ctx->nlev - 1;
}

void set_coarse(p3maze_ctx* ctx, int cmax) {
    ctx->cmax = cmax;
    ctx->lc = coarse_level(ctx, cmax);
    ctx->st.mg_levels = ctx->lc + 1;
    ctx->st.coarse_n = ctx->lev[ctx->lc].n;
}

// Hartley table H[k][x] = cos(2 pi k x / n) + sin(2 pi k x / n) and the
// pseudo-inverse eigenvalues D[kz][ky][kx] = 1 / (Lambda n^3) (0 at k = 0),
// Lambda = -4 sum_axes sin^2(pi k_axis / n), in FP64 on the host.
void hartley_tables(int n, std::vector<double>& H, std::vector<double>& D) {
    H.assign((size_t)n * n, 0.0);
    D.assign((size_t)n * n * n, 0.0);
    for (int k = 0; k < n; ++k)
        for (int x = 0; x < n; ++x) {
            const double a = 2.0 * kPi * (double)((int64_t)k * x % n) / n;
            H[(size_t)k * n + x] = std::cos(a) + std::sin(a);
        }
    std::vector<double> s2(n);
    for (int k = 0; k < n; ++k) {
        const double sk = std::sin(kPi * k / n);
        s2[k] = sk * sk;
    }
    const double n3 = (double)n * n * n;
    for (int kz = 0; kz < n; ++kz)
        for (int ky = 0; ky < n; ++ky)
            for (int kx = 0; kx < n; ++kx) {
                if (!kx && !ky && !kz) continue;
                D[((size_t)kz * n + ky) * n + kx] = 1.0 / (-4.0 * (s2[kx] + s2[ky] + s2[kz]) * n3);
            }
}

void release(p3maze_ctx* ctx) {
    destroy_graphs(ctx);
    if (ctx->snap) cudaFree(ctx->snap);
    ctx->snap = nullptr;
    for (int st = 0; st < P3MAZE_NSTAGES; ++st)
        for (int k = 0; k < 2; ++k)
            if (ctx->ev[st][k]) cudaEventDestroy(ctx->ev[st][k]);
    for (void* p : ctx->allocs) cudaFree(p);
    ctx->allocs.clear();
    if (ctx->hscal) cudaFreeHost(ctx->hscal);
    if (ctx->hmg) cudaFreeHost(ctx->hmg);
    ctx->hscal = nullptr;
    ctx->hmg = nullptr;
    if (ctx->body_stream) cudaStreamDestroy(ctx->body_stream);
    if (ctx->pair_stream) cudaStreamDestroy(ctx->pair_stream);
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
    if (ctx->ev_drift) cudaEventDestroy(ctx->ev_drift);
    if (ctx->ev_copied) cudaEventDestroy(ctx->ev_copied);
    if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
    ctx->pair_stream = nullptr;
    ctx->copy_stream = nullptr;
    ctx->ev_fork = ctx->ev_join = ctx->ev_drift = ctx->ev_copied = nullptr;
    if (ctx->stream) cudaStreamDestroy(ctx->stream);
    if (ctx->ev_in) cudaEventDestroy(ctx->ev_in);
    if (ctx->ev_out) cudaEventDestroy(ctx->ev_out);
    ctx->ev_in = ctx->ev_out = nullptr;
    ctx->body_stream = nullptr;
    ctx->stream = nullptr;
}

// pos/vel: host arrays to copy in; or d_pos/d_vel: caller-owned device
// arrays the context borrows as its r and v (never freed by it).
int setup(p3maze_ctx* ctx, const p3maze_params* p, const double* pos, const double* vel, double* d_pos,
          double* d_vel) {
    const int n = p->n_particles;
    const bool mixed = p->precision == P3MAZE_MIXED;
    const size_t tb = mixed ? sizeof(float) : sizeof(double);
    CK(cudaGetDevice(&ctx->device));
    CK(cudaDeviceGetAttribute(&ctx->nsm, cudaDevAttrMultiProcessorCount, ctx->device));
    if (const char* v = std::getenv("P3MAZE_PDL")) ctx->pdl = std::strcmp(v, "0") != 0;
    {
        // Work runs on an internal stream of the highest priority (graphs can
        // be captured on it whatever the caller passed), the short-range
        // branch on one of the lowest so its blocks fill SMs that the
        // latency-bound multigrid leaves idle.  Each call is fenced against
        // the caller's stream with events on entry and exit.
        int least = 0, greatest = 0;
        CK(cudaDeviceGetStreamPriorityRange(&least, &greatest));
        CK(cudaStreamCreateWithPriority(&ctx->stream, cudaStreamNonBlocking, greatest));
        CK(cudaStreamCreateWithPriority(&ctx->pair_stream, cudaStreamNonBlocking, least));
        CK(cudaEventCreateWithFlags(&ctx->ev_in, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&ctx->ev_out, cudaEventDisableTiming));
    }
    CK(cudaStreamCreateWithFlags(&ctx->body_stream, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&ctx->ev_drift, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&ctx->ev_copied, cudaEventDisableTiming));
    CK(cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
    // particle arrays
    if (d_pos) {
        ctx->r = d_pos;
        ctx->v = d_vel;
    } else {
        ALLOC(ctx->r, 24 * (size_t)n);
        ALLOC(ctx->v, 24 * (size_t)n);
    }
    ALLOC(ctx->F, 24 * (size_t)n);
    ALLOC(ctx->Fsr, 24 * (size_t)n);
    ALLOC(ctx->Flr, 24 * (size_t)n);
    ALLOC(ctx->Fb, 24 * (size_t)n);
    ALLOC(ctx->hdt_acc, 8 * (size_t)n);
    ALLOC(ctx->mass, 8 * (size_t)n);
    ALLOC(ctx->Q, 8 * (size_t)n);
    ALLOC(ctx->cell, 4 * (size_t)n);
    ALLOC(ctx->order, 4 * (size_t)n);
    ALLOC(ctx->ts, 4 * (size_t)n);
    ALLOC(ctx->ms, 4 * (size_t)n);
    ALLOC(ctx->cs, 4 * (size_t)n);
    ALLOC(ctx->xq, sizeof(PQ) * (size_t)n);
    ALLOC(ctx->xl64, sizeof(PQ) * (size_t)n);
    ALLOC(ctx->xl32, sizeof(float4) * (size_t)n);
    if (mixed) ALLOC(ctx->mp, sizeof(MeshPt) * (size_t)n);
    ALLOC(ctx->Fs, 24 * (size_t)n);
    ALLOC(ctx->ecs, 8 * (size_t)n);
    ALLOC(ctx->evs, 8 * (size_t)n);
    ALLOC(ctx->wsr, 8 * (size_t)n);
    ALLOC(ctx->count, 4 * (size_t)ctx->ncell);
    // zero before the first build (on the context's stream: the legacy default
    // stream of a plain cudaMemset is not ordered with it); k_cell_sort keeps
    // it zero between builds
    CK(cudaMemsetAsync(ctx->count, 0, 4 * (size_t)ctx->ncell, ctx->stream));
    ALLOC(ctx->fill, 4 * (size_t)ctx->ncell);
    ALLOC(ctx->start, 4 * ((size_t)ctx->ncell + 1));
    if (p->types) ALLOC(ctx->type, 4 * (size_t)n);
    // mesh arrays
    const int64_t P = ctx->P;
    ALLOC(ctx->q, tb * P);
    ALLOC(ctx->qs, tb * P);
    for (int k = 0; k < 2; ++k) {
        ALLOC(ctx->phi[k], 8 * P);
        ALLOC(ctx->psi[k], 8 * P);
    }
    ALLOC(ctx->rfin, 8 * P);
    if (mixed) ALLOC(ctx->phi32, 4 * P);
    for (int k = 0; k < 4; ++k) ALLOC(ctx->yh[k], 8 * (P + 1));  // + the buffer's sum (gauge mode)
    if (!mixed) ALLOC(ctx->sig, 8 * P);  // mixed: the prediction is folded into the first residual
    ctx->lev.resize(ctx->nlev);
    int nn = ctx->N;
    for (int l = 0; l < ctx->nlev; ++l) {
        Level& L = ctx->lev[l];
        L.n = nn;
        L.pts = (int64_t)nn * nn * nn;
        ALLOC(L.e, tb * L.pts);
        ALLOC(L.b, tb * L.pts);
        if (l == 0) ALLOC(L.r, tb * L.pts);  // smoothing ping-pong buffer
        if (mixed && nn % 4 == 0) {
            if (l == 0) L.e2 = L.r;
            else if (l + 1 < ctx->nlev) ALLOC(L.e2, tb * L.pts);  // the deepest level never sweeps
        }
        if (nn <= kCoarseMax) {
            ALLOC(L.H, tb * (size_t)nn * nn);
            ALLOC(L.D, tb * L.pts);
            ALLOC(L.t, tb * L.pts);
        }
        nn /= 2;
    }
    {
        // The shared-memory limit is an attribute of the kernel, shared by
        // every context in the process: only ever raise it.
        size_t sm = 0;
        for (const Level& L : ctx->lev)
            if (L.H) sm = std::max(sm, coarse_smem_bytes(L.n, tb));
        cudaError_t ea = cudaSuccess;
        auto raise = [&](const void* fn) {
            cudaFuncAttributes fa{};
            cudaError_t e = cudaFuncGetAttributes(&fa, fn);
            if (e == cudaSuccess && (size_t)fa.maxDynamicSharedSizeBytes < sm)
                e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            if (e != cudaSuccess) ea = e;
        };
        if (mixed) {
            raise((const void*)k_coarse_xy<float>);
            raise((const void*)k_coarse_z<float>);
        } else {
            raise((const void*)k_coarse_xy<double>);
            raise((const void*)k_coarse_z<double>);
        }
        if (mixed) {
            sm = spread_smem_bytes<float>();
            raise((const void*)k_spread_tile<float, MeshPt, true>);
            raise((const void*)k_spread_tile<float, MeshPt, false>);
            sm = tq_smem_bytes<1>();
            raise((const void*)k_diffuse_tq<1, true>);
            raise((const void*)k_diffuse_tq<1, false>);
            sm = tq_smem_bytes<2>();
            raise((const void*)k_diffuse_tq<2, true>);
            raise((const void*)k_diffuse_tq<2, false>);
            sm = tq_smem_bytes<3>();
            raise((const void*)k_diffuse_tq<3, true>);
            raise((const void*)k_diffuse_tq<3, false>);
            sm = tq_smem_bytes<4>();
            raise((const void*)k_diffuse_tq<4, true>);
            raise((const void*)k_diffuse_tq<4, false>);
        } else {
            sm = spread_smem_bytes<double>();
            raise((const void*)k_spread_tile<double, PQ, false>);
        }
        if (cells_in_one_block(ctx->np, ctx->ncell)) {
            sm = cells_block_smem(ctx->ncell);
            raise((const void*)k_cells_block);
        }
        if (ea != cudaSuccess)
            return fail(ctx, P3MAZE_ERR_CUDA, std::string("shared memory limits: ") + cudaGetErrorString(ea));
    }
    ALLOC(ctx->partial, 8 * (size_t)partial_slots(ctx->N));
    ALLOC(ctx->dscal, 8 * S_NSCAL);
    if (mixed && ctx->K > 0 && cluster_mesh_ok(ctx->N)) {
        // smoothing of the whole mesh in one cluster launch (mode 5) when the
        // device co-schedules the clusters; the table entry exists either way
        ALLOC(ctx->cltab, sizeof(ClusterMesh));
        const ClusterMesh cm{(const float*)ctx->q, (float*)ctx->qs, ctx->dscal + S_QSUM, ctx->N, ctx->K,
                             (float)ctx->c, 0};
        UPLOAD(ctx->cltab, &cm, sizeof cm);
        ctx->cluster_ok = cluster_smoothing_supported(cluster_size_for(ctx->N, 1, ctx->nsm));
        if (ctx->cluster_ok) ctx->fuse = 5;
    }
    {
        const dim3 gr = resid_grid(ctx->N);
        ALLOC(ctx->bmax, 8 * (size_t)gr.x * gr.y * gr.z);
    }
    ALLOC(ctx->dmg, sizeof(MGState));
    {
        cudaError_t e1 = cudaMallocHost((void**)&ctx->hscal, 8 * S_NSCAL);
        cudaError_t e2 = cudaMallocHost((void**)&ctx->hmg, sizeof(MGState));
        if (e1 != cudaSuccess || e2 != cudaSuccess) return fail(ctx, P3MAZE_ERR_OOM, "cudaMallocHost failed");
    }
    cudaStream_t s = ctx->stream;
    // host-side derived arrays
    std::vector<double> hacc(n);
    for (int i = 0; i < n; ++i) hacc[i] = 0.5 * ctx->dt * P3_ACCEL / p->masses[i];
    for (Level& L : ctx->lev) {
        if (!L.H) continue;
        std::vector<double> H, D;
        hartley_tables(L.n, H, D);
        if (mixed && fht_supported(L.n)) {
            // the FFT kernels: D bit-reversed in all three indices, 2^-6 for
            // their six doubled transforms
            const int n = L.n;
            const std::vector<int> pos = fht_positions(n);
            std::vector<float> Df(D.size());
            for (int kz = 0; kz < n; ++kz)
                for (int ky = 0; ky < n; ++ky)
                    for (int kx = 0; kx < n; ++kx)
                        Df[((size_t)pos[kz] * n + pos[ky]) * n + pos[kx]] =
                            (float)(D[((size_t)kz * n + ky) * n + kx] / 64.0);
            UPLOAD(L.D, Df.data(), 4 * Df.size());
            const std::vector<float2> tw = fht_twiddle_table(n);
            ALLOC(L.tw, sizeof(float2) * tw.size());
            UPLOAD(L.tw, tw.data(), sizeof(float2) * tw.size());
            CK(fht_raise_smem(n));
        } else if (mixed) {
            std::vector<float> Hf(H.begin(), H.end()), Df(D.begin(), D.end());
            UPLOAD(L.H, Hf.data(), 4 * Hf.size());
            UPLOAD(L.D, Df.data(), 4 * Df.size());
        } else {
            UPLOAD(L.H, H.data(), 8 * H.size());
            UPLOAD(L.D, D.data(), 8 * D.size());
        }
    }
    if (mixed && ctx->K > 0 && (ctx->lev[0].H || fht_supported(ctx->N))) {
        // the smoothing operator (I + cM)^K is diagonal in the Hartley basis:
        // eigenvalue (1 + c lambda_k)^K, lambda_k = -4 sum_axes sin^2(pi k_axis / N)
        const int N = ctx->N;
        std::vector<double> s2(N);
        for (int k = 0; k < N; ++k) {
            const double sk = std::sin(kPi * k / N);
            s2[k] = sk * sk;
        }
        std::vector<float> S((size_t)N * N * N);
        const double inv_n3 = 1.0 / ((double)N * N * N);
        // the FFT kernels form twice each Hartley transform (2^-6 for the six)
        // and keep the coefficients in bit-reversed order
        const bool fft = fht_supported(N);
        const double fht_scale = fft ? 1.0 / 64.0 : 1.0;
        std::vector<int> pos = fht_positions(N);
        if (!fft)
            for (int k = 0; k < N; ++k) pos[k] = k;
        for (int kz = 0; kz < N; ++kz)
            for (int ky = 0; ky < N; ++ky)
                for (int kx = 0; kx < N; ++kx) {
                    const double g = 1.0 - 4.0 * ctx->c * (s2[kx] + s2[ky] + s2[kz]);
                    S[((size_t)pos[kz] * N + pos[ky]) * N + pos[kx]] =
                        (float)(std::pow(g, ctx->K) * inv_n3 * fht_scale);
                }
        ALLOC(ctx->Ssm, 4 * S.size());
        UPLOAD(ctx->Ssm, S.data(), 4 * S.size());
        if (fft) {
            const std::vector<float2> tw = fht_twiddle_table(N);
            ALLOC(ctx->fht_tw, sizeof(float2) * tw.size());
            UPLOAD(ctx->fht_tw, tw.data(), sizeof(float2) * tw.size());
            CK(fht_raise_smem(N));
        }
        ctx->fuse = 6;  // the default for such meshes: fastest alone and in a batch graph
    }
    CK(cudaMemcpyAsync(ctx->hdt_acc, hacc.data(), 8 * (size_t)n, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ctx->mass, p->masses, 8 * (size_t)n, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ctx->Q, p->charges, 8 * (size_t)n, cudaMemcpyHostToDevice, s));
    if (p->types) CK(cudaMemcpyAsync(ctx->type, p->types, 4 * (size_t)n, cudaMemcpyHostToDevice, s));
    if (!d_pos) {
        CK(cudaMemcpyAsync(ctx->r, pos, 24 * (size_t)n, cudaMemcpyHostToDevice, s));
        if (vel) CK(cudaMemcpyAsync(ctx->v, vel, 24 * (size_t)n, cudaMemcpyHostToDevice, s));
        else CK(cudaMemsetAsync(ctx->v, 0, 24 * (size_t)n, s));
    }
    CK(cudaMemsetAsync(ctx->Fb, 0, 24 * (size_t)n, s));
    CK(cudaMemsetAsync(ctx->dscal, 0, 8 * S_NSCAL, s));
    if (ctx->nmol) {
        const p3maze_topology* tp = p->topology;
        std::vector<int> mol(n, -1);
        for (int m = 0; m < ctx->nmol; ++m)
            for (int a = 0; a < 3; ++a) mol[tp->triples[3 * m + a]] = m;
        ALLOC(ctx->mol, 4 * (size_t)n);
        ALLOC(ctx->tri, 12 * (size_t)ctx->nmol);
        ALLOC(ctx->eb, 8 * (size_t)ctx->nmol);
        ALLOC(ctx->ex, 8 * (size_t)ctx->nmol);
        CK(cudaMemcpyAsync(ctx->mol, mol.data(), 4 * (size_t)n, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(ctx->tri, tp->triples, 12 * (size_t)ctx->nmol, cudaMemcpyHostToDevice, s));
        CK(cudaStreamSynchronize(s));  // host vectors go out of scope
    }
    // wrap positions into the box; borrowed arrays are checked for NaN/Inf here
    CK(cudaMemsetAsync(ctx->dmg, 0, sizeof(MGState), s));
    k_wrap_check<<<nblk(3 * (int64_t)n), P3_THREADS, 0, s>>>(n, ctx->r, ctx->v, ctx->L, &ctx->dmg->status,
                                                             P3MAZE_ERR_INVALID);
    CKL();
    CK(cudaMemcpyAsync(ctx->hmg, ctx->dmg, sizeof(MGState), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (ctx->hmg->status) return fail(ctx, P3MAZE_ERR_INVALID, "non-finite position or velocity");
    return P3MAZE_OK;
}

int sync_scalars(p3maze_ctx* ctx) {
    CK(cudaMemcpyAsync(ctx->hscal, ctx->dscal, 8 * S_NSCAL, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return P3MAZE_OK;
}

}  // namespace

// Device bytes p3maze_init allocates for these parameters: the same list of
// arrays as setup() (requested sizes, before the allocator's rounding).
size_t planned_bytes(const p3maze_params* p, int nlev) {
    auto a = [](size_t b) { return b ? b : (size_t)16; };
    const size_t n = (size_t)p->n_particles;
    const bool mixed = p->precision == P3MAZE_MIXED;
    const size_t tb = mixed ? 4 : 8;
    const int N = p->mesh;
    const size_t P = (size_t)N * N * N;
    const int nc = std::max(1, (int)std::floor(p->box[0] / (0.5 * p->r_cut)));
    const size_t ncell = (size_t)nc * nc * nc;
    size_t b = 0;
    for (int k = 0; k < 6; ++k) b += a(24 * n);          // r v F Fsr Flr Fb
    for (int k = 0; k < 3; ++k) b += a(8 * n);           // hdt_acc mass Q
    for (int k = 0; k < 5; ++k) b += a(4 * n);           // cell order ts ms cs
    b += a(32 * n) + a(32 * n) + a(16 * n);              // xq xl64 xl32
    if (mixed) b += a(sizeof(MeshPt) * n);               // mp
    b += a(24 * n) + a(8 * n) + a(8 * n) + a(8 * n);     // Fs ecs evs wsr
    b += a(4 * ncell) + a(4 * ncell) + a(4 * (ncell + 1));
    if (p->types) b += a(4 * n);
    b += a(tb * P) + a(tb * P);                          // q qs
    for (int k = 0; k < 4; ++k) b += a(8 * P);           // phi, psi
    b += a(8 * P);                                       // rfin
    if (mixed) b += a(4 * P);                            // phi32
    for (int k = 0; k < 4; ++k) b += a(8 * (P + 1));     // y ring, each with its sum
    if (!mixed) b += a(8 * P);                           // sigma
    int nn = N;
    for (int l = 0; l < nlev; ++l) {
        const size_t pts = (size_t)nn * nn * nn;
        b += a(tb * pts) + a(tb * pts);
        if (l == 0) b += a(tb * pts);
        if (mixed && nn % 4 == 0 && l > 0 && l + 1 < nlev) b += a(tb * pts);  // e2
        if (nn <= kCoarseMax) b += a(tb * (size_t)nn * nn) + a(tb * pts) + a(tb * pts);  // H D t
        if (mixed && nn <= kCoarseMax && fht_supported(nn)) b += a(sizeof(float2) * (size_t)(nn / 2));  // tw
        nn /= 2;
    }
    b += a(8 * (size_t)partial_slots(N));
    b += a(8 * S_NSCAL);
    if (mixed && p->method != P3MAZE_METHOD_PMAZE && cluster_mesh_ok(N)) b += a(sizeof(ClusterMesh));
    if (mixed && p->method != P3MAZE_METHOD_PMAZE && (N <= kCoarseMax || fht_supported(N))) {
        b += a(4 * P);  // spectral smoothing table
        if (fht_supported(N)) b += a(sizeof(float2) * fht_twiddle_count(N));  // its FFT twiddles
    }
    {
        const dim3 gr = resid_grid(N);
        b += a(8 * (size_t)gr.x * gr.y * gr.z);
    }
    b += a(sizeof(MGState));
    if (p->topology && p->topology->n_molecules > 0) {
        const size_t m = (size_t)p->topology->n_molecules;
        b += a(4 * n) + a(12 * m) + a(8 * m) + a(8 * m);
    }
    return b;
}

// =============================================================== C ABI
extern "C" {

namespace {
int init_impl(const p3maze_params* p, const double* pos, const double* vel, double* d_pos, double* d_vel,
              void* cuda_stream, p3maze_ctx** out) {
    if (!out) return fail(nullptr, P3MAZE_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (!p || !(pos || (d_pos && d_vel))) return fail(nullptr, P3MAZE_ERR_INVALID, "params or positions NULL");
    const int n = p->n_particles;
    if (n < 1) return fail(nullptr, P3MAZE_ERR_INVALID, "n_particles must be >= 1");
    if (!p->charges || !p->masses) return fail(nullptr, P3MAZE_ERR_INVALID, "charges and masses are required");
    const double L = p->box[0];
    if (!(L > 0.0) || std::fabs(p->box[1] - L) > 1e-12 * L || std::fabs(p->box[2] - L) > 1e-12 * L)
        return fail(nullptr, P3MAZE_ERR_INVALID, "box must be cubic and positive");
    const bool pmaze = p->method == P3MAZE_METHOD_PMAZE;
    if (!pmaze && !(p->alpha > 0.0)) return fail(nullptr, P3MAZE_ERR_INVALID, "alpha must be > 0");
    if (pmaze && !(p->alpha >= 0.0)) return fail(nullptr, P3MAZE_ERR_INVALID, "alpha must be >= 0");
    if (!(p->r_cut > 0.0) || p->r_cut > L) return fail(nullptr, P3MAZE_ERR_INVALID, "need 0 < r_cut <= L");
    if (p->order != 4) return fail(nullptr, P3MAZE_ERR_INVALID, "only order 4 (cubic B-spline) is supported");
    if (!(p->tol > 0.0)) return fail(nullptr, P3MAZE_ERR_INVALID, "tol must be > 0");
    if (!(p->dt >= 0.0)) return fail(nullptr, P3MAZE_ERR_INVALID, "dt must be >= 0");
    if (p->predictor < 0 || p->predictor > 3) return fail(nullptr, P3MAZE_ERR_INVALID, "predictor must be 0..3");
    if (p->method != P3MAZE_METHOD_MAZE && p->method != P3MAZE_METHOD_P3M && !pmaze)
        return fail(nullptr, P3MAZE_ERR_INVALID,
                    "method must be P3MAZE_METHOD_MAZE, P3MAZE_METHOD_P3M or P3MAZE_METHOD_PMAZE");
    if (p->precision != P3MAZE_FP64 && p->precision != P3MAZE_MIXED)
        return fail(nullptr, P3MAZE_ERR_INVALID, "precision must be P3MAZE_FP64 or P3MAZE_MIXED");
    if (p->max_mg_iters < 0 || p->pre_sweeps < 0 || p->post_sweeps < 0)
        return fail(nullptr, P3MAZE_ERR_INVALID, "iteration counts must be >= 0");
    int nlev = 0, ncoarse = 0;
    if (!validate_mesh(p->mesh, &nlev, &ncoarse))
        return fail(nullptr, P3MAZE_ERR_INVALID, "mesh must be N >= 4 with N = m 2^l, m <= 64 (halving stops at 16)");
    if (p->coarse_max < 0) return fail(nullptr, P3MAZE_ERR_INVALID, "coarse_max must be >= 0");
    if (p->lr_force != P3MAZE_LR_FORCE_FD && p->lr_force != P3MAZE_LR_FORCE_ANALYTIC)
        return fail(nullptr, P3MAZE_ERR_INVALID, "lr_force must be P3MAZE_LR_FORCE_FD or P3MAZE_LR_FORCE_ANALYTIC");
    if (p->sr_shift != P3MAZE_SR_TRUNCATE && p->sr_shift != P3MAZE_SR_SHIFT_FORCE)
        return fail(nullptr, P3MAZE_ERR_INVALID, "sr_shift must be P3MAZE_SR_TRUNCATE or P3MAZE_SR_SHIFT_FORCE");
    if (pmaze && p->lr_force != P3MAZE_LR_FORCE_FD)
        return fail(nullptr, P3MAZE_ERR_INVALID,
                    "P3MAZE_METHOD_PMAZE takes the finite-difference force (the exact gradient carries the grid "
                    "self-force)");
    double qsum = 0.0, qabs = 0.0;
    for (int i = 0; i < n; ++i) {
        if (!(p->masses[i] > 0.0)) return fail(nullptr, P3MAZE_ERR_INVALID, "masses must be > 0");
        if (!std::isfinite(p->charges[i])) return fail(nullptr, P3MAZE_ERR_INVALID, "non-finite charge");
        qsum += p->charges[i];
        qabs += std::fabs(p->charges[i]);
    }
    if (std::fabs(qsum) > 1e-9 * std::max(qabs, 1e-300))
        return fail(nullptr, P3MAZE_ERR_INVALID, "system is not neutral (|sum Q| > 1e-9 sum |Q|)");
    for (int i = 0; pos && i < 3 * n; ++i)
        if (!std::isfinite(pos[i]) || (vel && !std::isfinite(vel[i])))
            return fail(nullptr, P3MAZE_ERR_INVALID, "non-finite position or velocity");
    SRTable tab{};
    if (p->sr && p->sr->kind != P3MAZE_SR_NONE) {
        const p3maze_sr_table* t = p->sr;
        if (t->kind != P3MAZE_SR_BMH && t->kind != P3MAZE_SR_LJ)
            return fail(nullptr, P3MAZE_ERR_INVALID, "unknown short-range kind");
        if (t->n_types < 1 || t->n_types > P3MAZE_MAX_TYPES)
            return fail(nullptr, P3MAZE_ERR_INVALID, "n_types out of range");
        if (!p->types) return fail(nullptr, P3MAZE_ERR_INVALID, "types are required with a short-range table");
        for (int i = 0; i < n; ++i)
            if (p->types[i] < 0 || p->types[i] >= t->n_types)
                return fail(nullptr, P3MAZE_ERR_INVALID, "particle type out of range");
        tab.kind = t->kind;
        tab.nt = t->n_types;
        for (int a = 0; a < 5; ++a)
            for (int k = 0; k < t->n_types * t->n_types; ++k) tab.p[a][k] = t->p[a][k];
        if (t->kind == P3MAZE_SR_BMH)
            for (int k = 0; k < t->n_types * t->n_types; ++k)
                if (!(tab.p[1][k] > 0.0)) return fail(nullptr, P3MAZE_ERR_INVALID, "BMH rho must be > 0");
    } else {
        tab.kind = 0;
        tab.nt = 1;
    }
    {
        // shifted-force constants at r_cut (used only with P3MAZE_SR_SHIFT_FORCE)
        const double rc = p->r_cut;
        tab.rc = rc;
        if (!pmaze) {
            const double x = p->alpha * rc;
            tab.cg = std::erfc(x) / rc;
            tab.cG = std::erfc(x) / (rc * rc) + 2.0 / std::sqrt(kPi) * p->alpha * std::exp(-x * x) / rc;
        }
        for (int k = 0; k < tab.nt * tab.nt; ++k) {
            if (tab.kind == P3MAZE_SR_BMH) {
                const double A = tab.p[0][k], rho = tab.p[1][k], sg = tab.p[2][k], Cc = tab.p[3][k],
                             Dc = tab.p[4][k];
                const double ex = A * std::exp((sg - rc) / rho);
                tab.urc[k] = ex - Cc / std::pow(rc, 6) - Dc / std::pow(rc, 8);
                tab.frc[k] = ex / rho - 6.0 * Cc / std::pow(rc, 7) - 8.0 * Dc / std::pow(rc, 9);
            } else if (tab.kind == P3MAZE_SR_LJ) {
                const double eps = tab.p[0][k], s6 = std::pow(tab.p[1][k] / rc, 6);
                tab.urc[k] = 4.0 * eps * (s6 * s6 - s6);
                tab.frc[k] = 24.0 * eps * (2.0 * s6 * s6 - s6) / rc;
            }
        }
    }
    int nmol = 0;
    if (p->topology && p->topology->n_molecules > 0) {
        const p3maze_topology* tp = p->topology;
        if (!tp->triples) return fail(nullptr, P3MAZE_ERR_INVALID, "topology triples missing");
        std::vector<char> seen(n, 0);
        for (int m = 0; m < tp->n_molecules; ++m)
            for (int a = 0; a < 3; ++a) {
                const int id = tp->triples[3 * m + a];
                if (id < 0 || id >= n || seen[id])
                    return fail(nullptr, P3MAZE_ERR_INVALID, "topology triples must be disjoint valid indices");
                seen[id] = 1;
            }
        nmol = tp->n_molecules;
        if (pmaze)
            return fail(nullptr, P3MAZE_ERR_INVALID,
                        "P3MAZE_METHOD_PMAZE takes no molecular topology (exclusions need the mesh pair term)");
    }
    const double h = L / p->mesh;
    // PMaZe: no Gaussian screening, the assigned charge is the source (K = 0)
    const double sigma = pmaze ? 0.0 : 1.0 / (std::sqrt(2.0) * p->alpha);
    // diffusion smoothing: per-axis variance sigma^2 - 4 h^2/6 in K steps of 2 c h^2
    const double kappa = pmaze ? 0.0 : (sigma * sigma - 4.0 * h * h / 6.0) / (2.0 * h * h);
    if (!pmaze && !(kappa > 0.0))
        return fail(nullptr, P3MAZE_ERR_INVALID, "mesh too coarse for alpha: need sigma^2 > 2 h^2/3");

    p3maze_ctx* ctx = new (std::nothrow) p3maze_ctx();
    if (!ctx) return fail(nullptr, P3MAZE_ERR_OOM, "host allocation failed");
    ctx->user_stream = (cudaStream_t)cuda_stream;
    ctx->np = n;
    ctx->N = p->mesh;
    ctx->P = (int64_t)p->mesh * p->mesh * p->mesh;
    ctx->L = L;
    ctx->h = h;
    ctx->inv_h = p->mesh / L;
    ctx->alpha = p->alpha;
    ctx->sigma = sigma;
    ctx->rc = p->r_cut;
    ctx->K = pmaze ? 0 : (int)std::ceil(6.0 * kappa);
    ctx->c = pmaze ? 0.0 : kappa / ctx->K;
    ctx->tol = p->tol;
    ctx->dt = p->dt;
    ctx->method = p->method;
    ctx->lr_force = p->lr_force;
    ctx->sr_shift = p->sr_shift;
    // one diffusion step per launch; FP32 quads take 2 planes per thread
    ctx->zc = (p->precision == P3MAZE_MIXED && p->mesh % 4 == 0) ? 2 : 8;
    ctx->fuse = 1;
    ctx->res_scale = p->method == P3MAZE_METHOD_P3M ? 4.0 * kPi / h : 1.0;
    ctx->res_unit = p->precision == P3MAZE_MIXED ? 4.0 * kPi / h : 1.0;
    // P3M has no multiplier: every solve starts from the Verlet-predicted field
    ctx->pred = p->method == P3MAZE_METHOD_P3M ? 0 : (p->predictor == 0 ? 3 : p->predictor);
    ctx->prec = p->precision;
    ctx->itmax = p->max_mg_iters ? p->max_mg_iters : 50;
    ctx->nu1 = p->pre_sweeps ? p->pre_sweeps : 2;
    ctx->nu2 = p->post_sweeps ? p->post_sweeps : 2;
    ctx->ke = p->coulomb_k != 0.0 ? p->coulomb_k : P3_COULOMB_K;
    ctx->nc = std::max(1, (int)std::floor(L / (0.5 * p->r_cut)));
    ctx->ncell = ctx->nc * ctx->nc * ctx->nc;
    ctx->inv_cell = ctx->nc / L;
    ctx->lcell = L / ctx->nc;
    ctx->nlev = nlev;
    ctx->tab = tab;
    ctx->nmol = nmol;
    if (nmol) {
        ctx->kb = p->topology->kb;
        ctx->r0 = p->topology->r0;
        ctx->ka = p->topology->ka;
        ctx->th0 = p->topology->theta0;
    }
    double q2 = 0.0;
    for (int i = 0; i < n; ++i) q2 += p->charges[i] * p->charges[i];
    ctx->v_self = pmaze ? 0.0 : -ctx->ke * q2 / (std::sqrt(2.0 * kPi) * sigma);
    ctx->ke_pair = pmaze ? 0.0 : ctx->ke;  // PMaZe pairs: non-Coulomb term only
    ctx->st.smooth_steps = ctx->K;
    ctx->st.smooth_coeff = ctx->c;
    (void)ncoarse;
    ctx->st.cells_per_axis = ctx->nc;
    ctx->st.sigma = sigma;

    int rc = setup(ctx, p, pos, vel, d_pos, d_vel);
    if (!rc) set_coarse(ctx, p->coarse_max ? p->coarse_max : (p->precision == P3MAZE_MIXED ? 64 : 16));
    if (!rc) rc = initialise_field(ctx);
    if (!rc) rc = leave(ctx);
    if (!rc) {
        cudaError_t e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) rc = fail(ctx, P3MAZE_ERR_CUDA, std::string("init: ") + cudaGetErrorString(e));
    }
    if (rc) {
        g_init_error = ctx->err;
        release(ctx);
        delete ctx;
        return rc;
    }
    *out = ctx;
    return P3MAZE_OK;
}

struct StateHeader {
    char magic[8];
    int32_t version, np, mesh, precision, method, nmol;
    int64_t steps;
    int32_t nhist, pad;
    MGState mg;
};

void state_segments(p3maze_ctx* ctx, std::vector<std::pair<void*, size_t>>& seg) {
    const size_t n3 = 24 * (size_t)ctx->np, n1 = 8 * (size_t)ctx->np, P8 = 8 * (size_t)ctx->P;
    const size_t tb = ctx->prec == P3MAZE_MIXED ? 4 : 8;
    seg = {{ctx->r, n3},   {ctx->v, n3},   {ctx->F, n3},   {ctx->Fsr, n3}, {ctx->Flr, n3}, {ctx->Fb, n3},
           {ctx->ecs, n1}, {ctx->evs, n1}, {ctx->wsr, n1}, {ctx->q, tb * (size_t)ctx->P},
           {ctx->phi[ctx->icur], P8}, {ctx->phi[1 - ctx->icur], P8},
           {ctx->psi[ctx->icur], P8}, {ctx->psi[1 - ctx->icur], P8},
           {ctx->yh[1], P8 + 8}, {ctx->yh[2], P8 + 8}, {ctx->yh[3], P8 + 8},
           {ctx->rfin, P8}, {ctx->dscal, 8 * (size_t)S_NSCAL}};
    if (ctx->sig) seg.push_back({ctx->sig, P8});
    if (ctx->phi32) seg.push_back({ctx->phi32, 4 * (size_t)ctx->P});
    if (ctx->nmol) {
        seg.push_back({ctx->eb, 8 * (size_t)ctx->nmol});
        seg.push_back({ctx->ex, 8 * (size_t)ctx->nmol});
    }
}

size_t state_size(p3maze_ctx* ctx) {
    std::vector<std::pair<void*, size_t>> seg;
    state_segments(ctx, seg);
    size_t b = sizeof(StateHeader);
    for (auto& s : seg) b += s.second;
    return b;
}

// Device copy of the state (the checkpoint's segments and the solver state),
// queued on the work stream; taken once until the next wait.
int take_snapshot(p3maze_ctx* ctx) {
    if (!ctx->rollback || ctx->snap_taken || !ctx->snap) return P3MAZE_OK;
    std::vector<std::pair<void*, size_t>> seg;
    state_segments(ctx, seg);
    unsigned char* p = static_cast<unsigned char*>(ctx->snap);
    for (auto& s : seg) {
        CK(cudaMemcpyAsync(p, s.first, s.second, cudaMemcpyDeviceToDevice, ctx->stream));
        p += s.second;
    }
    CK(cudaMemcpyAsync(p, ctx->dmg, sizeof(MGState), cudaMemcpyDeviceToDevice, ctx->stream));
    ctx->snap_steps = ctx->st.steps;
    ctx->snap_nhist = ctx->nhist;
    ctx->snap_taken = true;
    return P3MAZE_OK;
}

// Put the snapshot back (the segments by their roles at the current pointer
// phase, as p3maze_load_state does) and wait for it.
int restore_snapshot(p3maze_ctx* ctx) {
    std::vector<std::pair<void*, size_t>> seg;
    state_segments(ctx, seg);
    const unsigned char* p = static_cast<const unsigned char*>(ctx->snap);
    for (auto& s : seg) {
        CK(cudaMemcpyAsync(s.first, p, s.second, cudaMemcpyDeviceToDevice, ctx->stream));
        p += s.second;
    }
    CK(cudaMemcpyAsync(ctx->hmg, p, sizeof(MGState), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    MGState mg = *ctx->hmg;
    mg.it = 0;
    mg.cont = 0;
    mg.arrive = 0;
    mg.arrive_sum = 0;
    *ctx->hmg = mg;
    CK(cudaMemcpyAsync(ctx->dmg, ctx->hmg, sizeof(MGState), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->st.steps = ctx->snap_steps;
    ctx->nhist = ctx->snap_nhist;
    ctx->st.total_iters = mg.total_iters;
    ctx->eager_iters = mg.total_iters;  // as after p3maze_load_state
    ctx->graph_iters_seen = 0;
    return P3MAZE_OK;
}

// The solver state of the queued steps; with rollback on, a failed call's
// steps are undone.
int finish_steps(p3maze_ctx* ctx) {
    const int rc = read_solver_state(ctx);
    const bool undo = rc && ctx->rollback && ctx->snap_taken &&
                      (rc == P3MAZE_ERR_NOT_CONVERGED || rc == P3MAZE_ERR_NONFINITE || rc == P3MAZE_ERR_INVALID);
    if (undo) {
        const std::string msg = ctx->err;
        const int rrc = restore_snapshot(ctx);
        if (rrc) return rrc;
        ctx->err = msg + " (state rolled back to before the failed steps)";
    }
    ctx->snap_taken = false;
    return rc;
}
}  // namespace

int p3maze_init(const p3maze_params* p, const double* pos, const double* vel, void* cuda_stream,
                p3maze_ctx** out) {
    if (!pos) return fail(nullptr, P3MAZE_ERR_INVALID, "pos is NULL");
    return init_impl(p, pos, vel, nullptr, nullptr, cuda_stream, out);
}

int p3maze_init_device(const p3maze_params* p, double* d_pos, double* d_vel, void* cuda_stream,
                       p3maze_ctx** out) {
    if (!d_pos || !d_vel) return fail(nullptr, P3MAZE_ERR_INVALID, "d_pos and d_vel are required");
    if (((uintptr_t)d_pos | (uintptr_t)d_vel) & 7)
        return fail(nullptr, P3MAZE_ERR_INVALID, "d_pos and d_vel must be 8-byte aligned");
    return init_impl(p, nullptr, nullptr, d_pos, d_vel, cuda_stream, out);
}

int p3maze_step_async(p3maze_ctx* ctx, int32_t nsteps) {
    if (!ctx) return fail(nullptr, P3MAZE_ERR_INVALID, "ctx is NULL");
    if (nsteps < 0) return fail(ctx, P3MAZE_ERR_INVALID, "nsteps must be >= 0");
    int rc = enter(ctx);
    if (rc) return rc;
    rc = take_snapshot(ctx);
    if (rc) return rc;
    for (int k = 0; k < nsteps; ++k) {
        rc = step_once(ctx);
        if (rc) return rc;
    }
    return leave(ctx);
}

int p3maze_wait(p3maze_ctx* ctx) {
    if (!ctx) return fail(nullptr, P3MAZE_ERR_INVALID, "ctx is NULL");
    return finish_steps(ctx);
}

int p3maze_step(p3maze_ctx* ctx, int32_t nsteps) {
    int rc = p3maze_step_async(ctx, nsteps);
    if (rc) return rc;
    return finish_steps(ctx);
}

int p3maze_set_rollback(p3maze_ctx* ctx, int32_t enable) {
    if (!ctx) return fail(nullptr, P3MAZE_ERR_INVALID, "ctx is NULL");
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->snap_taken = false;
    if (!enable) {
        if (ctx->snap) cudaFree(ctx->snap);
        ctx->snap = nullptr;
        ctx->snap_bytes = 0;
        ctx->rollback = false;
        return P3MAZE_OK;
    }
    if (!ctx->snap) {
        const size_t bytes = state_size(ctx) - sizeof(StateHeader) + sizeof(MGState);
        cudaError_t e = cudaMalloc(&ctx->snap, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            ctx->snap = nullptr;
            return fail(ctx, P3MAZE_ERR_OOM, std::string("rollback copy: ") + cudaGetErrorString(e));
        }
        ctx->snap_bytes = bytes;
    }
    ctx->rollback = true;
    return P3MAZE_OK;
}

int p3maze_set_solver(p3maze_ctx* ctx, double tol, int32_t max_mg_iters) {
    if (!ctx) return fail(nullptr, P3MAZE_ERR_INVALID, "ctx is NULL");
    if (!(tol > 0.0) || !std::isfinite(tol)) return fail(ctx, P3MAZE_ERR_INVALID, "tol must be > 0");
    if (max_mg_iters < 1) return fail(ctx, P3MAZE_ERR_INVALID, "max_mg_iters must be >= 1");
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->tol = tol;
    ctx->itmax = max_mg_iters;
    destroy_graphs(ctx);  // the tolerance and the limit are recorded in the graphs
    ctx->settings_gen += 1;
    return P3MAZE_OK;
}

int p3maze_step_host(p3maze_ctx* ctx, const double* pos_in, const double* vel_in, int32_t nsteps, double* pos_out,
                     double* vel_out) {
    if (!ctx) return fail(nullptr, P3MAZE_ERR_INVALID, "ctx is NULL");
    if (nsteps < 0) return fail(ctx, P3MAZE_ERR_INVALID, "nsteps must be >= 0");
    cudaStream_t s = ctx->stream;
    const size_t bytes = 24 * (size_t)ctx->np;
    int rc = enter(ctx);
    if (rc) return rc;
    rc = take_snapshot(ctx);
    if (rc) return rc;
    if (pos_in) CK(cudaMemcpyAsync(ctx->r, pos_in, bytes, cudaMemcpyHostToDevice, s));
    if (vel_in) CK(cudaMemcpyAsync(ctx->v, vel_in, bytes, cudaMemcpyHostToDevice, s));
    if (pos_in || vel_in) {
        k_wrap_check<<<nblk(3 * (int64_t)ctx->np), P3_THREADS, 0, s>>>(ctx->np, ctx->r, ctx->v, ctx->L,
                                                                        &ctx->dmg->status, P3MAZE_ERR_INVALID);
        CKL();
    }
    for (int k = 0; k < nsteps; ++k) {
        rc = step_once(ctx);
        if (rc) return rc;
    }
    if (pos_out && nsteps > 0) {
        // the last step's positions, copied while its forces are formed
        CK(cudaStreamWaitEvent(ctx->copy_stream, ctx->ev_drift, 0));
        CK(cudaMemcpyAsync(pos_out, ctx->r, bytes, cudaMemcpyDeviceToHost, ctx->copy_stream));
        CK(cudaEventRecord(ctx->ev_copied, ctx->copy_stream));
        CK(cudaStreamWaitEvent(s, ctx->ev_copied, 0));
    } else if (pos_out) {
        CK(cudaMemcpyAsync(pos_out, ctx->r, bytes, cudaMemcpyDeviceToHost, s));
    }
    if (vel_out) CK(cudaMemcpyAsync(vel_out, ctx->v, bytes, cudaMemcpyDeviceToHost, s));
    rc = leave(ctx);
    if (rc) return rc;
    return finish_steps(ctx);
}

int p3maze_equilibrate(p3maze_ctx* ctx, int32_t nsteps, double temperature_K) {
    if (!ctx) return fail(nullptr, P3MAZE_ERR_INVALID, "ctx is NULL");
    if (nsteps < 0 || !(temperature_K > 0.0)) return fail(ctx, P3MAZE_ERR_INVALID, "need nsteps >= 0, T > 0");
    int rc = enter(ctx);
    if (rc) return rc;
    // sum m v^2 (g/mol A^2/fs^2) of (3n - 3) degrees of freedom at T
    const double kb = 0.0019872043;  // kcal/(mol K)
    const double target = (3.0 * ctx->np - 3.0) * kb * temperature_K * P3_ACCEL;
    cudaStream_t s = ctx->stream;
    for (int k = 0; k < nsteps; ++k) {
        rc = step_once(ctx);
        if (rc) return rc;
        k_mv2_partial<<<kReduceBlocks, P3_THREADS, 0, s>>>(ctx->np, ctx->v, ctx->mass, ctx->partial);
        k_sum_final<<<1, P3_THREADS, 0, s>>>(kReduceBlocks, ctx->partial, ctx->dscal + S_MV2);
        k_rescale_v<<<nblk(3 * (int64_t)ctx->np), P3_THREADS, 0, s>>>(ctx->np, ctx->v, ctx->dscal + S_MV2, target);
        CKL();
    }
    rc = leave(ctx);
    if (rc) return rc;
    return read_solver_state(ctx);
}

int p3maze_reinit(p3maze_ctx* ctx) {
    if (!ctx) return fail(nullptr, P3MAZE_ERR_INVALID, "ctx is NULL");
    int rc = enter(ctx);
    if (rc) return rc;
    rc = initialise_field(ctx);
    if (rc) return rc;
    rc = leave(ctx);
    if (rc) return rc;
    CK(cudaStreamSynchronize(ctx->stream));
    return P3MAZE_OK;
}

void p3maze_destroy(p3maze_ctx* ctx) {
    if (!ctx) return;
    cudaStreamSynchronize(ctx->stream);
    release(ctx);
    delete ctx;
}

int p3maze_energy(p3maze_ctx* ctx, p3maze_energies* out) {
    if (!ctx || !out) return fail(ctx, P3MAZE_ERR_INVALID, "NULL argument");
    cudaStream_t s = ctx->stream;
    const int nb = kReduceBlocks;
    int rc0 = enter(ctx);
    if (rc0) return rc0;
    k_sum_partial<double><<<nb, P3_THREADS, 0, s>>>(ctx->np, ctx->ecs, ctx->partial);
    k_sum_final<<<1, P3_THREADS, 0, s>>>(nb, ctx->partial, ctx->dscal + S_ESR);
    k_sum_partial<double><<<nb, P3_THREADS, 0, s>>>(ctx->np, ctx->evs, ctx->partial);
    k_sum_final<<<1, P3_THREADS, 0, s>>>(nb, ctx->partial, ctx->dscal + S_EVDW);
    k_sum_partial<double><<<nb, P3_THREADS, 0, s>>>(ctx->np, ctx->wsr, ctx->partial);
    k_sum_final<<<1, P3_THREADS, 0, s>>>(nb, ctx->partial, ctx->dscal + S_WSR);
    if (ctx->prec == P3MAZE_MIXED)
        k_dot_partial_fix<float><<<nb, P3_THREADS, 0, s>>>(ctx->P, fx(ctx->phi[ctx->icur]), (const float*)ctx->q,
                                                           ctx->partial);
    else
        k_dot_partial<double><<<nb, P3_THREADS, 0, s>>>(ctx->P, ctx->phi[ctx->icur], (const double*)ctx->q, ctx->partial);
    k_sum_final<<<1, P3_THREADS, 0, s>>>(nb, ctx->partial, ctx->dscal + S_VLR);
    k_mv2_partial<<<nb, P3_THREADS, 0, s>>>(ctx->np, ctx->v, ctx->mass, ctx->partial);
    k_sum_final<<<1, P3_THREADS, 0, s>>>(nb, ctx->partial, ctx->dscal + S_MV2);
    if (ctx->nmol) {
        k_sum_partial<double><<<nb, P3_THREADS, 0, s>>>(ctx->nmol, ctx->eb, ctx->partial);
        k_sum_final<<<1, P3_THREADS, 0, s>>>(nb, ctx->partial, ctx->dscal + S_EBOND);
        k_sum_partial<double><<<nb, P3_THREADS, 0, s>>>(ctx->nmol, ctx->ex, ctx->partial);
        k_sum_final<<<1, P3_THREADS, 0, s>>>(nb, ctx->partial, ctx->dscal + S_EXCL);
    }
    CKL();
    int rc = sync_scalars(ctx);
    if (rc) return rc;
    const double* h = ctx->hscal;
    out->v_sr = h[S_ESR];
    out->v_vdw = h[S_EVDW];
    out->v_lr = 0.5 * ctx->ke * h[S_VLR];
    out->v_self = ctx->v_self;
    out->v_bond = ctx->nmol ? h[S_EBOND] : 0.0;
    out->v_excl = ctx->nmol ? h[S_EXCL] : 0.0;
    out->kinetic = 0.5 * h[S_MV2] / P3_ACCEL;
    out->total = out->v_sr + out->v_lr + out->v_self + out->v_excl + out->v_vdw + out->v_bond + out->kinetic;
    out->w_sr = h[S_WSR];
    return P3MAZE_OK;
}

int p3maze_device_bytes(const p3maze_params* p, size_t* out) {
    if (!p || !out) return fail(nullptr, P3MAZE_ERR_INVALID, "NULL argument");
    int nlev = 0, ncoarse = 0;
    if (p->n_particles < 1 || !(p->box[0] > 0.0) || !(p->r_cut > 0.0) || !validate_mesh(p->mesh, &nlev, &ncoarse))
        return fail(nullptr, P3MAZE_ERR_INVALID, "invalid particle count, box, r_cut or mesh");
    *out = planned_bytes(p, nlev);
    return P3MAZE_OK;
}

int p3maze_get_stats(p3maze_ctx* ctx, p3maze_stats* out) {
    if (!ctx || !out) return fail(ctx, P3MAZE_ERR_INVALID, "NULL argument");
    read_solver_state(ctx);
    ctx->st.device_bytes = (int64_t)ctx->dev_bytes;
    *out = ctx->st;
    return P3MAZE_OK;
}

static int copy_out(p3maze_ctx* ctx, const void* dsrc, void* hdst, size_t bytes) {
    int rc = enter(ctx);
    if (rc) return rc;
    CK(cudaMemcpyAsync(hdst, dsrc, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return P3MAZE_OK;
}

int p3maze_get_positions(p3maze_ctx* ctx, double* out) {
    if (!ctx || !out) return fail(ctx, P3MAZE_ERR_INVALID, "NULL argument");
    return copy_out(ctx, ctx->r, out, 24 * (size_t)ctx->np);
}

int p3maze_get_velocities(p3maze_ctx* ctx, double* out) {
    if (!ctx || !out) return fail(ctx, P3MAZE_ERR_INVALID, "NULL argument");
    return copy_out(ctx, ctx->v, out, 24 * (size_t)ctx->np);
}

int p3maze_get_forces(p3maze_ctx* ctx, int32_t which, double* out) {
    if (!ctx || !out) return fail(ctx, P3MAZE_ERR_INVALID, "NULL argument");
    const double* src = which == P3MAZE_F_TOTAL ? ctx->F
                      : which == P3MAZE_F_SR    ? ctx->Fsr
                      : which == P3MAZE_F_LR    ? ctx->Flr
                      : which == P3MAZE_F_BOND  ? ctx->Fb
                                                : nullptr;
    if (!src) return fail(ctx, P3MAZE_ERR_INVALID, "unknown force part");
    return copy_out(ctx, src, out, 24 * (size_t)ctx->np);
}

// ---- checkpoint: every array the next step reads, plus the observables'
// inputs, in a fixed order (the field and correction histories in logical
// order, whatever the ring positions)

int p3maze_state_bytes(p3maze_ctx* ctx, size_t* out) {
    if (!ctx || !out) return fail(ctx, P3MAZE_ERR_INVALID, "NULL argument");
    *out = state_size(ctx);
    return P3MAZE_OK;
}

int p3maze_save_state(p3maze_ctx* ctx, void* buf, size_t bytes) {
    if (!ctx || !buf) return fail(ctx, P3MAZE_ERR_INVALID, "NULL argument");
    if (bytes < state_size(ctx)) return fail(ctx, P3MAZE_ERR_INVALID, "buffer smaller than p3maze_state_bytes");
    int rc = enter(ctx);
    if (rc) return rc;
    CK(cudaMemcpyAsync(ctx->hmg, ctx->dmg, sizeof(MGState), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    StateHeader h{};
    std::memcpy(h.magic, "P3MZSTAT", 8);
    h.version = 2;
    h.np = ctx->np;
    h.mesh = ctx->N;
    h.precision = ctx->prec;
    h.method = ctx->method;
    h.nmol = ctx->nmol;
    h.steps = ctx->st.steps;
    h.nhist = ctx->nhist;
    h.mg = *ctx->hmg;
    unsigned char* p = static_cast<unsigned char*>(buf);
    std::memcpy(p, &h, sizeof h);
    p += sizeof h;
    std::vector<std::pair<void*, size_t>> seg;
    state_segments(ctx, seg);
    for (auto& s : seg) {
        CK(cudaMemcpyAsync(p, s.first, s.second, cudaMemcpyDeviceToHost, ctx->stream));
        p += s.second;
    }
    CK(cudaStreamSynchronize(ctx->stream));
    return leave(ctx);
}

int p3maze_load_state(p3maze_ctx* ctx, const void* buf, size_t bytes) {
    if (!ctx || !buf) return fail(ctx, P3MAZE_ERR_INVALID, "NULL argument");
    if (bytes < state_size(ctx)) return fail(ctx, P3MAZE_ERR_INVALID, "buffer smaller than p3maze_state_bytes");
    StateHeader h{};
    std::memcpy(&h, buf, sizeof h);
    if (std::memcmp(h.magic, "P3MZSTAT", 8) || h.version != 2 || h.np != ctx->np || h.mesh != ctx->N ||
        h.precision != ctx->prec || h.method != ctx->method || h.nmol != ctx->nmol)
        return fail(ctx, P3MAZE_ERR_INVALID, "state was saved from a context with other parameters");
    int rc = enter(ctx);
    if (rc) return rc;
    const unsigned char* p = static_cast<const unsigned char*>(buf) + sizeof h;
    std::vector<std::pair<void*, size_t>> seg;
    state_segments(ctx, seg);
    for (auto& s : seg) {
        CK(cudaMemcpyAsync(s.first, p, s.second, cudaMemcpyHostToDevice, ctx->stream));
        p += s.second;
    }
    MGState mg = h.mg;
    mg.it = 0;
    mg.cont = 0;
    mg.arrive = 0;
    *ctx->hmg = mg;
    CK(cudaMemcpyAsync(ctx->dmg, ctx->hmg, sizeof(MGState), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));  // the pageable source is read before returning
    ctx->st.steps = h.steps;
    ctx->nhist = h.nhist;
    ctx->st.total_iters = mg.total_iters;
    ctx->eager_iters = mg.total_iters;  // V-cycles before the load are not graph body launches
    ctx->graph_iters_seen = 0;
    return leave(ctx);
}

int p3maze_set_state(p3maze_ctx* ctx, const double* pos, const double* vel) {
    if (!ctx || !pos || !vel) return fail(ctx, P3MAZE_ERR_INVALID, "NULL argument");
    for (int64_t i = 0; i < 3 * (int64_t)ctx->np; ++i)
        if (!std::isfinite(pos[i]) || !std::isfinite(vel[i]))
            return fail(ctx, P3MAZE_ERR_INVALID, "non-finite position or velocity");
    cudaStream_t s = ctx->stream;
    int rc = enter(ctx);
    if (rc) return rc;
    CK(cudaMemcpyAsync(ctx->r, pos, 24 * (size_t)ctx->np, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ctx->v, vel, 24 * (size_t)ctx->np, cudaMemcpyHostToDevice, s));
    k_wrap<<<nblk(3 * (int64_t)ctx->np), P3_THREADS, 0, s>>>(ctx->np, ctx->r, ctx->L);
    CKL();
    return leave(ctx);
}

int p3maze_get_mesh(p3maze_ctx* ctx, int32_t which, double* out) {
    if (!ctx || !out) return fail(ctx, P3MAZE_ERR_INVALID, "NULL argument");
    const int64_t P = ctx->P;
    const bool mixed = ctx->prec == P3MAZE_MIXED;
    if (which == P3MAZE_MESH_Q || which == P3MAZE_MESH_QS) {
        const void* src = which == P3MAZE_MESH_Q ? ctx->q : ctx->qs;
        if (mixed) {
            std::vector<float> tmp(P);
            int rc = copy_out(ctx, src, tmp.data(), 4 * (size_t)P);
            if (rc) return rc;
            for (int64_t i = 0; i < P; ++i) out[i] = tmp[i];
        } else {
            int rc = copy_out(ctx, src, out, 8 * (size_t)P);
            if (rc) return rc;
        }
        if (which == P3MAZE_MESH_QS) {
            double qsum = 0.0;
            int rc = copy_out(ctx, ctx->dscal + S_QSUM, &qsum, 8);
            if (rc) return rc;
            const double mean = qsum / (double)P;
            for (int64_t i = 0; i < P; ++i) out[i] -= mean;
        }
        return P3MAZE_OK;
    }
    if ((which == P3MAZE_MESH_Y || which == P3MAZE_MESH_SIGMA) && ctx->st.steps == 0)
        return fail(ctx, P3MAZE_ERR_INVALID, "no correction has been solved yet (take a step first)");
    if (mixed && which == P3MAZE_MESH_SIGMA) {
        // s = r* + M z* (exact in fixed point) from the last solve's final
        // residual and correction; sigma_p = s h/4pi
        std::vector<fix_t> r(P), z(P);
        int rc = copy_out(ctx, ctx->rfin, r.data(), 8 * (size_t)P);
        if (!rc) rc = copy_out(ctx, ctx->yh[1], z.data(), 8 * (size_t)P);
        if (rc) return rc;
        const int n = ctx->N;
        const double to_charge = 1.0 / (1099511627776.0 * ctx->res_unit);
        for (int zz = 0; zz < n; ++zz)
            for (int y = 0; y < n; ++y)
                for (int x = 0; x < n; ++x) {
                    auto at = [&](int a, int b, int c) {
                        return z[((int64_t)((c + n) % n) * n + (b + n) % n) * n + (a + n) % n];
                    };
                    const int64_t i = ((int64_t)zz * n + y) * n + x;
                    const fix_t mz = at(x - 1, y, zz) + at(x + 1, y, zz) + at(x, y - 1, zz) + at(x, y + 1, zz) +
                                     at(x, y, zz - 1) + at(x, y, zz + 1) - 6 * z[i];
                    out[i] = (double)(fix_t)(r[i] + mz) * to_charge;
                }
        return P3MAZE_OK;
    }
    const double* src = which == P3MAZE_MESH_PHI   ? ctx->phi[ctx->icur]
                      : which == P3MAZE_MESH_Y     ? ctx->yh[1]
                      : which == P3MAZE_MESH_SIGMA ? ctx->sig
                                                   : nullptr;
    if (!src) return fail(ctx, P3MAZE_ERR_INVALID, "unknown mesh array");
    if (!mixed) return copy_out(ctx, src, out, 8 * (size_t)P);
    // fixed point (x 2^40, potential units): phi relative to its first node
    // value (the gauge constant is arbitrary), y = z h/4pi, sigma_p = s h/4pi
    std::vector<fix_t> tmp(P);
    int rc = copy_out(ctx, src, tmp.data(), 8 * (size_t)P);
    if (rc) return rc;
    const double unit = 1.0 / 1099511627776.0;
    if (which == P3MAZE_MESH_PHI) {
        const fix_t ref = tmp[0];
        for (int64_t i = 0; i < P; ++i) out[i] = (double)(fix_t)(tmp[i] - ref) * unit;
    } else {
        const double to_charge = unit / ctx->res_unit;
        for (int64_t i = 0; i < P; ++i) out[i] = (double)tmp[i] * to_charge;
    }
    return P3MAZE_OK;
}

int p3maze_get_cells(p3maze_ctx* ctx, int32_t* cell_of, int32_t* cell_start, int32_t* order) {
    if (!ctx) return fail(nullptr, P3MAZE_ERR_INVALID, "ctx is NULL");
    int rc = 0;
    if (cell_of && (rc = copy_out(ctx, ctx->cell, cell_of, 4 * (size_t)ctx->np))) return rc;
    if (cell_start && (rc = copy_out(ctx, ctx->start, cell_start, 4 * ((size_t)ctx->ncell + 1)))) return rc;
    if (order && (rc = copy_out(ctx, ctx->order, order, 4 * (size_t)ctx->np))) return rc;
    return P3MAZE_OK;
}

int p3maze_set_timing(p3maze_ctx* ctx, int32_t enable) {
    if (!ctx) return fail(nullptr, P3MAZE_ERR_INVALID, "ctx is NULL");
    if (enable && !ctx->ev[0][0])
        for (int st = 0; st < P3MAZE_NSTAGES; ++st)
            for (int k = 0; k < 2; ++k) CK(cudaEventCreate(&ctx->ev[st][k]));
    CK(cudaStreamSynchronize(ctx->stream));
    if ((enable != 0) != ctx->timing) {  // event-record nodes differ
        destroy_graphs(ctx);
        ctx->settings_gen += 1;
    }
    ctx->timing = enable != 0;
    for (int st = 0; st < P3MAZE_NSTAGES; ++st) {
        ctx->stage_ms[st] = 0.0;
        ctx->launches[st] = 0;
        ctx->pending[st] = false;
    }
    ctx->timed_steps = 0;
    return P3MAZE_OK;
}

namespace {

struct Setting {
    int pred, nu1, nu2, zc, fuse, pair_fork, cmax, pblocks;
    bool operator==(const Setting& o) const {
        return pred == o.pred && nu1 == o.nu1 && nu2 == o.nu2 && zc == o.zc && fuse == o.fuse &&
               pair_fork == o.pair_fork && cmax == o.cmax && pblocks == o.pblocks;
    }
};

// Run `warm` + `steps` steps under setting `cfg`; ms per timed step.
int tune_trial(p3maze_ctx* ctx, const Setting& cfg, int warm, int steps, double* ms) {
    if (ctx->method != P3MAZE_METHOD_P3M) ctx->pred = cfg.pred;
    ctx->nu1 = cfg.nu1;
    ctx->nu2 = cfg.nu2;
    ctx->zc = cfg.zc;
    ctx->fuse = cfg.fuse;
    ctx->pair_fork = cfg.pair_fork;
    ctx->pair_blocks = cfg.pblocks;
    set_coarse(ctx, cfg.cmax);
    destroy_graphs(ctx);  // the setting is recorded in the graphs
    ctx->settings_gen += 1;
    for (int k = 0; k < warm; ++k) {
        int rc = step_once(ctx);
        if (rc) return rc;
    }
    cudaEvent_t a, b;
    CK(cudaEventCreate(&a));
    CK(cudaEventCreate(&b));
    CK(cudaEventRecord(a, ctx->stream));
    for (int k = 0; k < steps; ++k) {
        int rc = step_once(ctx);
        if (rc) {
            cudaEventDestroy(a);
            cudaEventDestroy(b);
            return rc;
        }
    }
    CK(cudaEventRecord(b, ctx->stream));
    CK(cudaEventSynchronize(b));
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, a, b));
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    *ms = t / std::max(steps, 1);
    return read_solver_state(ctx);
}

}  // namespace

int p3maze_autotune(p3maze_ctx* ctx, int32_t steps_per_trial, p3maze_tuning* out) {
    if (!ctx || !out) return fail(ctx, P3MAZE_ERR_INVALID, "NULL argument");
    if (steps_per_trial < 1) return fail(ctx, P3MAZE_ERR_INVALID, "steps_per_trial must be >= 1");
    int rc = enter(ctx);
    if (rc) return rc;
    const bool timing = ctx->timing;
    ctx->timing = false;
    const int warm = 2;
    const Setting start = {ctx->pred, ctx->nu1, ctx->nu2, ctx->zc, ctx->fuse, ctx->pair_fork, ctx->cmax,
                           ctx->pair_blocks};
    std::vector<Setting> cand;
    const int preds[3] = {1, 2, 3};
    const int sweeps[5][2] = {{1, 1}, {2, 1}, {1, 2}, {2, 2}, {3, 3}};
    const int np = ctx->method == P3MAZE_METHOD_P3M ? 1 : 3;
    for (int a = 0; a < np; ++a)
        for (auto& sw : sweeps)
            cand.push_back({ctx->method == P3MAZE_METHOD_P3M ? 0 : preds[a], sw[0], sw[1], start.zc, start.fuse,
                            start.pair_fork, start.cmax, start.pblocks});
    double initial = 0.0, best = 1e300;
    Setting chosen = start;
    int trials = 0, steps = 0;
    std::vector<std::pair<double, Setting>> log;  // every trial's time
    rc = tune_trial(ctx, start, warm, steps_per_trial, &initial);
    log.push_back({initial, start});
    trials += 1;
    steps += warm + steps_per_trial;
    if (!rc) {
        best = initial;
        for (const Setting& c : cand) {
            double ms = 0.0;
            rc = tune_trial(ctx, c, warm, steps_per_trial, &ms);
            trials += 1;
            steps += warm + steps_per_trial;
            if (rc) break;
            log.push_back({ms, c});
            if (ms < best) {
                best = ms;
                chosen = c;
            }
        }
    }
    // diffusion kernel: steps per launch (mixed: 1 to 4, or all in a
    // cluster) x z planes per thread (one or two steps per launch, N % 4 ==
    // 0: 1-8) or per block (temporal blocking: 8-64 in quads, else 4-32)
    auto diffusion_pass = [&]() {
        if (ctx->K == 0) return;  // no smoothing (PMaZe)
        const int fuses[6] = {1, 2, 3, 4, 5, 6};
        const int zcs_quad[4] = {1, 2, 4, 8}, zcs_tq[4] = {8, 16, 32, 64}, zcs_other[4] = {4, 8, 16, 32};
        const Setting base = chosen;
        for (int f : fuses) {
            if (f > 1 && ctx->prec != P3MAZE_MIXED) continue;
            if (f == 2 && ctx->N % 4 != 0) continue;
            if (f == 5 && !ctx->cluster_ok) continue;
            if (f == 6 && !ctx->Ssm) continue;
            const bool quad = f <= 2 && ctx->prec == P3MAZE_MIXED && ctx->N % 4 == 0;
            // the cluster kernel has no z planes per thread: one trial
            const bool tq = f >= 3 && f <= 4 && ctx->N % 4 == 0;
            std::vector<int> zcs = f >= 5 ? std::vector<int>{base.zc}
                                   : quad ? std::vector<int>(zcs_quad, zcs_quad + 4)
                                   : tq   ? std::vector<int>(zcs_tq, zcs_tq + 4)
                                          : std::vector<int>(zcs_other, zcs_other + 4);
            for (int z : zcs) {
                if (z == base.zc && f == base.fuse) continue;
                Setting c = chosen;
                c.zc = z;
                c.fuse = f;
                double ms = 0.0;
                rc = tune_trial(ctx, c, warm, steps_per_trial, &ms);
                trials += 1;
                steps += warm + steps_per_trial;
                if (rc) return;
                log.push_back({ms, c});
                if (ms < best) {
                    best = ms;
                    chosen = c;
                }
            }
        }
    };
    if (!rc) diffusion_pass();
    if (!rc) {
        // size of the exactly solved coarse level (distinct levels only)
        const int cms[3] = {16, 32, 64};
        for (int cm : cms) {
            if (coarse_level(ctx, cm) == coarse_level(ctx, chosen.cmax)) continue;
            Setting c = chosen;
            c.cmax = cm;
            double ms = 0.0;
            rc = tune_trial(ctx, c, warm, steps_per_trial, &ms);
            trials += 1;
            steps += warm + steps_per_trial;
            if (rc) break;
            log.push_back({ms, c});
            if (ms < best) {
                best = ms;
                chosen = c;
            }
        }
    }
    if (!rc) {
        // fork point and grid of the short-range branch: one block per home
        // box, or a persistent grid of one or two blocks per SM that leaves
        // room for the mesh kernels running beside it
        const Setting base = chosen;
        const int grids[4] = {0, ctx->nsm / 2, ctx->nsm, 2 * ctx->nsm};
        for (int pf = 0; pf < 2 && !rc; ++pf)
            for (int gb : grids) {
                if (pf == base.pair_fork && gb == base.pblocks) continue;
                Setting c = base;
                c.pair_fork = pf;
                c.pblocks = gb;
                double ms = 0.0;
                rc = tune_trial(ctx, c, warm, steps_per_trial, &ms);
                trials += 1;
                steps += warm + steps_per_trial;
                if (rc) break;
                log.push_back({ms, c});
                if (ms < best) {
                    best = ms;
                    chosen = c;
                }
            }
    }
    // the diffusion kernel again once the pair branch is placed: which kernel
    // is fastest depends on what runs beside it
    if (!rc && (chosen.pair_fork != start.pair_fork || chosen.pblocks != start.pblocks)) diffusion_pass();
    // confirmation: the starting setting and the three fastest other
    // settings timed again, twice as long, in two rounds of opposite order.
    // Single short trials are noisy and the state drifts while tuning, so a
    // close call is otherwise decided by chance (measured: at 10^6 ions the
    // greedy passes kept a persistent pair grid 6 % slower than the
    // per-box grid).  The reported times are these re-measurements.
    if (!rc && log.size() > 1) {
        std::stable_sort(log.begin(), log.end(),
                         [](const std::pair<double, Setting>& a, const std::pair<double, Setting>& b) {
                             return a.first < b.first;
                         });
        std::vector<Setting> top{start};
        for (const auto& e : log) {
            if (top.size() == 4) break;
            bool seen = false;
            for (const Setting& t : top) seen = seen || t == e.second;
            if (!seen) top.push_back(e.second);
        }
        std::vector<double> sum(top.size(), 0.0);
        for (int round = 0; round < 2 && !rc; ++round)
            for (size_t k = 0; k < top.size() && !rc; ++k) {
                const size_t i = round == 0 ? k : top.size() - 1 - k;
                double ms = 0.0;
                rc = tune_trial(ctx, top[i], warm, 2 * steps_per_trial, &ms);
                trials += 1;
                steps += warm + 2 * steps_per_trial;
                sum[i] += ms;
            }
        if (!rc) {
            size_t bi = 0;
            for (size_t i = 1; i < top.size(); ++i)
                if (sum[i] < sum[bi]) bi = i;
            chosen = top[bi];
            best = 0.5 * sum[bi];
            initial = 0.5 * sum[0];
        }
    }
    // keep the fastest setting
    if (ctx->method != P3MAZE_METHOD_P3M) ctx->pred = chosen.pred;
    ctx->nu1 = chosen.nu1;
    ctx->nu2 = chosen.nu2;
    ctx->zc = chosen.zc;
    ctx->fuse = chosen.fuse;
    ctx->pair_fork = chosen.pair_fork;
    ctx->pair_blocks = chosen.pblocks;
    set_coarse(ctx, chosen.cmax);
    destroy_graphs(ctx);
    ctx->settings_gen += 1;
    ctx->timing = timing;
    out->predictor = ctx->pred;
    out->pre_sweeps = ctx->nu1;
    out->post_sweeps = ctx->nu2;
    out->diffusion_zc = ctx->zc;
    out->diffusion_fuse = ctx->fuse;
    out->pair_fork = ctx->pair_fork;
    out->coarse_max = ctx->cmax;
    out->pair_blocks = ctx->pair_blocks;
    out->cluster_ctas = ctx->cl_ctas;
    out->sweep_fuse = ctx->sweep_fuse;
    out->ms_per_step = best;
    out->initial_ms_per_step = initial;
    out->trials = trials;
    out->steps = steps;
    if (rc) return rc;
    return leave(ctx);
}

int p3maze_set_tuning(p3maze_ctx* ctx, const p3maze_tuning* t) {
    if (!ctx || !t) return fail(ctx, P3MAZE_ERR_INVALID, "NULL argument");
    if (t->predictor < 1 || t->predictor > 3 || t->pre_sweeps < 1 || t->post_sweeps < 0 || t->diffusion_zc < 1 ||
        t->diffusion_fuse < 1 || t->diffusion_fuse > 6 || (t->pair_fork != 0 && t->pair_fork != 1) ||
        t->coarse_max < 1 || t->pair_blocks < 0 || t->cluster_ctas < 0 || t->cluster_ctas > kClMaxCTAs ||
        (t->cluster_ctas & (t->cluster_ctas - 1)) != 0 || (t->sweep_fuse != 0 && t->sweep_fuse != 1))
        return fail(ctx, P3MAZE_ERR_INVALID, "tuning field out of range");
    if (t->diffusion_fuse > 1 && ctx->prec != P3MAZE_MIXED)
        return fail(ctx, P3MAZE_ERR_INVALID, "fused diffusion steps need mixed precision");
    if (t->diffusion_fuse == 6 && !ctx->Ssm)
        return fail(ctx, P3MAZE_ERR_INVALID, "spectral smoothing needs mixed precision and N <= 64 or N in {128, 192, 256, 320, 384}");
    if (t->diffusion_fuse == 5 && !ctx->cluster_ok)
        return fail(ctx, P3MAZE_ERR_INVALID,
                    "cluster smoothing needs 16 <= N <= 64, N % 4 == 0 and a device that runs such clusters");
    if (t->diffusion_fuse == 5 && t->cluster_ctas &&
        (cluster_smem_bytes(ctx->N, t->cluster_ctas) > kClSmemBudget + 16 ||
         !cluster_smoothing_supported(t->cluster_ctas)))
        return fail(ctx, P3MAZE_ERR_INVALID, "cluster_ctas too small for this mesh or not run by the device");
    CK(cudaStreamSynchronize(ctx->stream));
    if (ctx->method != P3MAZE_METHOD_P3M) ctx->pred = t->predictor;
    ctx->nu1 = t->pre_sweeps;
    ctx->nu2 = t->post_sweeps;
    ctx->zc = t->diffusion_zc;
    ctx->fuse = t->diffusion_fuse;
    ctx->pair_fork = t->pair_fork;
    ctx->pair_blocks = t->pair_blocks;
    ctx->cl_ctas = t->cluster_ctas;
    ctx->sweep_fuse = t->sweep_fuse;
    set_coarse(ctx, t->coarse_max);
    destroy_graphs(ctx);
    ctx->settings_gen += 1;
    return P3MAZE_OK;
}

int p3maze_get_tuning(p3maze_ctx* ctx, p3maze_tuning* out) {
    if (!ctx || !out) return fail(ctx, P3MAZE_ERR_INVALID, "NULL argument");
    *out = p3maze_tuning{};
    out->predictor = ctx->pred;
    out->pre_sweeps = ctx->nu1;
    out->post_sweeps = ctx->nu2;
    out->diffusion_zc = ctx->zc;
    out->diffusion_fuse = ctx->fuse;
    out->pair_fork = ctx->pair_fork;
    out->coarse_max = ctx->cmax;
    out->pair_blocks = ctx->pair_blocks;
    out->cluster_ctas = ctx->cl_ctas;
    out->sweep_fuse = ctx->sweep_fuse;
    return P3MAZE_OK;
}

int p3maze_set_graphs(p3maze_ctx* ctx, int32_t enable) {
    if (!ctx) return fail(nullptr, P3MAZE_ERR_INVALID, "ctx is NULL");
    CK(cudaStreamSynchronize(ctx->stream));
    if (!enable) {
        destroy_graphs(ctx);
        ctx->settings_gen += 1;
    }
    ctx->use_graphs = enable != 0;
    return P3MAZE_OK;
}

int p3maze_get_timing(p3maze_ctx* ctx, p3maze_timing* out) {
    if (!ctx || !out) return fail(ctx, P3MAZE_ERR_INVALID, "NULL argument");
    int64_t tot = 0;
    for (int st = 0; st < P3MAZE_NSTAGES; ++st) {
        out->ms[st] = ctx->stage_ms[st];
        out->launches[st] = ctx->launches[st];
        tot += ctx->launches[st];
    }
    out->timed_steps = ctx->timed_steps;
    out->total_launches = tot;
    return P3MAZE_OK;
}

// ------------------------------------------------------------------ batches
}  // extern "C"


struct p3maze_batch {
    cudaStream_t origin = nullptr;      // capture and launch stream
    cudaStream_t user = nullptr;        // caller's stream (fenced on entry and exit)
    cudaEvent_t ev_in = nullptr, ev_out = nullptr, ev_fork = nullptr;
    std::vector<p3maze_ctx*> members;
    std::vector<cudaEvent_t> ev_done;   // per member: end of its branch
    struct Phase {
        bool valid = false;
        cudaGraph_t g = nullptr;
        cudaGraphExec_t x = nullptr;
        std::vector<int> icur;
        std::vector<std::array<double*, 4>> yh;
        std::vector<std::array<int64_t, P3MAZE_NSTAGES>> launches;  // per member and step
    };
    Phase phases[kMaxGraphs];
    int mode = 0;                       // P3MAZE_BATCH_SHARED_GRAPH or P3MAZE_BATCH_PER_MEMBER
    // the members smoothed by the batch's cluster launches (mode 5)
    ClusterMesh* cltab = nullptr;       // device table, cl_cap entries
    int cl_cap = 0;
    bool cl_dirty = true;               // membership or a member's setting changed: rebuild
    int fuse_smoothing = -1;            // smooth the mode-5 members together: 1 yes, 0 each in its own
                                        // step, -1 by mode (yes for per-member, no for the shared graph)
    std::vector<ClusterMesh> cl_host;
    std::vector<char> cl_member;        // per member: in the table
    std::vector<int64_t> gen_seen;      // per member: settings_gen when the table was built
    struct ClGroup {
        int cs, first, count, nmax;     // cluster size; table entries [first, first + count)
    };
    std::vector<ClGroup> cl_groups;     // one launch per cluster size
    std::string err = "no error";
};

namespace {

int bfail(p3maze_batch* b, int code, const std::string& msg) {
    if (b) b->err = msg;
    else g_init_error = msg;
    return code;
}

#define BCK(call)                                                                              \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess) {                                                               \
            cudaGetLastError();                                                                \
            return bfail(b, P3MAZE_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
        }                                                                                      \
    } while (0)

void batch_drop_graphs(p3maze_batch* b) {
    for (auto& ph : b->phases) {
        if (ph.x) cudaGraphExecDestroy(ph.x);
        if (ph.g) cudaGraphDestroy(ph.g);
        ph = p3maze_batch::Phase();
    }
}

bool phase_matches(const p3maze_batch::Phase& ph, const std::vector<p3maze_ctx*>& m) {
    if (!ph.valid || ph.icur.size() != m.size()) return false;
    for (size_t i = 0; i < m.size(); ++i) {
        if (ph.icur[i] != m[i]->icur) return false;
        for (int k = 0; k < 4; ++k)
            if (ph.yh[i][k] != m[i]->yh[k]) return false;
    }
    return true;
}

// One graph holding one MD step of every member, each member's step a branch
// from a common fork (with its own device-side multigrid while node).  The
// members smoothed by the batch's cluster launches (mode 5) branch twice:
// their heads (kick/drift, cell list, assignment) join the batch stream, the
// cluster launches smooth all their meshes, and their tails fork again.
int batch_capture(p3maze_batch* b, p3maze_batch::Phase& ph) {
    struct Saved {
        int icur;
        std::array<double*, 4> yh;
        bool timing;
        int64_t launches[P3MAZE_NSTAGES];
    };
    std::vector<Saved> sv(b->members.size());
    std::vector<char> held(b->members.size(), 0);  // state saved, not yet restored
    BCK(cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaEventRecord(b->ev_fork, b->origin);
    int rc = e == cudaSuccess ? P3MAZE_OK : bfail(b, P3MAZE_ERR_CUDA, cudaGetErrorString(e));
    ph.icur.clear();
    ph.yh.clear();
    ph.launches.assign(b->members.size(), {});
    auto restore = [&](size_t i) {
        p3maze_ctx* m = b->members[i];
        held[i] = 0;
        m->capturing = false;
        m->timing = sv[i].timing;
        for (int st = 0; st < P3MAZE_NSTAGES; ++st) {
            ph.launches[i][st] = m->launches[st] - sv[i].launches[st];
            m->launches[st] = sv[i].launches[st];
        }
        m->icur = sv[i].icur;
        for (int k = 0; k < 4; ++k) m->yh[k] = sv[i].yh[k];
    };
    auto join = [&](size_t i) {
        cudaError_t je = cudaEventRecord(b->ev_done[i], b->members[i]->stream);
        if (je == cudaSuccess) je = cudaStreamWaitEvent(b->origin, b->ev_done[i], 0);
        return je == cudaSuccess ? P3MAZE_OK : bfail(b, P3MAZE_ERR_CUDA, cudaGetErrorString(je));
    };
    bool any_split = false;
    for (size_t i = 0; i < b->members.size() && !rc; ++i) {
        p3maze_ctx* m = b->members[i];
        e = cudaStreamWaitEvent(m->stream, b->ev_fork, 0);
        if (e != cudaSuccess) {
            rc = bfail(b, P3MAZE_ERR_CUDA, cudaGetErrorString(e));
            break;
        }
        Saved& s = sv[i];
        s.icur = m->icur;
        for (int k = 0; k < 4; ++k) s.yh[k] = m->yh[k];
        s.timing = m->timing;
        for (int st = 0; st < P3MAZE_NSTAGES; ++st) s.launches[st] = m->launches[st];
        held[i] = 1;
        ph.icur.push_back(s.icur);
        ph.yh.push_back(s.yh);
        m->timing = false;
        m->capturing = true;
        const bool split = b->cl_member[i] != 0;
        any_split |= split;
        rc = split ? step_head(m) : step_body(m, m->pred);
        if (!split || rc) restore(i);
        if (rc) {
            rc = bfail(b, rc, std::string("member ") + std::to_string(i) + ": " + m->err);
            break;
        }
        m->capturing = false;
        if (split) rc = join(i);  // whole steps join at the end: the cluster launch waits for heads only
    }
    if (!rc && any_split) {
        for (const p3maze_batch::ClGroup& g : b->cl_groups) {
            e = launch_cluster_smoothing(b->cltab + g.first, g.count, g.cs, g.nmax, b->origin, false);
            if (e != cudaSuccess) {
                rc = bfail(b, P3MAZE_ERR_CUDA, std::string("cluster smoothing: ") + cudaGetErrorString(e));
                break;
            }
        }
        if (!rc) {
            e = cudaEventRecord(b->ev_fork, b->origin);
            if (e != cudaSuccess) rc = bfail(b, P3MAZE_ERR_CUDA, cudaGetErrorString(e));
        }
        for (size_t i = 0; i < b->members.size() && !rc; ++i) {
            if (!b->cl_member[i]) continue;
            p3maze_ctx* m = b->members[i];
            e = cudaStreamWaitEvent(m->stream, b->ev_fork, 0);
            if (e != cudaSuccess) {
                rc = bfail(b, P3MAZE_ERR_CUDA, cudaGetErrorString(e));
                break;
            }
            m->capturing = true;
            rc = step_tail(m, m->pred);
            restore(i);
            if (rc) {
                rc = bfail(b, rc, std::string("member ") + std::to_string(i) + ": " + m->err);
                break;
            }
            rc = join(i);
        }
    }
    for (size_t i = 0; i < b->members.size() && !rc; ++i)
        if (!b->cl_member[i]) rc = join(i);
    for (size_t i = 0; i < b->members.size(); ++i)  // after a failure: members left between head and tail
        if (held[i]) restore(i);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(b->origin, &g);
    if (rc || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return rc ? rc : bfail(b, P3MAZE_ERR_CUDA, std::string("batch capture: ") + cudaGetErrorString(e));
    }
    e = cudaGraphInstantiate(&ph.x, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return bfail(b, P3MAZE_ERR_CUDA, std::string("batch instantiate: ") + cudaGetErrorString(e));
    }
    ph.g = g;
    ph.valid = true;
    return P3MAZE_OK;
}

}  // namespace

extern "C" {

int p3maze_batch_create(void* cuda_stream, p3maze_batch** out) {
    if (!out) return bfail(nullptr, P3MAZE_ERR_INVALID, "out is NULL");
    *out = nullptr;
    p3maze_batch* b = new (std::nothrow) p3maze_batch();
    if (!b) return bfail(nullptr, P3MAZE_ERR_OOM, "host allocation failed");
    b->user = (cudaStream_t)cuda_stream;
    int least = 0, greatest = 0;
    cudaError_t e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&b->origin, cudaStreamNonBlocking, greatest);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        const std::string msg = std::string("batch create: ") + cudaGetErrorString(e);
        p3maze_batch_destroy(b);
        return bfail(nullptr, P3MAZE_ERR_CUDA, msg);
    }
    *out = b;
    return P3MAZE_OK;
}

int p3maze_batch_add(p3maze_batch* b, p3maze_ctx* ctx) {
    if (!b || !ctx) return bfail(b, P3MAZE_ERR_INVALID, "NULL argument");
    for (p3maze_ctx* m : b->members)
        if (m == ctx) return bfail(b, P3MAZE_ERR_INVALID, "context is already in the batch");
    int dev = 0;
    BCK(cudaGetDevice(&dev));
    if (dev != ctx->device) return bfail(b, P3MAZE_ERR_INVALID, "context belongs to another device");
    // a member joins with a full multiplier history (its first steps test
    // convergence on the host and cannot be recorded in the batch graph)
    if (ctx->nhist < ctx->pred) {
        int rc = p3maze_step(ctx, ctx->pred - ctx->nhist);
        if (rc) return bfail(b, rc, std::string("warm-up of the new member: ") + ctx->err);
    }
    BCK(cudaStreamSynchronize(ctx->stream));
    cudaEvent_t ev;
    BCK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    b->members.push_back(ctx);
    b->ev_done.push_back(ev);
    b->cl_dirty = true;
    batch_drop_graphs(b);
    return P3MAZE_OK;
}

int p3maze_batch_remove(p3maze_batch* b, p3maze_ctx* ctx) {
    if (!b || !ctx) return bfail(b, P3MAZE_ERR_INVALID, "NULL argument");
    for (size_t i = 0; i < b->members.size(); ++i)
        if (b->members[i] == ctx) {
            BCK(cudaStreamSynchronize(b->origin));
            cudaEventDestroy(b->ev_done[i]);
            b->members.erase(b->members.begin() + (long)i);
            b->ev_done.erase(b->ev_done.begin() + (long)i);
            b->cl_dirty = true;
            batch_drop_graphs(b);
            return P3MAZE_OK;
        }
    return bfail(b, P3MAZE_ERR_INVALID, "context is not in the batch");
}

int p3maze_batch_step(p3maze_batch* b, int32_t nsteps) {
    if (!b) return bfail(nullptr, P3MAZE_ERR_INVALID, "batch is NULL");
    if (nsteps < 0) return bfail(b, P3MAZE_ERR_INVALID, "nsteps must be >= 0");
    if (b->members.empty() || nsteps == 0) return P3MAZE_OK;
    BCK(cudaEventRecord(b->ev_in, b->user));
    BCK(cudaStreamWaitEvent(b->origin, b->ev_in, 0));
    if (!b->cl_dirty) {
        // a member's setting may have changed since (p3maze_set_tuning, p3maze_autotune, timing)
        for (size_t i = 0; i < b->members.size(); ++i)
            if (b->members[i]->settings_gen != b->gen_seen[i]) b->cl_dirty = true;
    }
    if (b->cl_dirty) {
        // members whose smoothing is a cluster launch (mode 5) share one
        // launch per cluster size; the size per mesh shrinks as the batch
        // grows (cluster_size_for), down to the smallest whose slabs fit.
        // The shared graphs record the table and the members' settings.
        batch_drop_graphs(b);
        b->cl_host.clear();
        b->cl_groups.clear();
        b->cl_member.assign(b->members.size(), 0);
        b->gen_seen.resize(b->members.size());
        for (size_t i = 0; i < b->members.size(); ++i) b->gen_seen[i] = b->members[i]->settings_gen;
        int ncl = 0, nsm = 148;
        for (p3maze_ctx* m : b->members) {
            ncl += m->fuse == 5;
            nsm = m->nsm;
        }
        std::vector<std::pair<int, int>> order;  // (cluster size, member)
        for (size_t i = 0; i < b->members.size(); ++i) {
            p3maze_ctx* m = b->members[i];
            const bool fused = b->fuse_smoothing < 0 ? b->mode == P3MAZE_BATCH_PER_MEMBER : b->fuse_smoothing != 0;
            if (m->fuse != 5 || !fused) continue;
            b->cl_member[i] = 1;
            int cs = m->cl_ctas ? m->cl_ctas : cluster_size_for(m->N, ncl, nsm);
            if (!cluster_smoothing_supported(cs)) cs = cluster_size_for(m->N, 1, nsm);  // its own, checked at init
            order.emplace_back(cs, (int)i);
        }
        std::stable_sort(order.begin(), order.end(),
                         [](const std::pair<int, int>& x, const std::pair<int, int>& y) { return x.first < y.first; });
        for (const auto& [cs, i] : order) {
            p3maze_ctx* m = b->members[i];
            if (b->cl_groups.empty() || b->cl_groups.back().cs != cs)
                b->cl_groups.push_back(p3maze_batch::ClGroup{cs, (int)b->cl_host.size(), 0, 0});
            b->cl_groups.back().count += 1;
            b->cl_groups.back().nmax = std::max(b->cl_groups.back().nmax, m->N);
            b->cl_host.push_back(ClusterMesh{(const float*)m->q, (float*)m->qs, m->dscal + S_QSUM, m->N, m->K,
                                             (float)m->c, 0});
        }
        if ((int)b->cl_host.size() > b->cl_cap) {
            BCK(cudaStreamSynchronize(b->origin));
            if (b->cltab) cudaFree(b->cltab);
            b->cltab = nullptr;
            b->cl_cap = 0;
            const int cap = std::max<int>(16, (int)b->cl_host.size() * 2);
            BCK(cudaMalloc(&b->cltab, sizeof(ClusterMesh) * cap));
            b->cl_cap = cap;
        }
        if (!b->cl_host.empty())
            BCK(cudaMemcpyAsync(b->cltab, b->cl_host.data(), sizeof(ClusterMesh) * b->cl_host.size(),
                                cudaMemcpyHostToDevice, b->origin));
        b->cl_dirty = false;
    }
    if (b->mode == P3MAZE_BATCH_PER_MEMBER && !b->cl_host.empty()) {
        // heads of every member's step on their own streams; the smoothing of
        // the cluster members as one launch per cluster size on the batch
        // stream; then the tails.  Members not smoothed there take whole
        // steps from the first fork and join at the end, so the cluster
        // launch waits for the heads only.
        for (int k = 0; k < nsteps; ++k) {
            BCK(cudaEventRecord(b->ev_fork, b->origin));
            for (size_t i = 0; i < b->members.size(); ++i) {
                p3maze_ctx* m = b->members[i];
                BCK(cudaStreamWaitEvent(m->stream, b->ev_fork, 0));
                int rc = b->cl_member[i] ? step_graph(m, PART_HEAD) : step_once(m);
                if (rc) return bfail(b, rc, std::string("member ") + std::to_string(i) + ": " + m->err);
                BCK(cudaEventRecord(b->ev_done[i], m->stream));
                if (b->cl_member[i]) BCK(cudaStreamWaitEvent(b->origin, b->ev_done[i], 0));
            }
            for (const p3maze_batch::ClGroup& g : b->cl_groups)
                BCK(launch_cluster_smoothing(b->cltab + g.first, g.count, g.cs, g.nmax, b->origin, false));
            BCK(cudaEventRecord(b->ev_fork, b->origin));
            for (size_t i = 0; i < b->members.size(); ++i) {
                if (!b->cl_member[i]) continue;
                p3maze_ctx* m = b->members[i];
                BCK(cudaStreamWaitEvent(m->stream, b->ev_fork, 0));
                int rc = step_graph(m, PART_TAIL);
                if (!rc) {
                    m->nhist = std::min(m->nhist + 1, 3);
                    m->st.steps += 1;
                    rc = collect_timing(m);
                }
                if (rc) return bfail(b, rc, std::string("member ") + std::to_string(i) + ": " + m->err);
                BCK(cudaEventRecord(b->ev_done[i], m->stream));
                BCK(cudaStreamWaitEvent(b->origin, b->ev_done[i], 0));
            }
            for (size_t i = 0; i < b->members.size(); ++i)
                if (!b->cl_member[i]) BCK(cudaStreamWaitEvent(b->origin, b->ev_done[i], 0));
        }
        BCK(cudaEventRecord(b->ev_out, b->origin));
        BCK(cudaStreamWaitEvent(b->user, b->ev_out, 0));
        return P3MAZE_OK;
    }
    if (b->mode == P3MAZE_BATCH_PER_MEMBER) {
        // each member replays its own cached step graph on its own stream,
        // forked from and joined to the batch stream
        for (int k = 0; k < nsteps; ++k) {
            BCK(cudaEventRecord(b->ev_fork, b->origin));
            for (size_t i = 0; i < b->members.size(); ++i) {
                p3maze_ctx* m = b->members[i];
                BCK(cudaStreamWaitEvent(m->stream, b->ev_fork, 0));
                int rc = step_once(m);
                if (rc) return bfail(b, rc, std::string("member ") + std::to_string(i) + ": " + m->err);
                BCK(cudaEventRecord(b->ev_done[i], m->stream));
                BCK(cudaStreamWaitEvent(b->origin, b->ev_done[i], 0));
            }
        }
        BCK(cudaEventRecord(b->ev_out, b->origin));
        BCK(cudaStreamWaitEvent(b->user, b->ev_out, 0));
        return P3MAZE_OK;
    }
    for (int k = 0; k < nsteps; ++k) {
        p3maze_batch::Phase* ph = nullptr;
        for (auto& c : b->phases)
            if (phase_matches(c, b->members)) ph = &c;
        if (!ph) {
            for (auto& c : b->phases)
                if (!c.valid) {
                    ph = &c;
                    break;
                }
            if (!ph) {
                batch_drop_graphs(b);
                ph = &b->phases[0];
            }
            int rc = batch_capture(b, *ph);
            if (rc) return rc;
        }
        BCK(cudaGraphLaunch(ph->x, b->origin));
        for (size_t i = 0; i < b->members.size(); ++i) {
            p3maze_ctx* m = b->members[i];
            for (int st = 0; st < P3MAZE_NSTAGES; ++st) m->launches[st] += ph->launches[i][st];
            m->icur = 1 - m->icur;
            double* oldest = m->yh[3];
            m->yh[3] = m->yh[2];
            m->yh[2] = m->yh[1];
            m->yh[1] = m->yh[0];
            m->yh[0] = oldest;
            m->st.steps += 1;
        }
    }
    BCK(cudaEventRecord(b->ev_out, b->origin));
    BCK(cudaStreamWaitEvent(b->user, b->ev_out, 0));
    return P3MAZE_OK;
}

int p3maze_batch_wait(p3maze_batch* b) {
    if (!b) return bfail(nullptr, P3MAZE_ERR_INVALID, "batch is NULL");
    BCK(cudaStreamSynchronize(b->origin));
    for (size_t i = 0; i < b->members.size(); ++i) {
        int rc = read_solver_state(b->members[i]);
        if (rc) return bfail(b, rc, std::string("member ") + std::to_string(i) + ": " + b->members[i]->err);
    }
    return P3MAZE_OK;
}

int p3maze_batch_size(const p3maze_batch* b) { return b ? (int)b->members.size() : 0; }

int p3maze_batch_set_fused_smoothing(p3maze_batch* b, int32_t enable) {
    if (!b) return bfail(nullptr, P3MAZE_ERR_INVALID, "batch is NULL");
    BCK(cudaStreamSynchronize(b->origin));
    b->fuse_smoothing = enable < 0 ? -1 : enable != 0;
    b->cl_dirty = true;
    return P3MAZE_OK;
}

int p3maze_batch_set_mode(p3maze_batch* b, int32_t mode) {
    if (!b) return bfail(nullptr, P3MAZE_ERR_INVALID, "batch is NULL");
    if (mode != P3MAZE_BATCH_SHARED_GRAPH && mode != P3MAZE_BATCH_PER_MEMBER)
        return bfail(b, P3MAZE_ERR_INVALID, "unknown batch mode");
    BCK(cudaStreamSynchronize(b->origin));
    b->mode = mode;
    b->cl_dirty = true;
    return P3MAZE_OK;
}

void p3maze_batch_destroy(p3maze_batch* b) {
    if (!b) return;
    if (b->origin) cudaStreamSynchronize(b->origin);
    batch_drop_graphs(b);
    for (cudaEvent_t e : b->ev_done) cudaEventDestroy(e);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    if (b->origin) cudaStreamDestroy(b->origin);
    if (b->cltab) cudaFree(b->cltab);
    delete b;
}

const char* p3maze_batch_last_error(const p3maze_batch* b) { return b ? b->err.c_str() : g_init_error.c_str(); }

const char* p3maze_last_error(const p3maze_ctx* ctx) {
    return ctx ? ctx->err.c_str() : g_init_error.c_str();
}

}  // extern "C"
