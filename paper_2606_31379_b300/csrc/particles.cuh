// Particle-side kernels: velocity-Verlet updates, the cell list and the
// short-range pair forces.
#pragma once

#include "common.cuh"

namespace p3 {

// Velocity-Verlet half kick (Sec. 2; supporting information Sec. 1):
// v += (dt/2) F / m.  hdt_acc[i] = 0.5 dt ACCEL / m_i.
static __global__ void k_kick(int n, double* __restrict__ v, const double* __restrict__ F,
                       const double* __restrict__ hdt_acc) {
    pdl_wait();
    pdl_trigger();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double a = hdt_acc[i];
#pragma unroll
    for (int d = 0; d < 3; ++d) v[3 * i + d] += a * F[3 * i + d];
}

// Velocity rescaling to a target sum m v^2 (one block sum in mv2[0]).
static __global__ void k_rescale_v(int n, double* __restrict__ v, const double* __restrict__ mv2, double target) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 3 * n) return;
    const double cur = mv2[0];
    if (cur > 0.0) v[i] *= sqrt(target / cur);
}

__device__ __forceinline__ double wrap_pos(double x, double L) {
    x = x - L * floor(x / L);
    if (x < 0.0) x += L;
    if (x >= L) x = 0.0;
    return x;
}

// Half kick, drift r += dt v, and wrap into [0, L).
static __global__ void k_kick_drift(int n, double* __restrict__ r, double* __restrict__ v,
                             const double* __restrict__ F, const double* __restrict__ hdt_acc,
                             double dt, double L) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double a = hdt_acc[i];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const double vv = v[3 * i + d] + a * F[3 * i + d];
        v[3 * i + d] = vv;
        r[3 * i + d] = wrap_pos(r[3 * i + d] + dt * vv, L);
    }
}

// k_kick_drift followed by k_cell_count's work on the wrapped position: the
// particle's cell and the per-cell count of the multi-kernel cell list (the
// counts are zero on entry).
static __global__ void k_kick_drift_count(int n, double* __restrict__ r, double* __restrict__ v,
                                          const double* __restrict__ F, const double* __restrict__ hdt_acc,
                                          double dt, double L, double inv_cell, int nc, int* __restrict__ cell,
                                          int* __restrict__ count) {
    pdl_wait();
    pdl_trigger();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double a = hdt_acc[i];
    int cd[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const double vv = v[3 * i + d] + a * F[3 * i + d];
        v[3 * i + d] = vv;
        const double x = wrap_pos(r[3 * i + d] + dt * vv, L);
        r[3 * i + d] = x;
        cd[d] = min(max((int)floor(x * inv_cell), 0), nc - 1);
    }
    const int c = (cd[2] * nc + cd[1]) * nc + cd[0];
    cell[i] = c;
    atomicAdd(&count[c], 1);
}

static __global__ void k_wrap(int n, double* __restrict__ r, double L) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 3 * n) return;
    r[i] = wrap_pos(r[i], L);
}

// Wrap positions uploaded from the host and flag a non-finite position or
// velocity: *status (the solver's first-failure word) becomes `code` unless
// an earlier failure is recorded.
static __global__ void k_wrap_check(int n, double* __restrict__ r, const double* __restrict__ v, double L,
                                    int* __restrict__ status, int code) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 3 * n) return;
    const double x = r[i];
    if (!isfinite(x) || !isfinite(v[i])) atomicCAS(status, 0, code);
    r[i] = wrap_pos(x, L);
}

// ---------------------------------------------------------------- cell list
// Cell of each particle, c = min(floor(r * nc/L), nc-1) per axis, x fastest,
// and per-cell counts.
static __global__ void k_cell_count(int n, const double* __restrict__ r, double inv_cell, int nc,
                             int* __restrict__ cell, int* __restrict__ count) {
    pdl_wait();
    pdl_trigger();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    // clamped on both sides so that a non-finite position cannot index out of
    // bounds (wrapped positions always give 0 <= c < nc)
    const int cx = min(max((int)floor(r[3 * i + 0] * inv_cell), 0), nc - 1);
    const int cy = min(max((int)floor(r[3 * i + 1] * inv_cell), 0), nc - 1);
    const int cz = min(max((int)floor(r[3 * i + 2] * inv_cell), 0), nc - 1);
    const int c = (cz * nc + cy) * nc + cx;
    cell[i] = c;
    atomicAdd(&count[c], 1);
}

// Exclusive scan of m counts into start[0..m] with one block; also clears the
// per-cell fill counters.  The counts pass through shared memory in tiles of
// kScanTile: coalesced loads, kScanPer consecutive entries summed by each
// thread, a warp and a block scan of the thread sums, the exclusive values
// written back into the tile and stored coalesced, and the tile total
// carried into the next tile.  Tile index j sits at j + j/32 in shared
// memory, so both the coalesced and the per-thread accesses are free of bank
// conflicts.
constexpr int kScanThreads = 1024;
constexpr int kScanPer = 8;
constexpr int kScanTile = kScanThreads * kScanPer;

__device__ __forceinline__ int scan_slot(int j) { return j + (j >> 5); }

static __global__ void __launch_bounds__(kScanThreads) k_scan_cells(int m, const int* __restrict__ count,
                                                                  int* __restrict__ start, int* __restrict__ fill) {
    __shared__ int tile[kScanTile + kScanTile / 32];
    __shared__ int warp_tot[kScanThreads / 32];
    pdl_wait();
    pdl_trigger();
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    int carry = 0;
    for (int t0 = 0; t0 < m; t0 += kScanTile) {
        const int len = min(kScanTile, m - t0);
#pragma unroll
        for (int k = 0; k < kScanPer; ++k) {
            const int j = k * kScanThreads + tid;
            if (j < len) {
                tile[scan_slot(j)] = count[t0 + j];
                fill[t0 + j] = 0;
            }
        }
        __syncthreads();
        int v[kScanPer];
        int local = 0;
#pragma unroll
        for (int k = 0; k < kScanPer; ++k) {
            const int j = tid * kScanPer + k;
            v[k] = j < len ? tile[scan_slot(j)] : 0;
            local += v[k];
        }
        int w = local;  // inclusive warp scan of the thread sums
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane == 31) warp_tot[wid] = w;
        __syncthreads();
        if (wid == 0) {
            int x = warp_tot[lane];
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            warp_tot[lane] = x;  // inclusive over warps
        }
        __syncthreads();
        int run = carry + w - local + (wid > 0 ? warp_tot[wid - 1] : 0);
#pragma unroll
        for (int k = 0; k < kScanPer; ++k) {
            const int j = tid * kScanPer + k;
            if (j < len) tile[scan_slot(j)] = run;
            run += v[k];
        }
        carry += warp_tot[kScanThreads / 32 - 1];
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kScanPer; ++k) {
            const int j = k * kScanThreads + tid;
            if (j < len) start[t0 + j] = tile[scan_slot(j)];
        }
        __syncthreads();  // the next tile reuses tile and warp_tot
    }
    if (tid == 0) start[m] = carry;
}

static __global__ void k_cell_scatter(int n, const int* __restrict__ cell, const int* __restrict__ start,
                               int* __restrict__ fill, int* __restrict__ order) {
    pdl_wait();
    pdl_trigger();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = cell[i];
    order[start[c] + atomicAdd(&fill[c], 1)] = i;
}

// The whole cell list of a small system in one block (kCellBlockThreads
// threads, shared memory 2 ncell ints): cell index and counts (shared-memory
// atomics), exclusive scan, scatter, and the in-cell sort by particle index.
// The outputs (cell, start, order) are identical to those of k_cell_count,
// k_scan_cells, k_cell_scatter and k_cell_sort, in one launch instead of
// four; one SM walks the particles, so it pays only for small systems.
constexpr int kCellBlockThreads = 1024;

static __global__ void __launch_bounds__(kCellBlockThreads)
k_cells_block(int n, const double* __restrict__ r, double inv_cell, int nc, int ncell, int* __restrict__ cell,
              int* __restrict__ start, int* __restrict__ order) {
    extern __shared__ int cell_smem[];
    int* cnt = cell_smem;            // counts, then fill counters
    int* st = cell_smem + ncell;     // exclusive prefix
    __shared__ int wsum[kCellBlockThreads / 32];
    pdl_wait();
    pdl_trigger();
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int c = tid; c < ncell; c += nt) cnt[c] = 0;
    __syncthreads();
    for (int i = tid; i < n; i += nt) {
        const int cx = min(max((int)floor(r[3 * i + 0] * inv_cell), 0), nc - 1);
        const int cy = min(max((int)floor(r[3 * i + 1] * inv_cell), 0), nc - 1);
        const int cz = min(max((int)floor(r[3 * i + 2] * inv_cell), 0), nc - 1);
        const int c = (cz * nc + cy) * nc + cx;
        cell[i] = c;
        atomicAdd(&cnt[c], 1);
    }
    __syncthreads();
    // exclusive scan: each thread sums a contiguous chunk, the chunk sums are
    // scanned across the block, then each chunk is written out
    const int chunk = (ncell + nt - 1) / nt;
    const int beg = min(tid * chunk, ncell), end = min(beg + chunk, ncell);
    int local = 0;
    for (int c = beg; c < end; ++c) local += cnt[c];
    const int lane = tid & 31, wid = tid >> 5;
    int v = local;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    if (lane == 31) wsum[wid] = v;
    __syncthreads();
    if (wid == 0) {
        const int nw = nt >> 5;
        int w = lane < nw ? wsum[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < nw) wsum[lane] = w;
    }
    __syncthreads();
    int run = v - local + (wid > 0 ? wsum[wid - 1] : 0);
    for (int c = beg; c < end; ++c) {
        st[c] = run;
        start[c] = run;
        run += cnt[c];
        cnt[c] = 0;
    }
    if (tid == 0) start[ncell] = n;
    __syncthreads();
    for (int i = tid; i < n; i += nt) {
        const int c = cell[i];
        order[st[c] + atomicAdd(&cnt[c], 1)] = i;
    }
    __syncthreads();
    for (int c = tid; c < ncell; c += nt) {
        const int b = st[c], e = b + cnt[c];
        for (int j = b + 1; j < e; ++j) {
            const int key = order[j];
            int k = j - 1;
            while (k >= b && order[k] > key) {
                order[k + 1] = order[k];
                --k;
            }
            order[k + 1] = key;
        }
    }
}

// Gather particle data into cell order: xq = (x, y, z, Q), the cell-local
// coordinates x - c l (FP64 and FP32 copies) used by the pair kernel, and
// (if mp is given) the mesh coordinates of the FP32 assignment and
// interpolation on the nm^3 mesh.
// Slot s of the cell-ordered copies from particle i of cell c.
__device__ __forceinline__ void gather_slot(int s, int i, int c, const double* __restrict__ r,
                                            const double* __restrict__ Q, const int* __restrict__ type,
                                            const int* __restrict__ mol, int nc, double lcell,
                                            PQ* __restrict__ xq, PQ* __restrict__ xl64, float4* __restrict__ xl32,
                                            int* __restrict__ ts, int* __restrict__ ms, int* __restrict__ cs,
                                            MeshPt* __restrict__ mp, int nm, double inv_h) {
    const double x = r[3 * i], y = r[3 * i + 1], z = r[3 * i + 2], q = Q[i];
    xq[s] = PQ{x, y, z, q};
    const double lx = x - (c % nc) * lcell, ly = y - ((c / nc) % nc) * lcell, lz = z - (c / (nc * nc)) * lcell;
    xl64[s] = PQ{lx, ly, lz, q};
    xl32[s] = make_float4((float)lx, (float)ly, (float)lz, (float)q);
    ts[s] = type ? type[i] : 0;
    ms[s] = mol ? mol[i] : -1;
    cs[s] = c;
    if (mp) {
        MeshPt m;
        m.bx = mesh_axis(x, inv_h, nm, &m.tx);
        m.by = mesh_axis(y, inv_h, nm, &m.ty);
        m.bz = mesh_axis(z, inv_h, nm, &m.tz);
        m.q = (float)q;
        m.pad = 0.0f;
        mp[s] = m;
    }
}

static __global__ void k_gather_sorted(int n, const int* __restrict__ order, const double* __restrict__ r,
                                const double* __restrict__ Q, const int* __restrict__ type,
                                const int* __restrict__ mol, const int* __restrict__ cell, int nc,
                                double lcell, PQ* __restrict__ xq, PQ* __restrict__ xl64,
                                float4* __restrict__ xl32, int* __restrict__ ts, int* __restrict__ ms,
                                int* __restrict__ cs, MeshPt* __restrict__ mp, int nm, double inv_h) {
    pdl_wait();
    pdl_trigger();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int i = order[s];
    gather_slot(s, i, cell[i], r, Q, type, mol, nc, lcell, xq, xl64, xl32, ts, ms, cs, mp, nm, inv_h);
}

// Sort each cell's members by particle index so the order is deterministic,
// and clear the cell's count for the next build (the scan has consumed it).
// (Measured and not kept: the sort and the cell-ordered copies in one
// launch, a thread per cell writing its slots in sequence -- the cell-list
// stage of the 32768-ion step took 35 us instead of 23.)
static __global__ void k_cell_sort(int m, const int* __restrict__ start, int* __restrict__ order,
                                   int* __restrict__ count) {
    pdl_wait();
    pdl_trigger();
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= m) return;
    count[c] = 0;
    const int b = start[c], e = start[c + 1];
    for (int j = b + 1; j < e; ++j) {
        const int key = order[j];
        int k = j - 1;
        while (k >= b && order[k] > key) {
            order[k + 1] = order[k];
            --k;
        }
        order[k + 1] = key;
    }
}

// ---------------------------------------------------------------- pair forces
struct SRTable {
    int kind;      // 0 none, 1 BMH, 2 LJ
    int nt;
    double p[5][16];
    // shifted-force cutoff (P3MAZE_SR_SHIFT_FORCE): non-Coulomb U(r_c) and
    // F(r_c) = -U'(r_c) per species pair; erfc Coulomb g(r_c) = erfc(alpha r_c)/r_c
    // and G(r_c) = -g'(r_c) per unit QQ
    double urc[16], frc[16];
    double cg, cG, rc;
};

// Math in the pair kernel's arithmetic type, with the FP32 versions named
// explicitly (no silent promotion to the FP64 pipe).
__device__ __forceinline__ float m_exp(float x) { return __expf(x); }
__device__ __forceinline__ double m_exp(double x) { return exp(x); }
__device__ __forceinline__ float m_rsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double m_rsqrt(double x) { return rsqrt(x); }

// Pair parameters of one species pair in the arithmetic type: BMH A, 1/rho,
// s, C, D or LJ eps, sigma^2.
template <typename R>
struct PairPar {
    R a, b, c, d, e;
    R urc, frc;  // shifted-force constants of the non-Coulomb term
};

// Per-pair screened Coulomb (Eq. 19 with alpha = 1/(sqrt2 sigma); energy
// Eq. 5) and the non-Coulomb term.  Returns the Coulomb F/r without ke;
// energies are returned unscaled.
// erfc for the pair kernel.  FP32 (mixed mode): Abramowitz & Stegun 7.1.26,
// erfc(x) = t (a1 + t (a2 + t (a3 + t (a4 + t a5)))) exp(-x^2),
// t = 1/(1 + p x), |error| <= 1.5e-7 for x >= 0, which reuses the exp(-x^2)
// the force needs anyway.  FP64: the CUDA math library's erfc.
__device__ __forceinline__ float erfc_with_exp(float x, float ex) {
    const float t = __frcp_rn(fmaf(0.3275911f, x, 1.0f));
    const float poly = fmaf(fmaf(fmaf(fmaf(1.061405429f, t, -1.453152027f), t, 1.421413741f), t, -0.284496736f), t,
                            0.254829592f);
    return t * poly * ex;
}
__device__ __forceinline__ double erfc_with_exp(double x, double) { return erfc(x); }

// Shifted-force cutoff (SHIFT): each term U(r) becomes U(r) - U(r_c) + (r - r_c) F(r_c)
// and its force F(r) - F(r_c); sc = (g(r_c), G(r_c), r_c) of the Coulomb term per unit QQ.
template <typename R>
struct ShiftC {
    R cg, cG, rc;
};

template <int KIND, bool SHIFT, typename R>
__device__ __forceinline__ R pair_terms(R r2, R qq, R alpha, const PairPar<R>& pp, const ShiftC<R>& sc, R& ec,
                                        R& ev, R& fvdw) {
    const R ir = m_rsqrt(r2);
    const R rr = r2 * ir;
    const R ar = alpha * rr;
    const R ex = m_exp(-ar * ar);
    const R erfcv = erfc_with_exp(ar, ex);
    const R ir2 = ir * ir;
    ec = qq * erfcv * ir;
    ev = (R)0;
    fvdw = (R)0;
    if (KIND == 1) {
        const R eb = pp.a * m_exp((pp.c - rr) * pp.b);
        const R ir6 = ir2 * ir2 * ir2, ir8 = ir6 * ir2;
        ev = eb - pp.d * ir6 - pp.e * ir8;
        fvdw = (eb * pp.b - (R)6 * pp.d * ir6 * ir - (R)8 * pp.e * ir8 * ir) * ir;
    } else if (KIND == 2) {
        if (pp.a != (R)0) {
            const R sr2 = pp.b * ir2;
            const R sr6 = sr2 * sr2 * sr2;
            ev = (R)4 * pp.a * (sr6 * sr6 - sr6);
            fvdw = (R)24 * pp.a * ((R)2 * sr6 * sr6 - sr6) * ir2;
        }
    }
    R fc = qq * (erfcv * ir + (R)kTwoOverSqrtPi * alpha * ex) * ir2;
    if (SHIFT) {
        const R dr = rr - sc.rc;
        ec += qq * (dr * sc.cG - sc.cg);
        fc -= qq * sc.cG * ir;
        if (KIND != 0) {
            ev += dr * pp.frc - pp.urc;
            fvdw -= pp.frc * ir;
        }
    }
    return fc;
}

// Short-range forces (Eq. 19 plus the Born-Mayer or Lennard-Jones term) on
// the particles of a "home box" of 2x2x2 cells (edge l >= r_cut/2), one block
// per box.  The block stages every particle image of the surrounding region
// (home cells +-2 cells, up to 6x6x6 cells, periodic images explicit) in
// shared memory with coordinates in the box frame, x_loc + (u - u0) l for a
// particle of unwrapped cell u, so separations need no periodic shift and, in
// mixed mode, no FP64.  One warp per home particle scans 32 candidates at a
// time and compacts those inside the cutoff into a per-warp queue
// (__ballot_sync), so the pair functions run with every lane on a real pair.
// Pairs within one molecule closer than L/2 (the nearest image) are excluded.
// Each particle's force and half of its pair energies and of its pair virial
// (sum of r_ij . F_ij) are accumulated in the
// arithmetic type in shared memory (FP32 sums of FP32 pair terms in mixed
// mode) and written as FP64; no global atomics.  Regions larger than the staging
// buffer are processed in chunks, home lists longer than 256 in passes.
template <typename R> struct Vec4;
template <> struct Vec4<float> { using type = float4; };
template <> struct Vec4<double> { using type = PQ; };

template <int KIND, bool SHIFT, typename R, typename V>
__device__ __forceinline__ void pair_accumulate(const V& pi, const V& pj, R alpha, R ke, const PairPar<R>& pp,
                                                const ShiftC<R>& sc, R& fx, R& fy, R& fz, R& ec, R& ev, R& w) {
    const R ddx = (R)pi.x - (R)pj.x;
    const R ddy = (R)pi.y - (R)pj.y;
    const R ddz = (R)pi.z - (R)pj.z;
    const R r2 = ddx * ddx + ddy * ddy + ddz * ddz;
    R e_c, e_v, f_v;
    const R fr = pair_terms<KIND, SHIFT, R>(r2, (R)pi.w * (R)pj.w, alpha, pp, sc, e_c, e_v, f_v);
    const R f = ke * fr + f_v;
    fx += f * ddx;
    fy += f * ddy;
    fz += f * ddz;
    ec += e_c;
    ev += e_v;
    w += f * r2;  // r_ij . F_ij
}

// MOL: the system has molecules, so intramolecular pairs are tested for.
// SHIFT: shifted-force cutoff (pair_terms).
template <int KIND, typename R, int CAP, bool MOL, bool SHIFT>
__global__ void __launch_bounds__(P3_THREADS)
k_pair(int n, const typename Vec4<R>::type* __restrict__ xl, const int* __restrict__ ts,
       const int* __restrict__ ms, const int* __restrict__ start, int nc, int nbox, double lcell, double rc2,
       double halfL2, double alpha, double ke, SRTable tab, double* __restrict__ Fs,
       double* __restrict__ ecs, double* __restrict__ evs, double* __restrict__ wsr) {
    using V = typename Vec4<R>::type;
    constexpr int HCAP = 256;
    constexpr int NW = P3_THREADS / 32;
    __shared__ V sp[CAP];
    __shared__ int styp[CAP], smol[MOL ? CAP : 1];
    __shared__ int rstart[216], roff[217];
    __shared__ V hpos[HCAP];
    __shared__ unsigned hidx[HCAP];           // sorted index | home-cell offset bits 29..31
    __shared__ R hacc[HCAP][6];               // per home particle: force, Coulomb and non-Coulomb energy, virial
    __shared__ int wq[NW][64];
    // per warp: the home particle's candidates (FP32: an explicit list of
    // chunk indices; FP64, whose staging leaves no room: kept rows' start and
    // prefix, searched per candidate)
    constexpr bool kList = sizeof(R) == 4;
    __shared__ unsigned short wlist[kList ? NW : 1][kList ? CAP : 1];
    __shared__ int wbeg[NW][32], wpre[NW][32];
    __shared__ int s_nh, s_total;
    __shared__ PairPar<R> spar[16];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid < tab.nt * tab.nt) {
        PairPar<R> pp;
        if (KIND == 1) {
            pp.a = (R)tab.p[0][tid];
            pp.b = (R)(1.0 / tab.p[1][tid]);
            pp.c = (R)tab.p[2][tid];
            pp.d = (R)tab.p[3][tid];
            pp.e = (R)tab.p[4][tid];
        } else {
            pp.a = (R)tab.p[0][tid];
            pp.b = (R)(tab.p[1][tid] * tab.p[1][tid]);
            pp.c = pp.d = pp.e = (R)0;
        }
        pp.urc = (R)tab.urc[tid];
        pp.frc = (R)tab.frc[tid];
        spar[tid] = pp;
    }
    const ShiftC<R> sc{(R)tab.cg, (R)tab.cG, (R)tab.rc};
    // one home box per iteration; the grid may be smaller than the number
    // of boxes (a persistent launch that leaves room on every SM)
    const int nbox3 = nbox * nbox * nbox;
    for (int b = blockIdx.x; b < nbox3; b += gridDim.x) {
        __syncthreads();  // shared arrays of the previous box are no longer read
        const int bx = b % nbox, by = (b / nbox) % nbox, bz = b / (nbox * nbox);
        const int h0[3] = {2 * bx, 2 * by, 2 * bz};
        int hw[3];
        for (int d = 0; d < 3; ++d) hw[d] = min(2, nc - h0[d]);
        const int wx = hw[0] + 4, wy = hw[1] + 4, wz = hw[2] + 4;
        const int nreg = wx * wy * wz;
        const R lc = (R)lcell;
        // region cells: unwrapped u = h0 - 2 + r
        if (tid < nreg) {
            const int rx = tid % wx, ry = (tid / wx) % wy, rz = tid / (wx * wy);
            int u[3] = {h0[0] - 2 + rx, h0[1] - 2 + ry, h0[2] - 2 + rz};
            int c3[3];
            for (int d = 0; d < 3; ++d) {
                int c = u[d] % nc;
                if (c < 0) c += nc;
                c3[d] = c;
            }
            const int c = (c3[2] * nc + c3[1]) * nc + c3[0];
            rstart[tid] = start[c];
            roff[tid + 1] = start[c + 1] - start[c];
        }
        __syncthreads();
        if (tid == 0) {
            roff[0] = 0;
            for (int r = 0; r < nreg; ++r) roff[r + 1] += roff[r];
            s_total = roff[nreg];
            int nh = 0;
            for (int rz = 2; rz < 2 + hw[2]; ++rz)
                for (int ry = 2; ry < 2 + hw[1]; ++ry)
                    for (int rx = 2; rx < 2 + hw[0]; ++rx) {
                        const int r = (rz * wy + ry) * wx + rx;
                        nh += roff[r + 1] - roff[r];
                    }
            s_nh = nh;
        }
        __syncthreads();
        const int nh_all = s_nh, total = s_total;
        const R rc2r = (R)rc2, hl2r = (R)halfL2, alr = (R)alpha, ker = (R)ke;
        for (int hbase = 0; hbase < nh_all; hbase += HCAP) {
            const int nh = min(HCAP, nh_all - hbase);
            // home list of this pass: home cells in region order
            if (tid == 0) {
                int k = 0;
                for (int rz = 2; rz < 2 + hw[2]; ++rz)
                    for (int ry = 2; ry < 2 + hw[1]; ++ry)
                        for (int rx = 2; rx < 2 + hw[0]; ++rx) {
                            const int r = (rz * wy + ry) * wx + rx;
                            for (int t = rstart[r], e = rstart[r] + (roff[r + 1] - roff[r]); t < e; ++t, ++k)
                                if (k >= hbase && k < hbase + HCAP)
                                    hidx[k - hbase] = (unsigned)t | ((unsigned)(rx - 2) << 29) |
                                                      ((unsigned)(ry - 2) << 30) | ((unsigned)(rz - 2) << 31);
                        }
            }
            __syncthreads();
            for (int k = tid; k < nh; k += blockDim.x) {
                const unsigned code = hidx[k];
                const int t = (int)(code & 0x1fffffffu);
                const V p = xl[t];
                V q = p;
                q.x = (R)p.x + (R)((code >> 29) & 1u) * lc;
                q.y = (R)p.y + (R)((code >> 30) & 1u) * lc;
                q.z = (R)p.z + (R)((code >> 31) & 1u) * lc;
                hpos[k] = q;
                for (int a = 0; a < 6; ++a) hacc[k][a] = (R)0;
            }
            for (int c0 = 0; c0 < total; c0 += CAP) {
                const int cn = min(CAP, total - c0);
                __syncthreads();
                for (int k = tid; k < cn; k += blockDim.x) {
                    const int gk = c0 + k;
                    int lo = 0, hi = nreg - 1;  // region cell holding candidate gk
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (roff[mid] <= gk) lo = mid;
                        else hi = mid - 1;
                    }
                    const int r = lo;
                    const int t = rstart[r] + (gk - roff[r]);
                    const int rx = r % wx, ry = (r / wx) % wy, rz = r / (wx * wy);
                    const V p = xl[t];
                    V q = p;
                    q.x = (R)p.x + (R)(rx - 2) * lc;
                    q.y = (R)p.y + (R)(ry - 2) * lc;
                    q.z = (R)p.z + (R)(rz - 2) * lc;
                    sp[k] = q;
                    styp[k] = ts[t];
                    if (MOL) smol[k] = ms[t];
                }
                __syncthreads();
                for (int h = warp; h < nh; h += NW) {
                    const unsigned code = hidx[h];
                    const int hs = (int)(code & 0x1fffffffu);
                    const int hx = (int)((code >> 29) & 1u), hy = (int)((code >> 30) & 1u), hz = (int)((code >> 31) & 1u);
                    const V pi = hpos[h];
                    const int prow = ts[hs] * tab.nt;
                    const int mi = ms[hs];
                    R fx = 0, fy = 0, fz = 0, ec = 0, ev = 0, wv = 0;
                    // Candidate ranges of this home particle within the chunk:
                    // lane l < 25 takes the cell row (dy, dz) = (l % 5 - 2, l / 5 - 2)
                    // of its own 5x5x5 neighbourhood, drops it if its (y, z) gap
                    // reaches r_c and otherwise keeps the contiguous run of x
                    // cells that can come within r_c (conservatively rounded).
                    // Cell r of the region spans [(r - 2) l, (r - 1) l) in the
                    // coordinates of hpos and sp.
                    int beg = 0, len = 0;
                    if (lane < 25) {
                        const int ry = 2 + hy + lane % 5 - 2, rz = 2 + hz + lane / 5 - 2;
                        const R ylo = (R)(ry - 2) * lc, zlo = (R)(rz - 2) * lc;
                        const R gy = max((R)0, max(ylo - (R)pi.y, (R)pi.y - (ylo + lc)));
                        const R gz = max((R)0, max(zlo - (R)pi.z, (R)pi.z - (zlo + lc)));
                        const R room = rc2r * (R)1.00001 - (gy * gy + gz * gz);
                        if (room > (R)0) {
                            const R sx = sqrt(room) + (R)1e-4 * lc;
                            const int xlo = max(hx, (int)floor(((R)pi.x - sx) / lc) + 2);
                            const int xhi = min(hx + 4, (int)floor(((R)pi.x + sx) / lc) + 2);
                            if (xlo <= xhi) {
                                const int r0 = (rz * wy + ry) * wx;
                                const int a = max(roff[r0 + xlo], c0), e = min(roff[r0 + xhi + 1], c0 + cn);
                                if (e > a) {
                                    beg = a - c0;
                                    len = e - a;
                                }
                            }
                        }
                    }
                    const unsigned rm = __ballot_sync(0xffffffffu, len > 0);
                    int incl = len;
    #pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int t = __shfl_up_sync(0xffffffffu, incl, o);
                        if (lane >= o) incl += t;
                    }
                    const int tot = __shfl_sync(0xffffffffu, incl, 31);
                    if constexpr (kList) {
                        // expand the kept rows into this warp's candidate list
                        for (int t = 0; t < len; ++t) wlist[warp][incl - len + t] = (unsigned short)(beg + t);
                    } else if (len > 0) {
                        const int slot = __popc(rm & ((1u << lane) - 1u));
                        wbeg[warp][slot] = beg;
                        wpre[warp][slot] = incl - len;
                    }
                    const int nrow = __popc(rm);
                    __syncwarp();
                    int qn = 0;
                    for (int base = 0; base < tot; base += 32) {
                        const int g = base + lane;
                        bool hit = false;
                        int k = 0;
                        if (g < tot) {
                            if constexpr (kList) {
                                k = wlist[warp][g];
                            } else {
                                int lo = 0, hi = nrow - 1;  // last kept row starting at or before g
                                while (lo < hi) {
                                    const int mid = (lo + hi + 1) >> 1;
                                    if (wpre[warp][mid] <= g) lo = mid;
                                    else hi = mid - 1;
                                }
                                k = wbeg[warp][lo] + (g - wpre[warp][lo]);
                            }
                            // the home particle's own staged copy is formed by
                            // the same arithmetic as hpos, so its r2 is exactly
                            // 0; its periodic images are at least L away
                            const V pj = sp[k];
                            const R ddx = (R)pi.x - (R)pj.x;
                            const R ddy = (R)pi.y - (R)pj.y;
                            const R ddz = (R)pi.z - (R)pj.z;
                            const R r2 = ddx * ddx + ddy * ddy + ddz * ddz;
                            hit = r2 > (R)0 && r2 < rc2r;
                            if (MOL) hit = hit && !(mi >= 0 && smol[k] == mi && r2 < hl2r);
                        }
                        const unsigned m = __ballot_sync(0xffffffffu, hit);
                        if (hit) wq[warp][qn + __popc(m & ((1u << lane) - 1u))] = k;
                        qn += __popc(m);
                        __syncwarp();
                        if (qn >= 32) {
                            const int kk = wq[warp][lane];
                            pair_accumulate<KIND, SHIFT, R, V>(pi, sp[kk], alr, ker, spar[prow + styp[kk]], sc, fx, fy, fz, ec, ev,
                                                               wv);
                            __syncwarp();
                            if (lane < qn - 32) wq[warp][lane] = wq[warp][32 + lane];
                            __syncwarp();
                            qn -= 32;
                        }
                    }
                    if (lane < qn) {
                        const int kk = wq[warp][lane];
                        pair_accumulate<KIND, SHIFT, R, V>(pi, sp[kk], alr, ker, spar[prow + styp[kk]], sc, fx, fy, fz, ec, ev,
                                                               wv);
                    }
                    __syncwarp();
                    // lane partials (a few pairs each) are reduced and accumulated
                    // in the arithmetic type -- FP64 warp instructions are
                    // expensive on this part -- and converted to FP64 once
    #pragma unroll
                    for (int w = 16; w > 0; w >>= 1) {
                        fx += __shfl_xor_sync(0xffffffffu, fx, w);
                        fy += __shfl_xor_sync(0xffffffffu, fy, w);
                        fz += __shfl_xor_sync(0xffffffffu, fz, w);
                        ec += __shfl_xor_sync(0xffffffffu, ec, w);
                        ev += __shfl_xor_sync(0xffffffffu, ev, w);
                        wv += __shfl_xor_sync(0xffffffffu, wv, w);
                    }
                    if (lane == 0) {
                        hacc[h][0] += fx;
                        hacc[h][1] += fy;
                        hacc[h][2] += fz;
                        hacc[h][3] += ec;
                        hacc[h][4] += ev;
                        hacc[h][5] += wv;
                    }
                }
            }
            __syncthreads();
            for (int k = tid; k < nh; k += blockDim.x) {
                const int hs = (int)(hidx[k] & 0x1fffffffu);
                Fs[3 * hs + 0] = (double)hacc[k][0];
                Fs[3 * hs + 1] = (double)hacc[k][1];
                Fs[3 * hs + 2] = (double)hacc[k][2];
                ecs[hs] = 0.5 * ke * (double)hacc[k][3];
                evs[hs] = 0.5 * (double)hacc[k][4];
                wsr[hs] = 0.5 * (double)hacc[k][5];
            }
            __syncthreads();
        }
    }
}

// SPC/Fw intramolecular terms, one thread per (h1, o, h2) molecule: harmonic
// bonds and angle (Table S1) and the subtraction of the mesh part
// ke QQ erf(r/(sqrt2 sigma))/r of the three intramolecular pairs.  Adds into
// F (original order) and writes the bonded force and energies.
static __global__ void k_water(int nmol, const int* __restrict__ tri, const double* __restrict__ r,
                        const double* __restrict__ Q, double L, double alpha, double ke, double kb,
                        double r0, double ka, double th0, double* __restrict__ F,
                        double* __restrict__ Fb, double* __restrict__ eb, double* __restrict__ ex) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= nmol) return;
    const int id[3] = {tri[3 * m], tri[3 * m + 1], tri[3 * m + 2]};  // h1, o, h2
    double p[3][3], f[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int a = 0; a < 3; ++a)
        for (int d = 0; d < 3; ++d) p[a][d] = r[3 * id[a] + d];
    auto mic = [&](int a, int b, double* dv) {
        double r2 = 0.0;
        for (int d = 0; d < 3; ++d) {
            double x = p[a][d] - p[b][d];
            x -= L * rint(x / L);
            dv[d] = x;
            r2 += x * x;
        }
        return sqrt(r2);
    };
    double ebond = 0.0, eexc = 0.0;
    // bonds o-h1 and o-h2
    for (int hb = 0; hb < 3; hb += 2) {
        double dv[3];
        const double rr = mic(hb, 1, dv);
        ebond += 0.5 * kb * (rr - r0) * (rr - r0);
        const double g = -kb * (rr - r0) / rr;
        for (int d = 0; d < 3; ++d) {
            f[hb][d] += g * dv[d];
            f[1][d] -= g * dv[d];
        }
    }
    // angle h1-o-h2
    {
        double a[3], c[3];
        const double ra = mic(0, 1, a), rc = mic(2, 1, c);
        double ct = (a[0] * c[0] + a[1] * c[1] + a[2] * c[2]) / (ra * rc);
        ct = fmin(1.0, fmax(-1.0, ct));
        const double th = acos(ct);
        ebond += 0.5 * ka * (th - th0) * (th - th0);
        const double dE = ka * (th - th0);
        const double st = fmax(sqrt(1.0 - ct * ct), 1e-12);
        for (int d = 0; d < 3; ++d) {
            const double ga = -(c[d] / (ra * rc) - ct * a[d] / (ra * ra)) / st;
            const double gc = -(a[d] / (ra * rc) - ct * c[d] / (rc * rc)) / st;
            f[0][d] -= dE * ga;
            f[2][d] -= dE * gc;
            f[1][d] += dE * (ga + gc);
        }
    }
    // intramolecular exclusion of the mesh (erf) part
    const int pa[3] = {1, 1, 0}, pb[3] = {0, 2, 2};
    for (int k = 0; k < 3; ++k) {
        double dv[3];
        const double rr = mic(pa[k], pb[k], dv);
        const double qq = Q[id[pa[k]]] * Q[id[pb[k]]];
        const double u = alpha * rr;
        const double erfv = erf(u);
        eexc -= ke * qq * erfv / rr;
        const double fr = -ke * qq * (erfv / (rr * rr * rr) - kTwoOverSqrtPi * alpha * exp(-u * u) / (rr * rr));
        for (int d = 0; d < 3; ++d) {
            f[pa[k]][d] += fr * dv[d];
            f[pb[k]][d] -= fr * dv[d];
        }
    }
    for (int a = 0; a < 3; ++a)
        for (int d = 0; d < 3; ++d) {
            F[3 * id[a] + d] += f[a][d];
            Fb[3 * id[a] + d] = f[a][d];
        }
    eb[m] = ebond;
    ex[m] = eexc;
}

}  // namespace p3
